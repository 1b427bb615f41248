// Serving loop over the solver: continuous batching of builds and solves.
//
// State is guarded by one mutex.  Worker threads pick jobs under it and run
// them outside it:
//   build  one hps_build_batch call of one problem; the handle gets its own
//          CUDA stream (options.stream = NULL), so work on different operators
//          overlaps on the device;
//   solve  the pending solves of one resident, idle operator, oldest first, up
//          to max_rhs_per_solve right-hand sides, as one hps_solve_ex call on
//          device buffers; each request's result is its slice of the call's u.
// Admission: a job starts only when its device memory (build: the estimated
// peak; solve: workspace plus result) fits in the budget next to what is
// already charged (resident operators, running jobs, results not released).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/hps_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

enum { kBuild = 0, kSolve = 1 };
enum OpState { kPending, kBuilding, kReady, kFailed, kEvicted };

// Device memory of one solve call's u, shared by the requests it served.
struct Result {
  void* p = nullptr;
  int64_t bytes = 0;
  int holders = 0;  // requests not yet released that share it (guarded by the server mutex)
  cudaStream_t free_stream = nullptr;
  ~Result() {
    if (p) cudaFreeAsync(p, free_stream);
  }
};

struct Request {
  int64_t id = 0, op = -1;
  int kind = kBuild;
  hps_problem prob{};
  hps_options opt{};
  std::vector<double> coef[6];
  std::vector<double> f;
  int nrhs = 0;
  int status = 1;
  double t_submit = 0, t_start = 0, t_end = 0;
  int batch_rhs = 0, iterations = 0;
  int64_t device_bytes = 0;
  int64_t est_peak = 0;
  std::shared_ptr<Result> res;
  int64_t res_off = 0;  // doubles
};

struct Operator {
  int64_t id = 0;
  OpState state = kPending;
  int status = 1;
  hps_handle h = nullptr;
  int64_t dof = 0, nbnd = 0;
  int64_t resident = 0;      // bytes charged while resident
  int64_t work_per_rhs = 0;  // solve workspace estimate per right-hand side
  bool busy = false;
  int queued = 0;            // solves waiting in the queue
  bool release_requested = false;
  double last_use = 0;
};

struct Job {
  int kind = kBuild;
  int64_t op = -1;
  std::vector<Request*> reqs;
  int64_t reserve = 0;
};

}  // namespace

struct hps_server_s {
  hps_server_options opt{};
  cudaMemPool_t pool = nullptr;
  cudaStream_t free_stream = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  std::deque<int64_t> queue;
  std::map<int64_t, Operator> ops;
  int64_t next_id = 0;
  int64_t used = 0, peak = 0;
  int running = 0;
  bool stopping = false;
  std::vector<std::thread> workers;
  Clock::time_point t0;
  hps_server_stats st{};

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  void charge(int64_t b) {
    used += b;
    peak = std::max(peak, used);
  }
};

namespace {

void complete(hps_server_s& S, Request& r, int status) {
  r.status = status;
  r.t_end = S.now();
  S.st.completed += 1;
  if (status != HPS_OK) S.st.failed += 1;
}

void evict(hps_server_s& S, Operator& o) {
  if (o.h) hps_free(o.h);
  o.h = nullptr;
  if (o.state == kReady) {
    S.used -= o.resident;
    S.st.resident_ops -= 1;
  }
  o.state = kEvicted;
  o.status = HPS_ENOMEM;
  S.st.evicted_ops += 1;
}

// Evict idle operators, least recently used first, until `need` more bytes fit.
bool make_room(hps_server_s& S, int64_t need, int64_t keep_op) {
  while (S.used + need > S.opt.hbm_budget) {
    Operator* victim = nullptr;
    for (auto& kv : S.ops) {
      Operator& o = kv.second;
      if (o.state != kReady || o.busy || o.queued > 0 || o.id == keep_op) continue;
      if (!victim || o.last_use < victim->last_use) victim = &o;
    }
    if (!victim) return false;
    evict(S, *victim);
  }
  return true;
}

// Choose the next job (mutex held).  Fails queued solves whose operator is gone.
bool pick(hps_server_s& S, Job& job) {
  bool build_blocked = false;
  for (size_t qi = 0; qi < S.queue.size();) {
    Request& r = *S.reqs.at(S.queue[qi]);
    if (r.kind == kBuild) {
      if (build_blocked) {
        ++qi;
        continue;
      }
      if (S.used + r.est_peak > S.opt.hbm_budget && !make_room(S, r.est_peak, -1)) {
        build_blocked = true;  // later builds wait: arrival order among builds
        ++qi;
        continue;
      }
      S.queue.erase(S.queue.begin() + qi);
      S.ops.at(r.op).state = kBuilding;
      job.kind = kBuild;
      job.op = r.op;
      job.reqs = {&r};
      job.reserve = r.est_peak;
      S.charge(job.reserve);
      return true;
    }
    Operator& o = S.ops.at(r.op);
    if (o.state == kFailed || o.state == kEvicted) {
      o.queued -= 1;
      complete(S, r, o.status);
      S.queue.erase(S.queue.begin() + qi);
      S.cv_done.notify_all();
      continue;
    }
    if (o.state != kReady || o.busy) {
      ++qi;
      continue;
    }
    // coalesce this operator's queued solves, oldest first
    std::vector<size_t> idx;
    int total = 0;
    for (size_t k = qi; k < S.queue.size(); ++k) {
      Request& x = *S.reqs.at(S.queue[k]);
      if (x.kind != kSolve || x.op != r.op) continue;
      if (!idx.empty() && total + x.nrhs > S.opt.max_rhs_per_solve) break;
      idx.push_back(k);
      total += x.nrhs;
    }
    auto need = [&](int n) { return (int64_t)n * (o.work_per_rhs + o.dof * 8 + o.nbnd * 8); };
    while (idx.size() > 1 && S.used + need(total) > S.opt.hbm_budget) {
      total -= S.reqs.at(S.queue[idx.back()])->nrhs;
      idx.pop_back();
    }
    if (idx.size() == 1 && o.resident + need(total) > S.opt.hbm_budget) {
      // too large even with everything else evicted and released: it can never start
      o.queued -= 1;
      complete(S, r, HPS_ENOMEM);
      S.queue.erase(S.queue.begin() + qi);
      S.cv_done.notify_all();
      continue;
    }
    if (S.used + need(total) > S.opt.hbm_budget && !make_room(S, need(total), o.id)) {
      ++qi;
      continue;
    }
    job.kind = kSolve;
    job.op = o.id;
    job.reqs.clear();
    for (size_t k : idx) job.reqs.push_back(S.reqs.at(S.queue[k]).get());
    for (size_t t = idx.size(); t-- > 0;) S.queue.erase(S.queue.begin() + idx[t]);
    o.busy = true;
    o.queued -= (int)idx.size();
    job.reserve = need(total);
    S.charge(job.reserve);
    return true;
  }
  return false;
}

void run_build(hps_server_s& S, Job& job) {
  Request& r = *job.reqs[0];
  hps_problem P = r.prob;
  const double** slots[6] = {&P.c11, &P.c12, &P.c22, &P.c1, &P.c2, &P.c};
  for (int k = 0; k < 6; ++k) *slots[k] = r.coef[k].empty() ? nullptr : r.coef[k].data();
  hps_options o = r.opt;
  o.device_ptrs = 0;
  o.stream = nullptr;  // the handle's own stream
  hps_handle h = nullptr;
  int st = hps_build_batch(&P, 1, &o, &h);
  int64_t bytes = 0;
  if (st == HPS_OK) hps_query(h, nullptr, nullptr, nullptr, nullptr, &bytes);
  for (auto& c : r.coef) std::vector<double>().swap(c);
  std::lock_guard<std::mutex> g(S.mu);
  S.used -= job.reserve;
  Operator& op = S.ops.at(r.op);
  if (st == HPS_OK) {
    op.h = h;
    op.state = kReady;
    op.resident = bytes;
    op.status = HPS_OK;
    op.last_use = S.now();
    S.charge(bytes);
    S.st.resident_ops += 1;
  } else {
    op.state = kFailed;
    op.status = st;
  }
  r.device_bytes = bytes;
  S.st.builds += 1;
  complete(S, r, st);
}

void run_solve(hps_server_s& S, Job& job, cudaStream_t ws) {
  Operator* op;
  {
    std::lock_guard<std::mutex> g(S.mu);
    op = &S.ops.at(job.op);  // std::map nodes are stable
  }
  int total = 0;
  for (Request* r : job.reqs) total += r->nrhs;
  std::vector<double> fcat((size_t)total * op->nbnd);
  size_t off = 0;
  for (Request* r : job.reqs) {
    std::memcpy(fcat.data() + off, r->f.data(), r->f.size() * sizeof(double));
    off += r->f.size();
  }
  auto res = std::make_shared<Result>();
  res->free_stream = S.free_stream;
  res->bytes = (int64_t)total * op->dof * 8;
  void* fd = nullptr;
  int st = HPS_OK;
  hps_solve_info info{};
  if (cudaMallocFromPoolAsync(&fd, fcat.size() * sizeof(double), S.pool, ws) != cudaSuccess ||
      cudaMallocFromPoolAsync(&res->p, (size_t)res->bytes, S.pool, ws) != cudaSuccess) {
    st = HPS_ENOMEM;
  } else if (cudaMemcpyAsync(fd, fcat.data(), fcat.size() * sizeof(double), cudaMemcpyHostToDevice,
                             ws) != cudaSuccess ||
             cudaStreamSynchronize(ws) != cudaSuccess) {
    st = HPS_EDEVICE;
  } else {
    st = hps_solve_ex(op->h, static_cast<const double*>(fd), total, static_cast<double*>(res->p),
                      1, &info);
    hps_release_workspace(op->h);
  }
  if (fd) cudaFreeAsync(fd, ws);
  cudaGetLastError();
  std::lock_guard<std::mutex> g(S.mu);
  S.used -= job.reserve;
  if (st == HPS_OK || st == HPS_ENOTCONVERGED) S.charge(res->bytes);
  else res.reset();
  int64_t r0 = 0;
  for (Request* r : job.reqs) {
    r->batch_rhs = total;
    r->iterations = info.iterations;
    if (res) {
      r->res = res;
      r->res_off = r0 * op->dof;
      res->holders += 1;
    }
    r0 += r->nrhs;
    std::vector<double>().swap(r->f);
    complete(S, *r, st);
    S.st.solves += 1;
    S.st.rhs_solved += r->nrhs;
  }
  S.st.solve_calls += 1;
  op->busy = false;
  op->last_use = S.now();
  if (op->release_requested && op->queued == 0 && op->state == kReady) evict(S, *op);
}

void worker_main(hps_server_s* S) {
  cudaSetDevice(S->opt.device);
  cudaStream_t ws = nullptr;
  cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking);
  for (;;) {
    Job job;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (pick(*S, job)) break;
        if (S->stopping && S->running == 0) {
          // nothing can start and nothing runs that would free memory: the
          // queued requests can never run
          for (int64_t id : S->queue) {
            Request& r = *S->reqs.at(id);
            if (r.kind == kSolve) S->ops.at(r.op).queued -= 1;
            complete(*S, r, HPS_ENOMEM);
          }
          S->queue.clear();
          S->cv_done.notify_all();
          S->cv_work.notify_all();
          cudaStreamDestroy(ws);
          return;
        }
        S->cv_work.wait(lk);
      }
      S->running += 1;
      const double t = S->now();
      for (Request* r : job.reqs) r->t_start = t;
    }
    if (job.kind == kBuild)
      run_build(*S, job);
    else
      run_solve(*S, job, ws);
    {
      std::lock_guard<std::mutex> g(S->mu);
      S->running -= 1;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

int64_t submit(hps_server_s& S, std::unique_ptr<Request> r) {
  std::lock_guard<std::mutex> g(S.mu);
  if (S.stopping) return HPS_EINVAL;
  const int64_t id = S.next_id++;
  r->id = id;
  if (r->kind == kBuild) r->op = id;
  r->t_submit = S.now();
  if (r->kind == kBuild) {
    Operator& o = S.ops[id];
    o.id = id;
    o.dof = (int64_t)r->prob.nx * r->prob.ny * r->prob.p * r->prob.p;
    o.nbnd = hps_boundary_count(r->prob.nx, r->prob.ny, r->prob.q);
  } else {
    S.ops.at(r->op).queued += 1;
  }
  S.queue.push_back(id);
  S.reqs[id] = std::move(r);
  S.st.submitted += 1;
  S.cv_work.notify_one();
  return id;
}

}  // namespace

extern "C" {

void hps_server_default_options(hps_server_options* opt) {
  if (!opt) return;
  opt->hbm_budget = 0;
  opt->workers = 4;
  opt->max_rhs_per_solve = 256;
  opt->device = 0;
}

int hps_server_create(const hps_server_options* opt_in, hps_server* out) {
  if (!out) return HPS_EINVAL;
  *out = nullptr;
  hps_server_options opt;
  hps_server_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.workers < 1 || opt.workers > 64 || opt.max_rhs_per_solve < 1 || opt.hbm_budget < 0)
    return HPS_EINVAL;
  if (cudaSetDevice(opt.device) != cudaSuccess) {
    cudaGetLastError();
    return HPS_EDEVICE;
  }
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return HPS_EDEVICE;
  }
  if (opt.hbm_budget == 0) opt.hbm_budget = (int64_t)(0.9 * (double)free_b);
  auto* S = new hps_server_s();
  S->opt = opt;
  S->t0 = Clock::now();
  S->st.budget = opt.hbm_budget;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = opt.device;
  uint64_t thr = UINT64_MAX;
  if (cudaMemPoolCreate(&S->pool, &props) != cudaSuccess ||
      cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &thr) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->free_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return HPS_EDEVICE;
  }
  for (int i = 0; i < opt.workers; ++i) S->workers.emplace_back(worker_main, S);
  *out = S;
  return HPS_OK;
}

int hps_server_destroy(hps_server S) {
  if (!S) return HPS_OK;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  cudaSetDevice(S->opt.device);
  S->reqs.clear();  // results free on the free stream
  for (auto& kv : S->ops)
    if (kv.second.h) hps_free(kv.second.h);
  cudaStreamSynchronize(S->free_stream);
  cudaStreamDestroy(S->free_stream);
  cudaMemPoolDestroy(S->pool);
  delete S;
  return HPS_OK;
}

int64_t hps_server_submit_build(hps_server S, const hps_problem* prob, const hps_options* opt) {
  if (!S || !prob) return HPS_EINVAL;
  auto r = std::make_unique<Request>();
  r->kind = kBuild;
  r->prob = *prob;
  hps_default_options(&r->opt);
  if (opt) r->opt = *opt;
  int64_t peak = 0, resident = 0, work = 0;
  const int est = hps_estimate_bytes(prob, 1, &r->opt, 1, &peak, &resident, &work);
  if (est != HPS_OK) return est;
  if (peak > S->opt.hbm_budget) return HPS_ENOMEM;  // could never start
  r->est_peak = peak;
  const int64_t n = (int64_t)prob->nx * prob->ny * prob->p * prob->p;
  const double* c[6] = {prob->c11, prob->c12, prob->c22, prob->c1, prob->c2, prob->c};
  for (int k = 0; k < 6; ++k)
    if (c[k]) r->coef[k].assign(c[k], c[k] + n);
  const int64_t id = submit(*S, std::move(r));
  if (id >= 0) {
    std::lock_guard<std::mutex> g(S->mu);
    S->ops.at(id).work_per_rhs = work;
  }
  return id;
}

int64_t hps_server_submit_solve(hps_server S, int64_t op, const double* f, int nrhs) {
  if (!S || !f || nrhs < 1) return HPS_EINVAL;
  int64_t nbnd = 0;
  {
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->ops.find(op);
    if (it == S->ops.end()) return HPS_EINVAL;
    nbnd = it->second.nbnd;
  }
  auto r = std::make_unique<Request>();
  r->kind = kSolve;
  r->op = op;
  r->nrhs = nrhs;
  r->f.assign(f, f + (size_t)nrhs * nbnd);
  return submit(*S, std::move(r));
}

int hps_server_wait(hps_server S, int64_t req, double timeout_s, hps_request_info* info) {
  if (!S) return HPS_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(req);
  if (it == S->reqs.end()) return HPS_EINVAL;
  Request& r = *it->second;
  auto done = [&] { return r.status != 1; };
  if (timeout_s < 0)
    S->cv_done.wait(lk, done);
  else
    S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done);
  if (info) {
    info->status = r.status;
    info->kind = r.kind;
    info->op = r.op;
    info->nrhs = r.nrhs;
    info->batch_rhs = r.batch_rhs;
    info->iterations = r.iterations;
    info->t_submit = r.t_submit;
    info->t_start = r.t_start;
    info->t_end = r.t_end;
    info->device_bytes = r.device_bytes;
  }
  return r.status;
}

int hps_server_result(hps_server S, int64_t req, double* u) {
  if (!S || !u) return HPS_EINVAL;
  std::shared_ptr<Result> res;
  int64_t off = 0, n = 0;
  {
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(req);
    if (it == S->reqs.end() || it->second->kind != kSolve || !it->second->res) return HPS_EINVAL;
    Request& r = *it->second;
    res = r.res;
    off = r.res_off;
    n = (int64_t)r.nrhs * S->ops.at(r.op).dof;
  }
  cudaSetDevice(S->opt.device);
  if (cudaMemcpy(u, static_cast<double*>(res->p) + off, (size_t)n * sizeof(double),
                 cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return HPS_EDEVICE;
  }
  return HPS_OK;
}

int hps_server_release(hps_server S, int64_t req) {
  if (!S) return HPS_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->reqs.find(req);
  if (it == S->reqs.end() || it->second->status == 1) return HPS_EINVAL;
  auto& res = it->second->res;
  if (res && --res->holders == 0) S->used -= res->bytes;
  S->reqs.erase(it);
  S->cv_work.notify_all();
  return HPS_OK;
}

int hps_server_release_operator(hps_server S, int64_t op) {
  if (!S) return HPS_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->ops.find(op);
  if (it == S->ops.end()) return HPS_EINVAL;
  Operator& o = it->second;
  o.release_requested = true;
  if (o.state == kReady && !o.busy && o.queued == 0) evict(*S, o);
  S->cv_work.notify_all();
  return HPS_OK;
}

int hps_server_get_stats(hps_server S, hps_server_stats* out) {
  if (!S || !out) return HPS_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  *out = S->st;
  out->bytes_in_use = S->used;
  out->peak_bytes_in_use = S->peak;
  return HPS_OK;
}

}  // extern "C"
