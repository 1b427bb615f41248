#include "hps_prof.hpp"

#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace hps {
namespace prof {

namespace {

struct Rec {
  std::string name;
  cudaEvent_t a, b;
  double flops, bytes;
};

struct Agg {
  int64_t launches = 0;
  double ms = 0, flops = 0, bytes = 0;
};

std::mutex mu;
bool on = false;
int64_t n_launches = 0;
std::vector<Rec> pending;
std::vector<cudaEvent_t> pool;
std::map<std::string, Agg> agg;
std::vector<std::string> names_out;

cudaEvent_t get_event() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void resolve_locked() {
  for (auto& r : pending) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    Agg& g = agg[r.name];
    g.launches += 1;
    g.ms += ms;
    g.flops += r.flops;
    g.bytes += r.bytes;
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  pending.clear();
}

}  // namespace

bool enabled() { return on; }

void set_enabled(bool v) {
  std::lock_guard<std::mutex> g(mu);
  on = v;
}

void reset() {
  std::lock_guard<std::mutex> g(mu);
  resolve_locked();
  agg.clear();
  n_launches = 0;
}

int64_t launches() {
  std::lock_guard<std::mutex> g(mu);
  return n_launches;
}

Scope::Scope(const char* name, cudaStream_t st, double flops, double bytes)
    : name_(name), st_(st), flops_(flops), bytes_(bytes) {
  std::lock_guard<std::mutex> g(mu);
  ++n_launches;
  if (!on) return;
  a_ = get_event();
  b_ = get_event();
  cudaEventRecord(a_, st);
}

Scope::~Scope() {
  if (!a_) return;
  cudaEventRecord(b_, st_);
  std::lock_guard<std::mutex> g(mu);
  Rec r;
  r.name = name_;
  r.a = a_;
  r.b = b_;
  r.flops = flops_;
  r.bytes = bytes_;
  pending.push_back(r);
}

int read(Stat* out, int max_out) {
  std::lock_guard<std::mutex> g(mu);
  resolve_locked();
  names_out.clear();
  for (auto& kv : agg) names_out.push_back(kv.first);
  int n = 0;
  for (auto& kv : agg) {
    if (n >= max_out) break;
    out[n].name = names_out[n].c_str();
    out[n].launches = kv.second.launches;
    out[n].ms = kv.second.ms;
    out[n].flops = kv.second.flops;
    out[n].bytes = kv.second.bytes;
    ++n;
  }
  return (int)agg.size();
}

}  // namespace prof

bool opt_in_smem(const void* kernel, int bytes) {
  static std::mutex m;
  static std::map<std::pair<const void*, int>, bool> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> g(m);
  auto key = std::make_pair(kernel, dev);
  auto it = done.find(key);
  if (it != done.end()) return it->second;
  const bool ok =
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
  done[key] = ok;
  return ok;
}

}  // namespace hps
