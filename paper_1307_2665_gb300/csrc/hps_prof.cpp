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

Scope::Scope(const char* name, cudaStream_t st, double flops, double bytes) : st_(st) {
  std::lock_guard<std::mutex> g(mu);
  ++n_launches;
  if (!on) return;
  Rec r;
  r.name = name;
  r.a = get_event();
  r.b = get_event();
  r.flops = flops;
  r.bytes = bytes;
  cudaEventRecord(r.a, st);
  pending.push_back(r);
  slot_ = (int)pending.size() - 1;
}

Scope::~Scope() {
  if (slot_ < 0) return;
  std::lock_guard<std::mutex> g(mu);
  if (slot_ < (int)pending.size()) cudaEventRecord(pending[slot_].b, st_);
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
}  // namespace hps
