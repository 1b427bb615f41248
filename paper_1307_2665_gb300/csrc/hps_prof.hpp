// Launch accounting of libhps: every kernel launch is counted; when profiling
// is on, each launch is bracketed by CUDA events on its own stream and charged
// with the algorithmic flops and bytes its caller states, per kernel name.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace hps {
namespace prof {

bool enabled();
void set_enabled(bool on);
void reset();
int64_t launches();

// Bracket one launch: construct before the launch, destroy after it.  Each
// scope owns its pair of events, so scopes on different threads and streams do
// not interfere.
class Scope {
 public:
  Scope(const char* name, cudaStream_t st, double flops, double bytes);
  ~Scope();
  Scope(const Scope&) = delete;
  Scope& operator=(const Scope&) = delete;

 private:
  const char* name_;
  cudaStream_t st_;
  double flops_, bytes_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};

struct Stat {
  const char* name;
  int64_t launches;
  double ms;
  double flops;
  double bytes;
};
// Resolve all recorded events (synchronises the device) and return per-name sums.
int read(Stat* out, int max_out);

}  // namespace prof

// Raise a kernel's dynamic shared-memory limit to `bytes` once per (kernel,
// device), thread-safe; false if the device refused (the launch then fails and
// the caller's launch check reports it).  Only the first call per (kernel,
// device) sets the limit: every caller passes the kernel's largest size.
bool opt_in_smem(const void* kernel, int bytes);

}  // namespace hps
