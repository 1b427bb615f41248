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

// Bracket one launch: construct before the launch, destroy after it.
class Scope {
 public:
  Scope(const char* name, cudaStream_t st, double flops, double bytes);
  ~Scope();

 private:
  int slot_ = -1;
  cudaStream_t st_;
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
}  // namespace hps
