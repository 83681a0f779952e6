// Optional per-launch CUDA-event timing of the library's kernels
// (frac_profile_enable / frac_profile_read in include/frac.h).
#pragma once

#include "common.cuh"

namespace frac {
namespace prof {

bool enabled();
// Records a start event on construction and an end event on destruction, on
// stream `st`, under `name`, when profiling is enabled.
class Scope {
 public:
  Scope(const char* name, cudaStream_t st);
  ~Scope();
  Scope(const Scope&) = delete;
  Scope& operator=(const Scope&) = delete;

 private:
  int slot_ = -1;
  cudaStream_t st_ = nullptr;
};

}  // namespace prof
}  // namespace frac
