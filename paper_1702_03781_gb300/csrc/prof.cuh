// prof.cuh -- optional per-kernel-class device timing (instrumentation).
//
// When enabled by harp_profile_begin, launch sites of the selected classes
// record a CUDA event pair on their own stream around the launch and add
// the launch's algorithmic flop count; harp_profile_end synchronises, sums
// the elapsed times and disables recording.
#pragma once

#include "common.cuh"

namespace harp {

struct ProfScope {
  int kind;
  double flops;
  cudaStream_t st;
  int slot;  // -1 when not recording
  ProfScope(int kind, double flops, cudaStream_t st);
  ~ProfScope();
};

}  // namespace harp
