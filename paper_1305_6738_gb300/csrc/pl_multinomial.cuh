// pl_multinomial.cuh -- launch wrapper of the multinomial histogram sampler
// (host side).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pl_kernels.cuh"

namespace pl {

constexpr uint32_t kWideReps = 8;  // replicates per block-form work item

// One wave of block-form work items (kWideReps replicates each): every
// replicate's record (dense counts, spills, meta) written for the finisher.
struct MnLaunch {
  const Cell *cells;
  const Law *laws;
  const WorkItem *items;
  uint32_t nitems;
  RoundKeys rk;
  Records rec;
  Counters *ctr;
};
cudaError_t launch_mn_sample(const MnLaunch &a, cudaStream_t st);

}  // namespace pl
