// pl_probe.cuh -- launch of the issue-rate probe kernels (pl_probe.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pl {

enum { kProbeMulWide = 0, kProbeLop3 = 1, kProbeDfma = 2, kProbePhilox = 3 };
constexpr int kProbeBlock = 1024;  // one block per SM
constexpr int kProbeChains = 8;  // independent chains per thread (ops per loop iteration)

// One probe kernel on grid x kProbeBlock threads, iters loop iterations per
// thread; out: uint32[grid * kProbeBlock]; cyc: the largest block's clock64
// cycles (zeroed on the stream first).
cudaError_t launch_probe(int kind, uint32_t *out, long long *cyc, int grid, int iters, uint32_t seed,
                         cudaStream_t st);

}  // namespace pl
