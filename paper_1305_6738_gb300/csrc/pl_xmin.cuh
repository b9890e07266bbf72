// pl_xmin.cuh -- launch wrapper of the x_min estimation (host side).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pl_device.cuh"

namespace pl {

struct XminOut {
  uint64_t xmin;
  double alpha_hat;
  double D;
  int64_t n_tail;
  int64_t candidates;
  int64_t best;
};

constexpr int kXHistBins = 8192;  // values counted in the shared histogram

// x: device int32[n] (values >= 1; a smaller one latches the data error).
// Scratch: ghist (kXHistBins uint32), nspill (1), spill (a power of two >= n,
// uint64), vals/cnts/Lt (n entries), S (n + 1), d (1).  Per-candidate outputs
// c_* have max_cand entries; out receives the choice.
cudaError_t launch_xmin(const int32_t *x, int64_t n, uint32_t *ghist, unsigned long long *nspill, uint64_t *spill,
                        uint64_t *vals, uint32_t *cnts, int64_t *S, double *Lt, int64_t *d, int64_t max_cand,
                        int64_t min_tail, uint64_t *c_xmin, double *c_alpha, double *c_D, int64_t *c_nt,
                        XminOut *out, Counters *ctr, int num_sms, cudaStream_t st);

}  // namespace pl
