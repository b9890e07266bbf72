// pl_lookup.cuh -- launch wrapper of the cutoff-table lookup (host side).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pl {

constexpr int kLookupGridMax = 1024;  // grid exponents and sizes, each at most

// out[q * nq + j] = the table's quantile j at (qa[q], qn[q]), bilinear in
// (alpha, ln n) over the grid (galpha strictly increasing, 1 <= na <=
// kLookupGridMax; gn strictly increasing, 1 <= nn <= kLookupGridMax),
// clamped to its edges.  table: cell
// (alpha_i, n_k) at row i * nn + k, nq values per row.  All pointers device.
cudaError_t launch_lookup(const double *galpha, int na, const int64_t *gn, int nn, const double *table, int nq,
                          const double *qa, const int64_t *qn, int64_t nquery, double *out, cudaStream_t st);

}  // namespace pl
