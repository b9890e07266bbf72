// pl_lookup.cu -- cutoffs at a fitted exponent from a tabulated grid.
//
// The paper's tables give cutoffs on a grid of exponents and sample sizes and
// advise using them with a close value of the fitted exponent (Section 3).
// Here the value at (alpha-hat, n) is bilinear in (alpha, ln n) between the
// four surrounding grid cells, clamped to the grid's edges; at a grid point
// it is that cell's value exactly.
#include <cstdint>
#include <cuda_runtime.h>

#include "pl_lookup.cuh"

namespace pl {
namespace {

// Largest i in [0, m - 2] with g[i] <= v (0 when m == 1), and the weight of
// cell i + 1 in [0, 1] (exactly 0 or 1 at a grid point).
__device__ __forceinline__ int bracket(const double *g, int m, double v, double &w) {
  if (m == 1) {
    w = 0.0;
    return 0;
  }
  int lo = 0, hi = m - 2;  // answer in [lo, hi]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g[mid] <= v)
      lo = mid;
    else
      hi = mid - 1;
  }
  const double t = (v - g[lo]) / (g[lo + 1] - g[lo]);
  w = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
  return lo;
}

// One thread per query: the grid's exponents and ln n (computed here, with
// the same log as the queries, so that a query at a grid size sits exactly on
// it) are staged in shared memory.
__global__ void __launch_bounds__(256) lookup_kernel(const double *galpha, int na, const int64_t *gn, int nn,
                                                     const double *table, int nq, const double *qa,
                                                     const int64_t *qn, int64_t nquery, double *out) {
  __shared__ double sa[kLookupGridMax], sl[kLookupGridMax];
  for (int k = threadIdx.x; k < na; k += blockDim.x) sa[k] = galpha[k];
  for (int k = threadIdx.x; k < nn; k += blockDim.x) sl[k] = log((double)gn[k]);
  __syncthreads();
  const int64_t qi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (qi >= nquery) return;
  double wa, wn;
  const int ia = bracket(sa, na, qa[qi], wa);
  const int in = bracket(sl, nn, log((double)qn[qi]), wn);
  const int ia1 = na > 1 ? ia + 1 : ia, in1 = nn > 1 ? in + 1 : in;
  const double *r00 = table + ((int64_t)ia * nn + in) * nq, *r10 = table + ((int64_t)ia1 * nn + in) * nq;
  const double *r01 = table + ((int64_t)ia * nn + in1) * nq, *r11 = table + ((int64_t)ia1 * nn + in1) * nq;
  for (int j = 0; j < nq; ++j)
    out[qi * nq + j] = (1.0 - wa) * ((1.0 - wn) * r00[j] + wn * r01[j]) + wa * ((1.0 - wn) * r10[j] + wn * r11[j]);
}

}  // namespace

cudaError_t launch_lookup(const double *galpha, int na, const int64_t *gn, int nn, const double *table, int nq,
                          const double *qa, const int64_t *qn, int64_t nquery, double *out, cudaStream_t st) {
  if (nquery == 0) return cudaSuccess;
  lookup_kernel<<<(unsigned)((nquery + 255) / 256), 256, 0, st>>>(galpha, na, gn, nn, table, nq, qa, qn, nquery,
                                                                 out);
  return cudaGetLastError();
}

}  // namespace pl
