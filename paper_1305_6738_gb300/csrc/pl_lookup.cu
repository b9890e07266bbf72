// pl_lookup.cu -- cutoffs at a fitted exponent from a tabulated grid.
//
// The paper's tables give cutoffs on a grid of exponents and sample sizes and
// advise using them with a close value of the fitted exponent (Section 3).
// Here the value at (alpha-hat, n) is bilinear in (alpha, ln n) between the
// four surrounding grid cells, clamped to the grid's edges; at a grid point
// it is that cell's value exactly.  One thread per (query, quantile).
#include <cstdint>
#include <cuda_runtime.h>

#include "pl_lookup.cuh"

namespace pl {
namespace {

// Largest i in [0, m - 2] with g(i) <= v (0 when m == 1), and the weight of
// cell i + 1 in [0, 1].
template <class G>
__device__ __forceinline__ int bracket(G g, int m, double v, double &w) {
  if (m == 1) {
    w = 0.0;
    return 0;
  }
  int lo = 0, hi = m - 2;  // answer in [lo, hi]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g(mid) <= v)
      lo = mid;
    else
      hi = mid - 1;
  }
  const double a = g(lo), b = g(lo + 1);
  double t = (v - a) / (b - a);
  w = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
  return lo;
}

__global__ void lookup_kernel(const double *galpha, int na, const int64_t *gn, int nn, const double *table, int nq,
                              const double *qa, const int64_t *qn, int64_t nquery, double *out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nquery * nq) return;
  const int64_t qi = i / nq;
  const int j = (int)(i - qi * nq);
  double wa, wn;
  const int ia = bracket([&](int k) { return galpha[k]; }, na, qa[qi], wa);
  const int in = bracket([&](int k) { return log((double)gn[k]); }, nn, log((double)qn[qi]), wn);
  const int ia1 = na > 1 ? ia + 1 : ia, in1 = nn > 1 ? in + 1 : in;
  const double v00 = table[((int64_t)ia * nn + in) * nq + j], v10 = table[((int64_t)ia1 * nn + in) * nq + j];
  const double v01 = table[((int64_t)ia * nn + in1) * nq + j], v11 = table[((int64_t)ia1 * nn + in1) * nq + j];
  out[i] = (1.0 - wa) * ((1.0 - wn) * v00 + wn * v01) + wa * ((1.0 - wn) * v10 + wn * v11);
}

}  // namespace

cudaError_t launch_lookup(const double *galpha, int na, const int64_t *gn, int nn, const double *table, int nq,
                          const double *qa, const int64_t *qn, int64_t nquery, double *out, cudaStream_t st) {
  const int64_t total = nquery * nq;
  if (total == 0) return cudaSuccess;
  lookup_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(galpha, na, gn, nn, table, nq, qa, qn, nquery, out);
  return cudaGetLastError();
}

}  // namespace pl
