// pl_multinomial.cu -- the multinomial histogram sampler (a large-n variant of
// the sampler; not in the paper): a replicate's histogram drawn by conditional
// binomials on a binary tree of its first kMnBins values, the few values
// beyond one by one, written as a block-form replicate record that the
// finisher fits and tests as usual.
//
// Law: the inverse-CDF sampler's, through its integer thresholds T (with
// T[-1] = 2^53 + 1 the index range [l, r) has mass (T[l-1] - T[r-1]) 2^-53).
// The count beyond the tree is Bin(n, (T[B-1] - 1) 2^-53), B = kMnBins; node 1
// (range [0, B)) holds the rest, and node k of range [l, r) passes
// Bin(c_k, (T[l-1] - T[mid-1]) / (T[l-1] - T[r-1])) of its count to its left
// child 2k ([l, mid)) and the others to 2k+1; leaves B..2B-1 are the values
// xmin .. xmin + B - 1.  The values beyond are the inverse CDF of m' uniform
// on [1, T[B-1] - 1] (the multiply-high of a 64-bit random word).  Random
// words: draw index 0 for the count beyond, k for node k, 2B + t for the t-th
// value beyond.
//
// One warp per replicate: the binomials of a tree level are independent, so
// the lanes take a level's nodes together; the work grows with the occupied
// values, not with n.
#include <cmath>

#include "pl_multinomial.cuh"

namespace pl {
namespace {

constexpr int kMnBins = 2048;  // values in the binomial tree
constexpr int kMnWarps = 4;     // replicates per block

// ln k! minus Stirling's formula: the asymptotic series (Bernoulli numbers)
// above 15, the sum of logs below.
__device__ double mn_stirling_err(double k) {
  if (k > 15.0) {
    const double r = 1.0 / (k * k);
    return (1.0 / 12.0 - r * (1.0 / 360.0 - r * (1.0 / 1260.0 - r * (1.0 / 1680.0 - r / 1188.0)))) / k;
  }
  double lf = 0.0;
  for (int i = 2; i <= (int)k; ++i) lf += log((double)i);
  return lf - ((k + 0.5) * log(k) - k + 0.918938533204672741780329736406);
}

// x ln(x/M) + M - x, by its series in v = (x - M)/(x + M) near x = M
// (|v| < 0.1: the terms fall by 100 per step, so 9 of them reach 2^-53).
__device__ double mn_deviance(double x, double M) {
  if (fabs(x - M) < 0.1 * (x + M)) {
    const double v = (x - M) / (x + M), v2 = v * v;
    double s = (x - M) * v, e = 2.0 * x * v;
#pragma unroll
    for (int j = 1; j <= 9; ++j) {
      e *= v2;
      s += e * (1.0 / (double)(2 * j + 1));
    }
    return s;
  }
  return x * log(x / M) + M - x;
}

// 1 / x for x >= 1 (an integer-valued count): the binary32 reciprocal refined
// by two binary64 Newton steps (relative error below 1 ulp).
__device__ __forceinline__ double mn_rcp(double x) {
  double r = (double)__frcp_rn((float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  return fma(r, fma(-x, r, 1.0), r);
}

// P(Bin(n, p) = x) (q = 1 - p passed separately), saddle-point form
// (Loader 2000) inside, powers at the ends.
__device__ double mn_binom_pmf(int64_t x, int64_t n, double p, double q) {
  if (x < 0 || x > n) return 0.0;
  if (x == 0) return exp((double)n * (p < 0.5 ? log1p(-p) : log(q)));
  if (x == n) return exp((double)n * (q < 0.5 ? log1p(-q) : log(p)));
  const double dn = (double)n, dx = (double)x, dy = (double)(n - x);
  const double lc = mn_stirling_err(dn) - mn_stirling_err(dx) - mn_stirling_err(dy) - mn_deviance(dx, dn * p) -
                    mn_deviance(dy, dn * q);
  return exp(lc) * sqrt(dn / (6.283185307179586476925286766559 * dx * dy));
}

// Bin(n, p), p = num / den (integers, num <= den), from one uniform u by
// inversion along a fixed order of the outcomes: 0, 1, 2, ... for a mean
// below 30, else from M = floor((n+1) p) (the mode to within a part in 2^24
// of p) outward, M+1, M-1, M+2, ... (one side alone once the other is
// exhausted or has underflowed).  The branch and M come from integer
// arithmetic on num and den cut to their top 24 bits: the thresholds behind
// them may differ from another implementation's in their last units, and p is
// often an exact ratio for which (n+1) p is an integer.
__device__ int64_t mn_binomial(int64_t n, uint64_t num, uint64_t den, double u) {
  if (n <= 0 || num == 0) return 0;
  if (num >= den) return n;
  const double p = (double)num / (double)den, q = (double)(den - num) / (double)den;
  const double r = p / q;
  const int bits = 64 - __clzll((long long)den);
  const int sh = bits > 24 ? bits - 24 : 0;
  const uint64_t nc = num >> sh, dc = den >> sh;
  if ((uint64_t)n * nc < 30ull * dc) {
    double f;
    if (n <= 64) {  // q^n by squaring (a few ulps) for the many small counts
      double b = q;
      f = 1.0;
      for (int64_t e = n; e > 0; e >>= 1) {
        if (e & 1) f *= b;
        b *= b;
      }
    } else {
      f = mn_binom_pmf(0, n, p, q);
    }
    double c = f;
    int64_t k = 0;
    while (c < u && k < n) {
      f *= (double)(n - k) * mn_rcp((double)(k + 1)) * r;
      ++k;
      c += f;
      if (f == 0.0 && (double)k > (double)n * p) break;
    }
    return k;
  }
  int64_t M = (int64_t)(((uint64_t)(n + 1) * nc) / dc);
  if (M > n) M = n;
  const double fM = mn_binom_pmf(M, n, p, q);
  double rest = u - fM;
  if (rest <= 0.0) return M;
  int64_t lo = M - 1, hi = M + 1, last = M;
  const double ir = q / p;
  double flo = lo >= 0 ? fM * (double)M * mn_rcp((double)(n - M + 1)) * ir : 0.0;
  double fhi = hi <= n ? fM * (double)(n - M) * mn_rcp((double)(M + 1)) * r : 0.0;
  bool up = true;
  while (flo > 0.0 || fhi > 0.0) {
    if (up ? fhi > 0.0 : !(flo > 0.0)) {
      rest -= fhi;
      last = hi;
      if (rest <= 0.0) return hi;
      fhi = hi < n ? fhi * (double)(n - hi) * mn_rcp((double)(hi + 1)) * r : 0.0;
      ++hi;
    } else {
      rest -= flo;
      last = lo;
      if (rest <= 0.0) return lo;
      flo = lo > 0 ? flo * (double)lo * mn_rcp((double)(n - lo + 1)) * ir : 0.0;
      --lo;
    }
    up = !up;
  }
  return last;
}

__device__ __forceinline__ uint64_t mn_word(uint64_t i, uint32_t rep, uint32_t cell, uint32_t purpose,
                                            const RoundKeys &rk) {
  const uint4 w = philox4x32_10_rk(make_uint4((uint32_t)(i >> 1), rep, cell, purpose), rk);
  return (i & 1) ? ((uint64_t)w.w << 32) | w.z : ((uint64_t)w.y << 32) | w.x;
}

__device__ __forceinline__ uint64_t mn_tm1(const uint64_t *T, uint32_t i) {
  return i == 0 ? (1ull << 53) + 1 : T[i - 1];
}

// One warp per replicate.  The tree's level L (nodes 2^L .. 2^(L+1) - 1) is
// split by the lanes in parallel; internal counts wait in the record's dense
// area above kMnScratch (cleared later where the finisher reads it), the
// leaves are the dense counts of the first kMnBins values.
constexpr uint32_t kMnScratch = 4096;
static_assert(kMnScratch + kMnBins <= kHWide, "tree scratch inside the dense record");

__global__ void __launch_bounds__(kMnWarps * 32) mn_sample_kernel(MnLaunch a) {
  const uint64_t wid = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const uint64_t it = wid / kWideReps, j = wid % kWideReps;
  if (it >= a.nitems) return;  // warp-uniform
  const WorkItem wi = a.items[it];
  if (j >= wi.nrep) return;
  const Cell &cell = a.cells[wi.cell];
  const Law &law = a.laws[cell.law];
  const uint32_t H = cell.H, L2 = law.L2;
  const int64_t n = cell.n;
  const uint32_t rep = wi.r0 + (uint32_t)j;
  uint32_t *dense = reinterpret_cast<uint32_t *>(a.rec.dense + wi.dense_off + j * 2 * (uint64_t)H);
  uint64_t *spill = a.rec.spill + wi.spill_off + j * (uint64_t)cell.scap;
  const uint64_t *T = law.T;
  // the count beyond the tree, then the tree level by level
  const uint64_t TB = T[kMnBins - 1];
  int64_t beyond = 0;
  if (lane == 0) {
    const uint64_t m = (mn_word(0, rep, cell.cell_id, cell.purpose, a.rk) >> 11) + 1;
    beyond = mn_binomial(n, TB - 1, 1ull << 53, (double)m * 0x1p-53);
    dense[kMnScratch + 1] = (uint32_t)(n - beyond);
  }
  beyond = __shfl_sync(0xffffffffu, beyond, 0);
  __syncwarp();
  uint32_t last = 0;  // 1 + the largest leaf with a count (this lane's)
  for (uint32_t level = 0, first = 1; first < (uint32_t)kMnBins; ++level, first <<= 1) {
    const uint32_t width = (uint32_t)kMnBins >> level;
    for (uint32_t k = first + lane; k < 2 * first; k += 32) {
      const int64_t c = dense[kMnScratch + k];
      int64_t cl = 0;
      const uint32_t l = (k - first) * width, r = l + width, mid = l + width / 2;
      if (c > 0) {
        const uint64_t A = mn_tm1(T, l), Bm = mn_tm1(T, mid), E = mn_tm1(T, r);
        if (A > E) {
          const uint64_t m = (mn_word(k, rep, cell.cell_id, cell.purpose, a.rk) >> 11) + 1;
          cl = mn_binomial(c, A - Bm, A - E, (double)m * 0x1p-53);
        }
      }
      if (2 * first < (uint32_t)kMnBins) {
        dense[kMnScratch + 2 * k] = (uint32_t)cl;
        dense[kMnScratch + 2 * k + 1] = (uint32_t)(c - cl);
      } else {  // the children are leaves: values l and l + 1
        dense[l] = (uint32_t)cl;
        dense[l + 1] = (uint32_t)(c - cl);
        if (c - cl > 0) last = l + 2;
        else if (cl > 0) last = l + 1;
      }
    }
    __syncwarp();
  }
  int64_t tmax = (int64_t)__reduce_max_sync(0xffffffffu, last) - 1;
  // the values beyond the tree, conditional on X >= xmin + kMnBins: first the
  // largest histogram index they reach (to clear the bins up to it), then counted
  const uint64_t span = TB - 1;
  auto draw = [&](int64_t t, uint64_t &mp) {
    mp = __umul64hi(mn_word(2 * (uint64_t)kMnBins + (uint64_t)t, rep, cell.cell_id, cell.purpose, a.rk), span) + 1;
    return lookup_index(T, law.guide, T, L2, law.xmin_f, law.tail_c, law.tail_e, mp);
  };
  uint32_t top = 0;
  for (int64_t t = lane; t < beyond; t += 32) {
    uint64_t mp;
    const uint32_t i = draw(t, mp);
    if (i < H && i + 1 > top) top = i + 1;
  }
  top = __reduce_max_sync(0xffffffffu, top);
  for (uint32_t i = kMnBins + lane; i < top; i += 32) dense[i] = 0u;
  __syncwarp();
  uint32_t ns = 0;
  for (int64_t t0 = 0; t0 < beyond; t0 += 32) {
    const int64_t t = t0 + lane;
    uint64_t v = 0;
    bool sp = false;
    if (t < beyond) {
      uint64_t mp;
      const uint32_t i = draw(t, mp);
      if (i < H) {
        atomicAdd(&dense[i], 1u);
      } else {
        sp = true;
        v = i < L2 ? cell.xmin + i : tail_invert(cell.alpha, law.Z, cell.xmin + L2, mp);
      }
    }
    const unsigned b = __ballot_sync(0xffffffffu, sp);
    const uint32_t slot = ns + __popc(b & ((1u << lane) - 1u));
    if (sp && slot < cell.scap) spill[slot] = v;
    ns += __popc(b);
  }
  if (top > 0) tmax = max(tmax, (int64_t)top - 1);
  if (lane == 0) {
    if (ns > cell.scap) atomicOr(&a.ctr->status, kErrArena);  // the finisher must not redraw
    a.rec.meta[wi.meta_off + j] = make_int2((int)tmax, (int)ns);
  }
}

}  // namespace

cudaError_t launch_mn_sample(const MnLaunch &a, cudaStream_t st) {
  const uint64_t warps = (uint64_t)a.nitems * kWideReps;
  if (warps == 0) return cudaSuccess;
  mn_sample_kernel<<<(unsigned)((warps + kMnWarps - 1) / kMnWarps), kMnWarps * 32, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace pl
