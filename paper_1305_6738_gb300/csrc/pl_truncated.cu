// pl_truncated.cu -- sm_103a kernels of the truncated law on 1..K
// (p(k) = k^-gamma / zeta_K(gamma), the cutoffs of Tables 2-6).
//
// Set-up: thresholds of the inverse CDF from finite suffix sums (block scan),
// ln k tables, and the fit nodes: Taylor coefficients of zeta_K around
// gamma_j = -64 + j/32, so that the MLE of Eq. 2 needs no per-replicate sum
// over the support.  Replicates: one warp per replicate draws n values from
// Philox streams through the thresholds staged in shared memory, counts them
// in a shared-memory histogram of the K support points, takes the log-sum,
// solves Eq. 2 by Newton on the node polynomial and computes D (Eq. 3) in one
// pass over the support.
#include <algorithm>
#include <cmath>

#include "pl_truncated.cuh"

namespace pl {
namespace {

constexpr double kLn2 = 0.69314718055994530942;

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ uint32_t warp_scan_u32(uint32_t x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}
__device__ __forceinline__ uint64_t warp_scan_max_u64(uint64_t x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o && y > x) x = y;
  }
  return x;
}

// ---------------------------------------------------------------------------
// ln k, its float split, and the float split of ln(k / K) = -log1p((K - k) / k)
// (exact to the last bit near k = K, where ln k - ln K would cancel).
__global__ void tz_log_kernel(const TzTable *tables) {
  const TzTable t = tables[blockIdx.y];
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > t.K) return;
  double l = 0.0, q = 0.0;
  if (k > 0) {
    l = log((double)k);
    q = -log1p((double)(t.K - k) / (double)k);
  }
  t.lnk[k] = l;
  const float lh = (float)l, qh = (float)q;
  t.lnk_hi[k] = lh;
  t.lnk_lo[k] = (float)(l - (double)lh);
  t.lnq_hi[k] = qh;
  t.lnq_lo[k] = (float)(q - (double)qh);
}

// Fit nodes, one warp per node gamma_j: a_r = sum_k (-ln k)^r k^-gamma_j / r!,
// r < kTzTerms (all terms of one a_r share a sign), stored as a_0 and
// b_r = a_r / a_0; E_j = -b_1 (the mean of ln X) and V_j = 2 b_2 - b_1^2 (its
// variance).
__global__ void __launch_bounds__(256) tz_node_kernel(const TzTable *tables) {
  const TzTable &t = tables[blockIdx.y];
  const int j = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (j >= kTzNodes) return;
  const double g = kTzGammaLo + (double)j / kTzNodeInv;
  double a[kTzTerms];
#pragma unroll
  for (int r = 0; r < kTzTerms; ++r) a[r] = 0.0;
  for (uint32_t k = 1 + lane; k <= t.K; k += 32) {
    const double u = -t.lnk[k];
    double w = pow((double)k, -g);
#pragma unroll
    for (int r = 0; r < kTzTerms; ++r) {
      a[r] += w;
      w *= u * (1.0 / (double)(r + 1));
    }
  }
#pragma unroll
  for (int r = 0; r < kTzTerms; ++r) a[r] = warp_sum(a[r]);
  if (lane == 0) {
    double *nd = t.node + (size_t)j * kTzNodeStride;
    const double inv = 1.0 / a[0];
    nd[0] = a[0];
#pragma unroll
    for (int r = 1; r < kTzTerms; ++r) nd[r] = a[r] * inv;
    const double E = -nd[1];
    nd[kTzE] = E;
    nd[kTzV] = 2.0 * nd[2] - E * E;
    nd[kTzInvA0] = inv;
    t.E[j] = E;
  }
}

// The Hermite start terms of each node interval (after every node is built).
__global__ void tz_node_interval_kernel(const TzTable *tables) {
  const TzTable &t = tables[blockIdx.y];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kTzNodes) return;
  double *nd = t.node + (size_t)j * kTzNodeStride;
  if (j == kTzNodes - 1) {
    nd[kTzInvDE] = nd[kTzS0] = nd[kTzS1] = 0.0;
    return;
  }
  const double dE = nd[kTzE] - nd[kTzNodeStride + kTzE];
  nd[kTzInvDE] = 1.0 / dE;
  nd[kTzS0] = dE / nd[kTzV];
  nd[kTzS1] = dE / nd[kTzNodeStride + kTzV];
}

// Thresholds of one law, one block of 1024 threads: thread i holds the term
// of k = K - i, so an inclusive scan gives the suffix sums
// S(K - 1 - i) = sum_{j > K-1-i} j^-gamma; Q(k) = S(k) / S(0).  A max-scan
// keeps T non-increasing in k whatever the rounding of the scan.  Then the
// guide by binary search on the staged thresholds.
__global__ void __launch_bounds__(1024) tz_law_kernel(const TzLaw *laws) {
  const TzLaw L = laws[blockIdx.x];
  __shared__ double s_sum[32];
  __shared__ uint64_t s_max[32];
  __shared__ double s_Z;
  __shared__ uint64_t sT[kTzKMax + 1];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t K = L.K;
  const double v = tid < (int)K ? pow((double)(K - tid), -L.gamma) : 0.0;
  const double incl = warp_scan(v, lane);
  if (lane == 31) s_sum[wid] = incl;
  __syncthreads();
  if (wid == 0) s_sum[lane] = warp_scan(s_sum[lane], lane);
  __syncthreads();
  const double S = incl + (wid ? s_sum[wid - 1] : 0.0);
  if (tid == (int)K - 1) s_Z = S;
  __syncthreads();
  // T in thread order (k = K - 1 - tid decreasing): non-decreasing in tid
  uint64_t T = 0;
  if (tid < (int)K - 1) {
    T = (uint64_t)floor(S / s_Z * 9007199254740992.0) + 1ull;
  } else if (tid == (int)K - 1) {
    T = (1ull << 53) + 1ull;  // Q(0) = 1
  }
  T = warp_scan_max_u64(T, lane);
  if (lane == 31) s_max[wid] = T;
  __syncthreads();
  if (wid == 0) s_max[lane] = warp_scan_max_u64(s_max[lane], lane);
  __syncthreads();
  if (wid && s_max[wid - 1] > T) T = s_max[wid - 1];
  if (tid < (int)K) sT[K - 1 - tid] = T;
  if (tid == 0) sT[K] = 1ull;  // Q(K) = 0
  __syncthreads();
  for (int i = tid; i <= (int)K; i += blockDim.x) L.T[i] = sT[i];
  for (int jb = tid; jb < kTzGuide; jb += blockDim.x) {
    const uint64_t bound = (uint64_t)(jb + 1) << (53 - kTzGuideBits);
    uint32_t lo = 1, hi = K;  // answer in [lo, hi]: T[K] = 1 <= bound
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (sT[mid] <= bound)
        hi = mid;
      else
        lo = mid + 1;
    }
    L.guide[jb] = (uint16_t)lo;
  }
}

// X = min{k in 1..K : T[k] <= m}: from the guide's answer for the largest m
// of the bucket, step up while the threshold is above m (T[K] = 1 ends it).
__device__ __forceinline__ uint32_t tz_lookup(const uint64_t *T, const uint16_t *G, uint64_t m) {
  uint32_t k = G[(m - 1) >> (53 - kTzGuideBits)];
  while (T[k] > m) ++k;
  return k;
}

// X of a draw known by its high word h: the answer at m_first(h), or, when
// the threshold above that answer lies inside the draw's interval of m
// (T[X - 1] <= m_last(h)), the answer at m itself (m_full(), the low word's
// block).  T[0] = 2^53 + 1 exceeds every m.
template <class MFull>
__device__ __forceinline__ uint32_t tz_lookup_hi(const uint64_t *T, const uint16_t *G, uint32_t h, MFull m_full) {
  const uint32_t k = tz_lookup(T, G, m_first(h));
  if (T[k - 1] > m_last(h)) return k;
  return tz_lookup(T, G, m_full());
}

// Sampling only: one thread per draw, m taken whole (both words).
__global__ void tz_sample_kernel(const TzLaw *law, RoundKeys rk, uint32_t cell_id, uint32_t purpose,
                                 uint32_t rep0, uint64_t nrep, uint64_t n, uint64_t *out) {
  const uint64_t total = nrep * n;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t r = i / n, d = i - r * n;
    const uint4 wh = philox4x32_10_rk(make_uint4((uint32_t)(d >> 2), rep0 + (uint32_t)r, cell_id, purpose), rk);
    const uint4 wl =
        philox4x32_10_rk(make_uint4((uint32_t)(d >> 2), rep0 + (uint32_t)r, cell_id, purpose | kLowStream), rk);
    const uint32_t j = (uint32_t)d & 3u;
    out[i] = tz_lookup(law->T, law->guide, draw_m(quad_word(wh, j), quad_word(wl, j)));
  }
}

// ---------------------------------------------------------------------------
// Replicates.

// Count one value: support points 1..4 in per-lane packed 16-bit registers
// (no shared-memory conflicts on the heavy head of the law), the others by
// shared-memory atomics on packed 16-bit bins (bin k in half k & 1 of word
// k >> 1).  Per-lane counts stay below 2^12, totals below 2^16.
__device__ __forceinline__ void tz_count(uint32_t k, uint32_t *h, uint32_t &c12, uint32_t &c34) {
  c12 += (k == 1u ? 1u : 0u) + (k == 2u ? 0x10000u : 0u);
  c34 += (k == 3u ? 1u : 0u) + (k == 4u ? 0x10000u : 0u);
  if (k > 4u) atomicAdd(&h[k >> 1], (k & 1u) ? 0x10000u : 1u);
}

__device__ __forceinline__ uint32_t tz_bin(const uint32_t *h, uint32_t k) {
  return (h[k >> 1] >> ((k & 1u) << 4)) & 0xffffu;
}

// The normalised scaling factor P(delta) = zeta_K(gamma_j + delta) / a_0 and
// its first two derivatives from node j's polynomial (Horner with
// derivatives; b_0 = 1).
__device__ __forceinline__ void tz_poly(const double *nd, double d, double &p, double &dp, double &ddp) {
  p = nd[kTzTerms - 1];
  dp = 0.0;
  ddp = 0.0;
#pragma unroll
  for (int r = kTzTerms - 2; r >= 1; --r) {
    ddp = fma(ddp, d, dp);
    dp = fma(dp, d, p);
    p = fma(p, d, nd[r]);
  }
  ddp = fma(ddp, d, dp);
  dp = fma(dp, d, p);
  p = fma(p, d, 1.0);
  ddp *= 2.0;
}

// 1 / x for x in [2^-8, 2^8]: the binary32 reciprocal refined by two
// binary64 Newton steps (relative error 1e-7 -> 1e-14 -> below 1 ulp).
__device__ __forceinline__ double tz_rcp(double x) {
  double r = (double)__frcp_rn((float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  return fma(r, fma(-x, r, 1.0), r);
}

// MLE (Eq. 2 with the finite scaling factor): the root of
// E_gamma[ln X] = mbar, E decreasing in gamma.  Every lane of the warp runs
// the same steps.  The node bracket E_j >= mbar > E_{j+1} is found by a
// 32-way search (three rounds of ballots over the node means), the start by
// cubic Hermite interpolation of gamma(E) between the two nodes (its
// interpolation error is of order 1e-8 or below), and the root by Newton on
// the node polynomial with the slope -Var[ln X] rounded to binary32,
// safeguarded by bisection on [gamma_j, gamma_j + 1/32].  A Newton step
// below 2^-27 max(|gamma|, 1) is the last: the error left after it is below
// the square of the step plus 1e-7 of it, under 1e-15.  Means at or beyond the
// ends of [-64, 64] give the end, and so does a sample of only K (all_top:
// an integer test, since the equation then has no finite root and E is flat
// to the last bit near -64 for small K).  Returns the number of polynomial
// evaluations (kTzNewtonCap + 1 if the cap was hit); *Z = zeta_K(gamma-hat),
// *invZ its reciprocal.
__device__ __forceinline__ int tz_fit(const TzTable &tb, double mbar, bool all_top, int lane, double &g_out,
                                      double &Z, double &invZ) {
  const double *E = tb.E;
  if (all_top || !(mbar < E[0])) {
    g_out = kTzGammaLo;
    Z = tb.node[0];
    invZ = tb.node[kTzInvA0];
    return 0;
  }
  if (!(mbar > E[kTzNodes - 1])) {
    const double *nd = tb.node + (size_t)(kTzNodes - 1) * kTzNodeStride;
    g_out = kTzGammaHi;
    Z = nd[0];
    invZ = nd[kTzInvA0];
    return 0;
  }
  uint32_t base = 0;
  {
    const bool ge = E[base + lane * 128] >= mbar;
    base += (__popc(__ballot_sync(0xffffffffu, ge)) - 1) * 128;
  }
  {
    const bool ge = E[base + lane * 4] >= mbar;
    base += (__popc(__ballot_sync(0xffffffffu, ge)) - 1) * 4;
  }
  {
    const bool ge = lane < 4 && E[base + lane] >= mbar;
    base += __popc(__ballot_sync(0xffffffffu, ge)) - 1;
  }
  const uint32_t j = base;
  const double h = 1.0 / kTzNodeInv;
  const double gj = kTzGammaLo + (double)j * h;
  const double *nd = tb.node + (size_t)j * kTzNodeStride;
  const double t = (nd[kTzE] - mbar) * nd[kTzInvDE];
  const double t2 = t * t, t3 = t2 * t;
  double d = (t3 - 2.0 * t2 + t) * nd[kTzS0] + (3.0 * t2 - 2.0 * t3) * h + (t3 - t2) * nd[kTzS1];
  if (!(d >= 0.0 && d <= h)) d = t * h;
  const double scale = fmax(fabs(gj), 1.0);
  const double small = 0x1p-27 * scale;
  const double tol = 4.0 * 0x1p-52 * scale;
  double lo = 0.0, hi = h, zr = 1.0, izr = 1.0;
  int it = 1;
  for (; it <= kTzNewtonCap; ++it) {
    double p, dp, ddp;
    tz_poly(nd, d, p, dp, ddp);
    const double iz = tz_rcp(p);
    const double e = -dp * iz;
    const double var = fma(ddp, iz, -e * e);
    const double f = e - mbar;
    if (f > 0.0)
      lo = d;
    else
      hi = d;
    double nx = d + f * (double)__frcp_rn((float)var);
    const bool newton = nx >= lo && nx <= hi;  // f = 0 gives a zero step
    if (!newton) nx = 0.5 * (lo + hi);
    const double step = nx - d;
    d = nx;
    // P and 1/P at the new point to second order in the step (the error left,
    // of order E^3 step^3, is below 1e-16 for a final step)
    zr = fma(fma(0.5 * ddp, step, dp), step, p);
    const double u = (zr - p) * iz;
    izr = iz * fma(u, u, 1.0 - u);
    if ((newton && fabs(step) <= small) || hi - lo <= tol) break;
  }
  g_out = gj + d;
  Z = nd[0] * zr;
  invZ = nd[kTzInvA0] * izr;
  return it;
}

// Table-driven exponential (Tang, "Table-driven implementation of the
// exponential function in IEEE floating-point arithmetic", ACM TOMS 15(2),
// 1989), in the form e^x = 2^(y/64) with y = 64 x / ln 2 passed in: m =
// round(y) splits 2^(m/64) = 2^(m >> 6) tab[m & 63] (tab[i] = 2^(i/64)), and
// the rest e^u, u = (y - m) ln 2 / 64, |u| <= ln 2 / 128, is its Taylor
// polynomial of degree 5 (truncation below u^6 / 720 < 4e-17).  The scaling by
// 2^(m >> 6) adds to the exponent field, exact for |y| < 64 * 1000.  The
// error is a few ulps plus the rounding of y (|y| 2^-53 relative to e^x).
__device__ __forceinline__ double tz_exp64(double y, const double *tab) {
  const double magic = 6755399441055744.0;  // 1.5 * 2^52: rounds to an integer
  const double md = y + magic;
  const int m = (int)(uint32_t)__double_as_longlong(md);
  const double u = (y - (md - magic)) * (0.69314718055994530942 / 64.0);
  double p = fma(u, 1.0 / 120.0, 1.0 / 24.0);
  p = fma(p, u, 1.0 / 6.0);
  p = fma(p, u, 0.5);
  p = fma(p, u, 1.0);
  p = fma(p, u, 1.0);
  const double v = tab[m & 63] * p;
  return __longlong_as_double(__double_as_longlong(v) + ((long long)(m >> 6) << 52));
}

// D (Eq. 3) over t = 1..K for the law at exponent g (invZ = 1 / zeta_K(g))
// against the histogram read by bin(k), one chunk of 32 support points per
// step, every lane of the warp taking part.  FP64 form: k^-g by the
// table-driven exponential (sX = 2^(i/64)), prefix sums and comparisons in
// binary64.  FP32-bulk form: terms scaled by K^g when g < 0 (so that every
// term is at most 1), exponent g ln k as a float pair, t = exp(-p) (1 - corr),
// compensated float-pair prefix sums, comparisons in binary32.
template <bool F32, class Bin>
__device__ __forceinline__ double tz_ks(const TzTable &tb, uint32_t K, double g, double invZ, double inv_n, int lane,
                                        const double *sX, Bin bin) {
  uint32_t carryC = 0;
  if (!F32) {
    double carryP = 0.0, best = 0.0;
    const double cg = -g * (64.0 / 0.69314718055994530942);  // k^-g = 2^(cg ln k / 64)
    const double *lnk = tb.lnk;
    for (uint32_t k0 = 1; k0 <= K; k0 += 32) {
      const uint32_t k = k0 + lane;
      const bool valid = k <= K;
      const double t = valid ? tz_exp64(cg * lnk[k], sX) : 0.0;
      const uint32_t C = warp_scan_u32(valid ? bin(k) : 0u, lane) + carryC;
      const double P = warp_scan(t, lane) + carryP;
      if (valid) best = fmax(best, fabs(P * invZ - (double)C * inv_n));
      carryP = __shfl_sync(0xffffffffu, P, 31);
      carryC = __shfl_sync(0xffffffffu, C, 31);
    }
    return warp_max(best);
  }
  const bool neg = g < 0.0;
  const float *lh = neg ? tb.lnq_hi : tb.lnk_hi, *ll = neg ? tb.lnq_lo : tb.lnk_lo;
  const float gh = (float)g, gl = (float)(g - (double)gh);
  const float invZf = neg ? (float)(invZ * exp(-g * tb.lnK)) : (float)invZ, invn = (float)inv_n;
  float ch = 0.0f, cl = 0.0f, best = 0.0f;
  for (uint32_t k0 = 1; k0 <= K; k0 += 32) {
    const uint32_t k = k0 + lane;
    const bool valid = k <= K;
    float th = 0.0f, tl = 0.0f;
    if (valid) {
      const float l_h = lh[k], l_l = ll[k];
      const float p = gh * l_h;
      const float corr = fmaf(gh, l_h, -p) + fmaf(gh, l_l, gl * l_h);
      th = expf(-p) * (1.0f - corr);
    }
    warp_scan_ff(th, tl, lane);
    ff_add(th, tl, ch, cl);
    const uint32_t C = warp_scan_u32(valid ? bin(k) : 0u, lane) + carryC;
    if (valid) best = fmaxf(best, fabsf(fmaf(th, invZf, tl * invZf) - (float)C * invn));
    ch = __shfl_sync(0xffffffffu, th, 31);
    cl = __shfl_sync(0xffffffffu, tl, 31);
    carryC = __shfl_sync(0xffffffffu, C, 31);
  }
  return (double)warp_maxf(best);
}

// zeta_K(g) and its reciprocal at a given exponent in [-64, 64], from the
// node polynomial of the node at or below g.
__device__ __forceinline__ void tz_zeta_at(const TzTable &tb, double g, double &Z, double &invZ) {
  int j = (int)floor((g - kTzGammaLo) * kTzNodeInv);
  j = j < 0 ? 0 : (j > kTzNodes - 2 ? kTzNodes - 2 : j);
  const double *nd = tb.node + (size_t)j * kTzNodeStride;
  double p, dp, ddp;
  tz_poly(nd, g - (kTzGammaLo + (double)j / kTzNodeInv), p, dp, ddp);
  Z = nd[0] * p;
  invZ = nd[kTzInvA0] * tz_rcp(p);
}

template <bool F32>
__global__ void __launch_bounds__(kTzWarps * 32, PL_TZ_MIN_BLOCKS) tz_replicate_kernel(TzLaunch a) {
  __shared__ uint64_t sT[kTzKMax + 1];
  __shared__ uint16_t sG[kTzGuide];
  __shared__ uint32_t sH[kTzWarps][kTzKMax / 2 + 4];
  __shared__ double sX[64];  // 2^(i/64)
  const TzItem item = a.items[blockIdx.x];
  const TzCell &c = a.cells[item.cell];
  const TzLaw &law = a.laws[c.law];
  const TzTable &tb = a.tables[law.table];
  const uint32_t K = law.K;
  {
    const uint64_t *T = law.T;
    const uint16_t *G = law.guide;
    for (uint32_t i = threadIdx.x; i <= K; i += blockDim.x) sT[i] = T[i];
    for (uint32_t i = threadIdx.x; i < (uint32_t)kTzGuide; i += blockDim.x) sG[i] = G[i];
  }
  if (!F32 && threadIdx.x < 64) sX[threadIdx.x] = exp2((double)threadIdx.x / 64.0);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *h = sH[warp];
  const uint32_t n = (uint32_t)c.n;
  const uint32_t nwords = (K >> 1) + 1;
  const uint32_t nquads = (n + 3) >> 2;
  const double inv_n = 1.0 / (double)n;
  for (uint32_t rr = warp; rr < item.nrep; rr += kTzWarps) {
    const uint32_t r = item.r0 + rr;
    for (uint32_t i = lane; i < nwords; i += 32) h[i] = 0u;
    __syncwarp();
    uint32_t c12 = 0, c34 = 0;
    // draw i's high word is word i mod 4 of block i / 4; its low word is
    // drawn only when a threshold lies inside its interval of m
    auto one = [&](uint32_t hw, uint32_t i) {
      auto m_full = [&] { return draw_m_full(hw, i, r, c.cell_id, c.purpose, a.rk.k[0], a.rk.k[1]); };
      tz_count(tz_lookup_hi(sT, sG, hw, m_full), h, c12, c34);
    };
    for (uint32_t p = lane; p < nquads; p += 32) {
      const uint4 w = philox4x32_10_rk(make_uint4(p, r, c.cell_id, c.purpose), a.rk);
      const uint32_t i0 = 4 * p;
      one(w.x, i0);
      if (i0 + 1 < n) one(w.y, i0 + 1);
      if (i0 + 2 < n) one(w.z, i0 + 2);
      if (i0 + 3 < n) one(w.w, i0 + 3);
    }
    c12 = warp_sum_u32(c12);
    c34 = warp_sum_u32(c34);
    __syncwarp();
    if (lane == 0) {
      h[0] += (c12 & 0xffffu) << 16;
      h[1] += (c12 >> 16) | ((c34 & 0xffffu) << 16);
      if (K >= 4) h[2] += c34 >> 16;
    }
    __syncwarp();
    // log-sum (with one point counted as 2 when every value is 1)
    double Ls = 0.0;
    for (uint32_t k = 2 + lane; k <= K; k += 32) Ls += (double)tz_bin(h, k) * tb.lnk[k];
    Ls = warp_sum(Ls);
    if ((c12 & 0xffffu) == n) Ls += kLn2;
    double g, Z, invZ;
    const int its = tz_fit(tb, Ls * inv_n, tz_bin(h, K) == n, lane, g, Z, invZ);
    if (its > kTzNewtonCap && lane == 0) atomicAdd(&a.ctr->newton_capped, 1ull);
    const double D = tz_ks<F32>(tb, K, g, invZ, inv_n, lane, sX, [&](uint32_t k) { return tz_bin(h, k); });
    if (lane == 0) {
      if (F32)
        static_cast<float *>(a.D_out)[c.out_off + r] = (float)D;
      else
        static_cast<double *>(a.D_out)[c.out_off + r] = D;
    }
    if (lane == 0 && a.A_out) a.A_out[c.out_off + r] = g;
    __syncwarp();
  }
}

// One data set of the truncated law, one block of 1024 threads: histogram of
// the values (1..K; any other value latches the data error and gives NaN
// outputs), then the first warp takes the log-sum (with the all-ones rule),
// the fit (or the given exponent) and D.  out = (gamma, D, zeta_K(gamma)).
template <bool F32>
__global__ void __launch_bounds__(1024) tz_dataset_kernel(const int32_t *x, int64_t n, const TzTable *tab, int fit,
                                                          double gamma, double *out, Counters *ctr) {
  __shared__ uint32_t sC[kTzKMax + 1];
  __shared__ double sX[64];
  __shared__ int s_bad;
  const TzTable &tb = *tab;
  const uint32_t K = tb.K;
  for (uint32_t i = threadIdx.x; i <= K; i += blockDim.x) sC[i] = 0u;
  if (threadIdx.x < 64) sX[threadIdx.x] = exp2((double)threadIdx.x / 64.0);
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int32_t v = x[i];
    if (v < 1 || (uint32_t)v > K)
      s_bad = 1;
    else
      atomicAdd(&sC[v], 1u);
  }
  __syncthreads();
  if (s_bad) {
    if (threadIdx.x == 0) {
      atomicOr(&ctr->status, kErrData);
      out[0] = out[1] = out[2] = __longlong_as_double(0x7ff8000000000000ll);
    }
    return;
  }
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const double inv_n = 1.0 / (double)n;
  double Ls = 0.0;
  for (uint32_t k = 2 + lane; k <= K; k += 32) Ls += (double)sC[k] * tb.lnk[k];
  Ls = warp_sum(Ls);
  if ((int64_t)sC[1] == n) Ls += kLn2;
  double g, Z, invZ;
  if (fit) {
    const int its = tz_fit(tb, Ls * inv_n, (int64_t)sC[K] == n, lane, g, Z, invZ);
    if (its > kTzNewtonCap && lane == 0) atomicAdd(&ctr->newton_capped, 1ull);
  } else {
    g = gamma;
    tz_zeta_at(tb, g, Z, invZ);
  }
  const double D = tz_ks<F32>(tb, K, g, invZ, inv_n, lane, sX, [&](uint32_t k) { return sC[k]; });
  if (lane == 0) {
    out[0] = g;
    out[1] = D;
    out[2] = Z;
  }
}

}  // namespace

cudaError_t launch_tz_dataset(const int32_t *x, int64_t n, const TzTable *tab, bool fit, double gamma, bool f32,
                              double *out, Counters *ctr, cudaStream_t st) {
  if (f32)
    tz_dataset_kernel<true><<<1, 1024, 0, st>>>(x, n, tab, fit ? 1 : 0, gamma, out, ctr);
  else
    tz_dataset_kernel<false><<<1, 1024, 0, st>>>(x, n, tab, fit ? 1 : 0, gamma, out, ctr);
  return cudaGetLastError();
}

cudaError_t launch_tz_setup(TzLaw *laws, int nlaws, TzTable *tables, int ntables, cudaStream_t st) {
  if (ntables > 0) {
    tz_log_kernel<<<dim3((kTzKMax + 1 + 255) / 256, ntables), 256, 0, st>>>(tables);
    tz_node_kernel<<<dim3((kTzNodes * 32 + 255) / 256, ntables), 256, 0, st>>>(tables);
    tz_node_interval_kernel<<<dim3((kTzNodes + 255) / 256, ntables), 256, 0, st>>>(tables);
  }
  if (nlaws > 0) tz_law_kernel<<<nlaws, 1024, 0, st>>>(laws);
  return cudaGetLastError();
}

cudaError_t launch_tz_sample(const TzLaw *law, uint64_t seed, uint32_t cell_id, uint32_t purpose,
                             uint32_t rep0, int64_t nrep, int64_t n, uint64_t *out, cudaStream_t st) {
  const uint64_t total = (uint64_t)nrep * (uint64_t)n;
  const uint64_t blocks = std::min<uint64_t>((total + 255) / 256, 152ull * 64);
  tz_sample_kernel<<<(unsigned)blocks, 256, 0, st>>>(law, round_keys(seed), cell_id, purpose, rep0, (uint64_t)nrep,
                                                   (uint64_t)n, out);
  return cudaGetLastError();
}

cudaError_t launch_tz_replicates(const TzLaunch &a, bool f32, cudaStream_t st) {
  if (f32)
    tz_replicate_kernel<true><<<a.nitems, kTzWarps * 32, 0, st>>>(a);
  else
    tz_replicate_kernel<false><<<a.nitems, kTzWarps * 32, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace pl
