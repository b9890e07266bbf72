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
// r < kTzTerms (all terms of one a_r share a sign), E_j = -a_1 / a_0 (the
// mean of ln X) and V_j = 2 a_2 / a_0 - E_j^2 (its variance).
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
#pragma unroll
    for (int r = 0; r < kTzTerms; ++r) nd[r] = a[r];
    const double E = -a[1] / a[0];
    nd[kTzTerms] = E;
    nd[kTzTerms + 1] = 2.0 * a[2] / a[0] - E * E;
    t.E[j] = E;
  }
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

__global__ void tz_sample_kernel(const TzLaw *law, RoundKeys rk, uint32_t cell_id, uint32_t purpose,
                                 uint32_t rep0, uint64_t nrep, uint64_t n, uint64_t *out) {
  const uint64_t total = nrep * n;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t r = i / n, d = i - r * n;
    const uint4 w = philox4x32_10_rk(make_uint4((uint32_t)(d >> 1), rep0 + (uint32_t)r, cell_id, purpose), rk);
    const uint64_t m = (d & 1) ? draw_bits(w.z, w.w) : draw_bits(w.x, w.y);
    out[i] = tz_lookup(law->T, law->guide, m);
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

// zeta_K and its first two gamma-derivatives at gamma_j + delta from node j's
// polynomial (Horner with derivatives).
__device__ __forceinline__ void tz_poly(const double *nd, double d, double &z0, double &z1, double &z2) {
  double p = nd[kTzTerms - 1], dp = 0.0, ddp = 0.0;
#pragma unroll
  for (int r = kTzTerms - 2; r >= 0; --r) {
    ddp = fma(ddp, d, dp);
    dp = fma(dp, d, p);
    p = fma(p, d, nd[r]);
  }
  z0 = p;
  z1 = dp;
  z2 = 2.0 * ddp;
}
__device__ __forceinline__ double tz_poly0(const double *nd, double d) {
  double p = nd[kTzTerms - 1];
#pragma unroll
  for (int r = kTzTerms - 2; r >= 0; --r) p = fma(p, d, nd[r]);
  return p;
}

// MLE (Eq. 2 with the finite scaling factor): the root of
// E_gamma[ln X] = mbar, E decreasing in gamma.  Every lane of the warp runs
// the same steps.  The node bracket E_j >= mbar > E_{j+1} is found by a
// 32-way search (three rounds of ballots over the node means), the start by
// cubic Hermite interpolation of gamma(E) between the two nodes, and the
// root by Newton on the node polynomial, safeguarded by bisection on
// [gamma_j, gamma_j + 1/32] to 4 ulp of max(|gamma|, 1).  Means at or
// beyond the ends of [-64, 64] give the end.  Returns the iterations
// (kTzNewtonCap + 1 if the cap was hit); *Z = zeta_K(gamma-hat).
__device__ __forceinline__ int tz_fit(const TzTable &tb, double mbar, int lane, double &g_out, double &Z) {
  const double *E = tb.E;
  if (!(mbar < E[0])) {
    g_out = kTzGammaLo;
    Z = tb.node[0];
    return 0;
  }
  if (!(mbar > E[kTzNodes - 1])) {
    g_out = kTzGammaHi;
    Z = tb.node[(size_t)(kTzNodes - 1) * kTzNodeStride];
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
  const double E0 = nd[kTzTerms], V0 = nd[kTzTerms + 1];
  const double E1 = nd[kTzNodeStride + kTzTerms], V1 = nd[kTzNodeStride + kTzTerms + 1];
  const double dE = E0 - E1;
  const double t = (E0 - mbar) / dE;
  const double t2 = t * t, t3 = t2 * t;
  double d = (t3 - 2.0 * t2 + t) * (dE / V0) + (3.0 * t2 - 2.0 * t3) * h + (t3 - t2) * (dE / V1);
  if (!(d >= 0.0 && d <= h)) d = t * h;
  const double tol = 4.0 * ldexp(1.0, ilogb(fmax(fabs(gj), 1.0)) - 52);
  double lo = 0.0, hi = h;
  int it = 1;
  for (; it <= kTzNewtonCap; ++it) {
    double z0, z1, z2;
    tz_poly(nd, d, z0, z1, z2);
    const double iz = 1.0 / z0;
    const double e = -z1 * iz;
    const double var = z2 * iz - e * e;
    const double f = e - mbar;
    if (f > 0.0)
      lo = d;
    else
      hi = d;
    double nx = d + f / var;
    if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
    const double step = fabs(nx - d);
    d = nx;
    if (step <= tol || hi - lo <= tol) break;
  }
  g_out = gj + d;
  Z = tz_poly0(nd, d);
  return it;
}

template <bool F32>
__global__ void __launch_bounds__(kTzWarps * 32, 2) tz_replicate_kernel(TzLaunch a) {
  __shared__ uint64_t sT[kTzKMax + 1];
  __shared__ uint16_t sG[kTzGuide];
  __shared__ uint32_t sH[kTzWarps][kTzKMax / 2 + 4];
  const TzItem item = a.items[blockIdx.x];
  const TzCell c = a.cells[item.cell];
  const TzLaw law = a.laws[c.law];
  const TzTable tb = a.tables[law.table];
  const uint32_t K = law.K;
  for (uint32_t i = threadIdx.x; i <= K; i += blockDim.x) sT[i] = law.T[i];
  for (uint32_t i = threadIdx.x; i < (uint32_t)kTzGuide; i += blockDim.x) sG[i] = law.guide[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *h = sH[warp];
  const uint32_t n = (uint32_t)c.n;
  const uint32_t nwords = (K >> 1) + 1;
  const uint32_t npairs = (n + 1) >> 1;
  const double inv_n = 1.0 / (double)n;
  for (uint32_t rr = warp; rr < item.nrep; rr += kTzWarps) {
    const uint32_t r = item.r0 + rr;
    for (uint32_t i = lane; i < nwords; i += 32) h[i] = 0u;
    __syncwarp();
    uint32_t c12 = 0, c34 = 0;
    for (uint32_t p = lane; p < npairs; p += 32) {
      const uint4 w = philox4x32_10_rk(make_uint4(p, r, c.cell_id, c.purpose), a.rk);
      tz_count(tz_lookup(sT, sG, draw_bits(w.x, w.y)), h, c12, c34);
      if (2 * p + 1 < n) tz_count(tz_lookup(sT, sG, draw_bits(w.z, w.w)), h, c12, c34);
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
    double g, Z;
    const int its = tz_fit(tb, Ls * inv_n, lane, g, Z);
    if (its > kTzNewtonCap && lane == 0) atomicAdd(&a.ctr->newton_capped, 1ull);
    // D over the support, one chunk of 32 support points per step
    uint32_t carryC = 0;
    if (!F32) {
      const double invZ = 1.0 / Z;
      double carryP = 0.0, best = 0.0;
      for (uint32_t k0 = 1; k0 <= K; k0 += 32) {
        const uint32_t k = k0 + lane;
        const bool valid = k <= K;
        const double t = valid ? exp(-g * tb.lnk[k]) : 0.0;
        const uint32_t C = warp_scan_u32(valid ? tz_bin(h, k) : 0u, lane) + carryC;
        const double P = warp_scan(t, lane) + carryP;
        if (valid) best = fmax(best, fabs(P * invZ - (double)C * inv_n));
        carryP = __shfl_sync(0xffffffffu, P, 31);
        carryC = __shfl_sync(0xffffffffu, C, 31);
      }
      best = warp_max(best);
      if (lane == 0) static_cast<double *>(a.D_out)[c.out_off + r] = best;
    } else {
      // terms k^-g scaled by K^g when g < 0 (so that every term is at most 1),
      // exponent g ln k as a float pair: t = exp(-p) (1 - corr)
      const bool neg = g < 0.0;
      const float *lh = neg ? tb.lnq_hi : tb.lnk_hi, *ll = neg ? tb.lnq_lo : tb.lnk_lo;
      const float gh = (float)g, gl = (float)(g - (double)gh);
      const double Zs = neg ? Z * exp(g * tb.lnK) : Z;
      const float invZ = (float)(1.0 / Zs), invn = (float)inv_n;
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
        const uint32_t C = warp_scan_u32(valid ? tz_bin(h, k) : 0u, lane) + carryC;
        if (valid) best = fmaxf(best, fabsf(fmaf(th, invZ, tl * invZ) - (float)C * invn));
        ch = __shfl_sync(0xffffffffu, th, 31);
        cl = __shfl_sync(0xffffffffu, tl, 31);
        carryC = __shfl_sync(0xffffffffu, C, 31);
      }
      best = warp_maxf(best);
      if (lane == 0) static_cast<float *>(a.D_out)[c.out_off + r] = best;
    }
    if (lane == 0 && a.A_out) a.A_out[c.out_off + r] = g;
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_tz_setup(TzLaw *laws, int nlaws, TzTable *tables, int ntables, cudaStream_t st) {
  if (ntables > 0) {
    tz_log_kernel<<<dim3((kTzKMax + 1 + 255) / 256, ntables), 256, 0, st>>>(tables);
    tz_node_kernel<<<dim3((kTzNodes * 32 + 255) / 256, ntables), 256, 0, st>>>(tables);
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
