// pl_kernels.cu -- sm_103a kernels of the KS-cutoff simulation.
//
// Per replicate (Section 4 of the paper): n draws from the law
// p(k) = k^-alpha / zeta(alpha, xmin) (Eq. 1), the maximum-likelihood exponent
// (Eq. 2), and the KS distance at the fitted exponent (Eq. 3); per cell the
// order statistics of D (the cutoffs of Table 1).
#include <cfloat>
#include <cstdio>

#include "pl_kernels.cuh"

namespace pl {

#ifdef PL_PHASE_TIMING
#define PL_PHASE(i)                                                                     \
  do {                                                                                  \
    const long long t_ = clock64();                                                     \
    if (lane == 0) atomicAdd(&a.ctr->phase_cycles[i], (unsigned long long)(t_ - pt_)); \
    pt_ = t_;                                                                           \
  } while (0)
#else
#define PL_PHASE(i) \
  do {              \
  } while (0)
#endif

// ===========================================================================
// Shared-memory staging of a law's level-1 thresholds and guide table by the
// bulk-copy (TMA) engine.  Every thread waits (bounded); the outcome is made
// uniform across the block so that no thread leaves a barrier early.  The
// kernels keep two mbarriers: mbar[0] for the copies, mbar[1] never arrived at
// (the flag a test makes the first wait run out on).
struct StagedLaw {
  uint64_t *sT;
  uint32_t *sG;
  uint64_t *mbar;
  uint32_t *sInc = nullptr;  // the increment table too, when given (with the fine guide in sG)
  float *sLn = nullptr;      // and the binary32 splits of ln(xmin + i), i < kHMax (hi, then lo)
};

constexpr uint32_t kIncBytes = (uint32_t)kIncBuckets * 32 * sizeof(uint32_t);
constexpr uint32_t kLnBytes = (uint32_t)kHMax * sizeof(float);

__device__ bool stage_law(const StagedLaw &s, const Law &law, uint32_t &phase, Counters *ctr) {
  if (threadIdx.x == 0) {
    const uint32_t gbytes = (uint32_t)((s.sInc ? kFine : kGuide) * sizeof(uint32_t));
    mbar_expect_tx(s.mbar, (uint32_t)(kL1 * sizeof(uint64_t)) + gbytes + (s.sInc ? kIncBytes : 0u) +
                               (s.sLn ? 2u * kLnBytes : 0u));
    bulk_g2s(s.sT, law.T, (uint32_t)(kL1 * sizeof(uint64_t)), s.mbar);
    bulk_g2s(s.sG, s.sInc ? law.fine : law.guide, gbytes, s.mbar);
    if (s.sInc) bulk_g2s(s.sInc, law.inc, kIncBytes, s.mbar);
    if (s.sLn) {
      bulk_g2s(s.sLn, law.lnT_hi, kLnBytes, s.mbar);
      bulk_g2s(s.sLn + kHMax, law.lnT_lo, kLnBytes, s.mbar);
    }
  }
  // test hook (wait_limit set): wait instead on the block's second barrier,
  // at which nothing ever arrives, for wait_limit cycles
  const bool ok = ctr->wait_limit ? mbar_wait_bounded(s.mbar + 1, 0u, (long long)ctr->wait_limit)
                                  : mbar_wait_bounded(s.mbar, phase);
  const int any_fail = __syncthreads_or(!ok);
  if (any_fail) {
    if (threadIdx.x == 0) atomicOr(&ctr->status, kErrTimeout);
    mbar_wait_bounded(s.mbar, phase);  // full bound: let copies in flight land before exit
    return false;
  }
  phase ^= 1u;
  return true;
}

// ===========================================================================
// Sampling only (pl_sample): one thread per four draws, each m taken whole
// (both words).
__global__ void __launch_bounds__(256) sample_kernel(const Law *law_p, uint64_t seed,
                                                     uint32_t cell_id, uint32_t purpose,
                                                     uint32_t rep0, int64_t nrep, int64_t n,
                                                     uint64_t *out, Counters *ctr) {
  extern __shared__ __align__(16) uint8_t smem[];
  StagedLaw s{(uint64_t *)smem, (uint32_t *)(smem + kL1 * 8), (uint64_t *)(smem + kL1 * 8 + kGuide * 4)};
  const Law law = *law_p;
  if (threadIdx.x == 0) {
    mbar_init(s.mbar, 1);
    mbar_init(s.mbar + 1, 1);
  }
  __syncthreads();
  uint32_t phase = 0;
  if (!stage_law(s, law, phase, ctr)) return;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const int64_t nquads = (n + 3) >> 2;
  const int64_t total = nquads * nrep;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / nquads;
    const int64_t p = idx - r * nquads;
    const uint4 wh = philox4x32_10(make_uint4((uint32_t)p, rep0 + (uint32_t)r, cell_id, purpose), key);
    const uint4 wl = philox4x32_10(make_uint4((uint32_t)p, rep0 + (uint32_t)r, cell_id, purpose | kLowStream), key);
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
      const int64_t i = 4 * p + j;
      if (i < n) {
        const uint64_t m = draw_m(quad_word(wh, j), quad_word(wl, j));
        out[r * n + i] = lookup(s.sT, s.sG, law.T, law.L2, law.xmin, law.alpha, law.Z, law.xmin_f,
                                law.tail_c, law.tail_e, m, &ctr->tail_draws);
      }
    }
  }
}

cudaError_t launch_sample(const Law *law_dev, uint64_t seed, uint32_t cell_id, uint32_t purpose,
                          uint32_t rep0, int64_t nrep, int64_t n, uint64_t *out, Counters *ctr,
                          int num_sms, cudaStream_t st) {
  const size_t smem = kL1 * 8 + kGuide * 4 + 16;
  const int64_t quads = ((n + 3) / 4) * nrep;
  int64_t blocks = (quads + 255) / 256;
  const int64_t cap = (int64_t)num_sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  sample_kernel<<<(unsigned)blocks, 256, smem, st>>>(law_dev, seed, cell_id, purpose, rep0, nrep, n,
                                                     out, ctr);
  return cudaGetLastError();
}

// ===========================================================================
// Newton-Raphson for the MLE (Eq. 2), one lane per replicate, binary64:
// f(a) = zeta'(a,xmin)/zeta(a,xmin) + mbar is increasing in a (f' is the
// variance of ln X), safeguarded by bisection on (1 + 2^-40, 64], stopped when
// a step is within 4 ulp.  Returns the number of iterations (kNewtonCap + 1
// if the cap was hit); *Z receives zeta(alpha-hat, xmin).
template <bool PRECISE = false>
__device__ int newton_mle(double mbar, uint64_t xmin, double ln_xmin_half, const double *lnT,
                          double *alpha_hat, double *Z) {
  double lo = 1.0 + 0x1p-40, hi = 64.0;
  double a = 1.0 + 1.0 / (mbar - ln_xmin_half);
  if (!(a > lo && a < hi)) a = 0.5 * (lo + hi);
  const double x0 = (double)xmin;
  int it = 1;
  for (; it <= kNewtonCap; ++it) {
    double z[3];
    hurwitz_em<2, PRECISE>(a, x0, z, lnT, x0, kLnTable);
    const double g = z[1] / z[0];
    const double f = g + mbar;
    const double fp = z[2] / z[0] - g * g;
    if (f > 0.0) hi = a;
    else lo = a;
    double next = a - f / fp;
    if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
    const double step = fabs(next - a);
    a = next;
    const double tol = 4.0 * ldexp(1.0, ilogb(a) - 52);
    if (step <= tol || hi - lo <= tol) break;
  }
  *alpha_hat = a;
  double z0;
  hurwitz_em<0, PRECISE>(a, x0, &z0, lnT, x0, kLnTable);
  *Z = z0;
  return it;
}

// ln(a) of a uint64 as a float pair hi + lo: exponent * ln2 (split) + ln(mantissa).
__device__ __forceinline__ void ln_u64_ff(uint64_t a, float &hi, float &lo) {
  const int e = 63 - __clzll((long long)a);
  const uint64_t norm = a << (63 - e);          // leading one at bit 63
  const uint32_t m25 = (uint32_t)(norm >> 39);  // 1 + 23 fraction bits + 1 rounding bit
  const float mant = (float)((m25 + 1u) >> 1) * 0x1p-23f;  // mantissa in [1, 2], rounded
  const float lm = logf(mant);
  const float ln2_hi = 0.693145751953125f;  // 45425 / 2^16: e * ln2_hi is exact for e < 256
  const float ln2_lo = 1.4286068203094172e-06f;
  const float ef = (float)e;
  hi = ef * ln2_hi;  // exact
  float s, err;
  two_sum(hi, lm, s, err);
  lo = err + ef * ln2_lo;
  hi = s;
}

// uint64 to binary32 through 32-bit conversions (64-bit integer conversions run
// on the slow binary64 unit); within one ulp.
__device__ __forceinline__ float u64_to_f32(uint64_t v) {
  return fmaf((float)(uint32_t)(v >> 32), 4294967296.0f, (float)(uint32_t)v);
}

// exp(-(a_hi + a_lo)(l_hi + l_lo)) in binary32, the product's rounding error
// carried to first order.
__device__ __forceinline__ float exp_neg_prod(float a_hi, float a_lo, float l_hi, float l_lo) {
  const float prod = a_hi * l_hi;
  const float err = fmaf(a_hi, l_hi, -prod);
  const float tail = err + fmaf(a_hi, l_lo, a_lo * l_hi);
  return expf(-prod) * (1.0f - tail);
}

// Per-replicate fitted quantities handed to the KS step.
struct FitOut {
  double ahat;
  double Z;
  // binary32 form only
  float a_hi, a_lo, invZ, lnZ;
  float lnc, lnc_lo;                  // ln((ahat - 1) Z) as an unevaluated float pair
};

__device__ __forceinline__ FitOut fit_from_logsum(double L, int64_t n, uint64_t xmin,
                                                  const CellConst &cc, const double *lnT,
                                                  bool f32, Counters *ctr) {
  FitOut o;
  const int it = newton_mle(L / (double)n, xmin, cc.ln_xmin_half, lnT, &o.ahat, &o.Z);
  if (it > kNewtonCap) atomicAdd(&ctr->newton_capped, 1ull);
  if (f32) {
    o.a_hi = (float)o.ahat;
    o.a_lo = (float)(o.ahat - (double)o.a_hi);
    o.invZ = (float)(1.0 / o.Z);
    o.lnZ = (float)log(o.Z);
    const double lncd = log((o.ahat - 1.0) * o.Z);
    o.lnc = (float)lncd;
    o.lnc_lo = (float)(lncd - (double)o.lnc);
  }
  return o;
}

// Lane-parallel fit (one replicate per lane; every lane of the warp calls it,
// lanes without a replicate pass a harmless log-sum).  The fit table's cubic
// Hermite interpolation gives alpha-hat and ln zeta(alpha-hat) to ~1e-11
// below kFitTableOnlyMax: the binary32 form (tolerance 1e-6) takes them as
// they are.  The binary64 form polishes: one Euler-Maclaurin evaluation at
// the interpolated start gives the FP64 root (the step's error is quadratic
// in the start's), and zeta(alpha-hat) follows from the same evaluation by a
// second-order Taylor step.  A start outside the table or a step larger than
// 1e-8 alpha falls back to the full iteration.
__device__ __forceinline__ FitOut fit_lanes(double L, int64_t n, uint64_t xmin, const CellConst &cc,
                                            const FitTable &ft, const double *lnT, bool f32,
                                            Counters *ctr) {
  const double mbar = L / (double)n;
  const double h = mbar - cc.ln_xmin;
  bool ok = false;
  double a0 = 1.2, lz0 = 0.0;
  if (h > 0.0) {
    const double u = log(h);
    const double pos = (u - ft.ug0) * ft.inv_dug;
    if (pos >= 0.0 && pos < (double)ft.guides) {
      int k = ft.guide[(int)pos];
      for (int it = 0; it < 16 && k + 1 < ft.nodes - 1 && ft.node[k + 1].u <= u; ++it) ++k;
      const FitNode A = ft.node[k], B = ft.node[k + 1];
      if (u >= A.u && u <= B.u) {
        const double du = B.u - A.u;
        const double t = (u - A.u) * A.inv_du, t2 = t * t, t3 = t2 * t;
        const double h00 = 2.0 * t3 - 3.0 * t2 + 1.0, h10 = (t3 - 2.0 * t2 + t) * du,
                     h01 = 3.0 * t2 - 2.0 * t3, h11 = (t3 - t2) * du;
        a0 = h00 * A.alpha + h10 * A.dadu + h01 * B.alpha + h11 * B.dadu;
        lz0 = h00 * A.lnZ + h10 * A.dlnZdu + h01 * B.lnZ + h11 * B.dlnZdu;
        ok = true;
      }
    }
  }
  if (f32 && ok && a0 < kFitTableOnlyMax) {
    FitOut o;
    o.ahat = a0;
    o.Z = 0.0;  // the binary32 form reads invZ, lnZ and lnc only
    o.a_hi = (float)a0;
    o.a_lo = (float)(a0 - (double)o.a_hi);
    // ln zeta as a float pair: 1/zeta and the survival's constant keep the
    // pair's low part (ln zeta reaches -60 for large xmin)
    o.lnZ = (float)lz0;
    const float lz_lo = (float)(lz0 - (double)o.lnZ);
    o.invZ = expf(-o.lnZ) * (1.0f - lz_lo);
    float e;
    two_sum(logf((float)(a0 - 1.0)), o.lnZ, o.lnc, e);
    o.lnc_lo = e + lz_lo;
    return o;
  }
  // the shift is the lane's own (not a warp maximum), so a replicate's result
  // does not depend on which replicates share its warp
  double z[3];
  hurwitz_polish(a0, xmin, polish_shift_n(a0, xmin), lnT, z);
  FitOut o;
  if (ok) {
    const double inv = 1.0 / z[0];
    const double g = z[1] * inv;
    const double step = (g + mbar) / (z[2] * inv - g * g);
    if (fabs(step) <= 1e-8 * a0) {
      o.ahat = a0 - step;
      o.Z = z[0] - step * (z[1] - 0.5 * step * z[2]);
    } else {
      ok = false;
    }
  }
  if (!ok) {
    atomicAdd(&ctr->fit_fallbacks, 1ull);
    const int it = newton_mle(mbar, xmin, cc.ln_xmin_half, lnT, &o.ahat, &o.Z);
    if (it > kNewtonCap) atomicAdd(&ctr->newton_capped, 1ull);
  }
  if (f32) {
    o.a_hi = (float)o.ahat;
    o.a_lo = (float)(o.ahat - (double)o.a_hi);
    o.invZ = (float)(1.0 / o.Z);
    o.lnZ = logf((float)o.Z);
    const double lncd = log((o.ahat - 1.0) * o.Z);
    o.lnc = (float)lncd;
    o.lnc_lo = (float)(lncd - (double)o.lnc);
  }
  return o;
}

__device__ __forceinline__ FitOut shfl_fit(const FitOut &f, int src) {
  FitOut o;
  o.ahat = __shfl_sync(0xffffffffu, f.ahat, src);
  o.Z = __shfl_sync(0xffffffffu, f.Z, src);
  o.a_hi = __shfl_sync(0xffffffffu, f.a_hi, src);
  o.a_lo = __shfl_sync(0xffffffffu, f.a_lo, src);
  o.invZ = __shfl_sync(0xffffffffu, f.invZ, src);
  o.lnZ = __shfl_sync(0xffffffffu, f.lnZ, src);
  o.lnc = __shfl_sync(0xffffffffu, f.lnc, src);
  o.lnc_lo = __shfl_sync(0xffffffffu, f.lnc_lo, src);
  return o;
}

// ===========================================================================
// KS distance (Eq. 3) of one replicate by one warp.
//   Dense part: every integer t = xmin + i, i <= tmax; F(t) is the prefix sum
//   of p(k) = k^-ahat / Z, S(t) = C(t)/n; D >= |F(t) - S(t)| at each t.
//   Spill part: distinct values v beyond the dense range, ascending, with
//   counts; on each run of integers where S is constant F increases, so the
//   maximum is at v (S = C(v)/n) or v - 1 (S = C(v-1)/n):
//   F(v) = 1 - zeta(ahat, v+1)/Z and F(v-1) = F(v) - p(v).
// FP64 form: everything binary64.  FP32 form: p and F in binary32 with
// compensated (two-sum) prefix sums; Q(v) by a 4-term Euler-Maclaurin in
// binary32 (v - xmin >= 32 keeps it below 1e-8 relative).
// Q(a - 1) = zeta(s, a) / Z for a large argument a (a >= 10 + 1.5 s), binary32:
//   a^(1-s)/((s-1) Z) * [1 + (s-1)/(2a) + sum_j B2j/(2j)! s(s+1)..(s+2j-2)(s-1) a^-2j],
// with ln a = la_hi + la_lo and the product's rounding error carried.
__device__ __forceinline__ float survival_em_f32(float af, float la_hi, float la_lo, const FitOut &f) {
  // s - 1 = (a_hi - 1) + a_lo, the first part exact in binary32 (a_hi >= 1)
  const float s = f.a_hi, sm1 = f.a_hi - 1.0f;
  const float ia = 1.0f / af, ia2 = ia * ia;
  float P = s, br = 1.0f + 0.5f * sm1 * ia, w = ia2;
  const float cj[4] = {1.0f / 12.0f, -1.0f / 720.0f, 1.0f / 30240.0f, -1.0f / 1209600.0f};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    br += cj[j] * P * sm1 * w;
    P *= (s + (float)(2 * j + 1)) * (s + (float)(2 * j + 2));
    w *= ia2;
  }
  const float prod = sm1 * la_hi;
  const float perr = fmaf(sm1, la_hi, -prod) + fmaf(sm1, la_lo, f.a_lo * la_hi);
  return expf(-prod - f.lnc) * (1.0f - perr - f.lnc_lo) * br;
}

// The two candidates of a run of spilled values ending at v: |F(v) - Ca/n|
// and |F(v - 1) - Cb/n| (Ca values at most v, Cb below v).
__device__ __forceinline__ double spill_point_f64(uint64_t v, int64_t Ca, int64_t Cb, double a, double invZ,
                                                  double inv_n) {
  double q;
  hurwitz_em<0, false>(a, (double)v + 1.0, &q);
  const double Q = q * invZ;
  const double pv = exp(-a * log((double)v)) * invZ;
  const double Fv = 1.0 - Q;
  const double Fb = 1.0 - (Q + pv);
  return fmax(fabs(Fv - (double)Ca * inv_n), fabs(Fb - (double)Cb * inv_n));
}

__device__ __forceinline__ float spill_point_f32(uint64_t v, int64_t Ca, int64_t Cb, float inv_n, const FitOut &f) {
  float Q, pv;
  if (u64_to_f32(v + 1ull) < 10.0f + 1.5f * f.a_hi) {
    // exponent too large for the short binary32 series at this argument
    double q;
    hurwitz_em<0, false>(f.ahat, (double)v + 1.0, &q);
    Q = (float)(q * (double)f.invZ);
    pv = (float)(exp(-f.ahat * log((double)v)) * (double)f.invZ);
  } else {
    float la_hi, la_lo, lv_hi, lv_lo;
    ln_u64_ff(v + 1ull, la_hi, la_lo);
    ln_u64_ff(v, lv_hi, lv_lo);
    // Q(v) = zeta(s, v + 1)/Z
    Q = survival_em_f32(u64_to_f32(v + 1ull), la_hi, la_lo, f);
    pv = exp_neg_prod(f.a_hi, f.a_lo, lv_hi, lv_lo) * f.invZ;
  }
  const float Fv = 1.0f - Q;
  const float Fb = 1.0f - (Q + pv);
  return fmaxf(fabsf(Fv - (float)(uint32_t)Ca * inv_n), fabsf(Fb - (float)(uint32_t)Cb * inv_n));
}

template <bool F32, typename DT>
__device__ double ks_warp(const DT *dense, int64_t tmax, const uint64_t *pairs, int64_t nsd,
                          int64_t n, uint64_t xmin, const FitOut &f, const double *lnT, const float *lnT_hi,
                          const float *lnT_lo, int lane) {
  if (!F32) {
    const double invZ = 1.0 / f.Z;
    const double inv_n = 1.0 / (double)n;
    const double a = f.ahat;
    double carryF = 0.0, best = 0.0;
    int64_t carryC = 0;
    for (int64_t i0 = 0; i0 <= tmax; i0 += 32) {
      const int64_t i = i0 + lane;
      const bool ok = i <= tmax;
      const double p = ok ? exp(-a * lnT[i]) * invZ : 0.0;
      const int64_t c = ok ? (int64_t)dense[i] : 0;
      const double F = carryF + warp_scan(p, lane);
      const int64_t C = carryC + warp_scan_i64(c, lane);
      if (ok) best = fmax(best, fabs(F - (double)C * inv_n));
      carryF = __shfl_sync(0xffffffffu, F, 31);
      carryC = __shfl_sync(0xffffffffu, C, 31);
    }
    for (int64_t k0 = 0; k0 < nsd; k0 += 32) {
      const int64_t k = k0 + lane;
      const bool ok = k < nsd;
      const uint64_t v = ok ? pairs[2 * k] : 0;
      const int64_t c = ok ? (int64_t)pairs[2 * k + 1] : 0;
      const int64_t Ca = carryC + warp_scan_i64(c, lane);
      if (ok) best = fmax(best, spill_point_f64(v, Ca, Ca - c, a, invZ, inv_n));
      carryC = __shfl_sync(0xffffffffu, Ca, 31);
    }
    return warp_max(best);
  } else {
    const float inv_n = 1.0f / (float)(uint32_t)n;  // n < 2^31: 32-bit conversions only
    float best = 0.0f;
    // dense part, one contiguous chunk of bins per lane.  The chunk's starting
    // F = 1 - zeta(s, xmin + i0)/Z comes from the short Euler-Maclaurin series
    // once the argument is large enough, else from the compensated sum of the
    // bins below it; then one compensated pass over the chunk.
    const int64_t nbins = tmax + 1;
    // odd chunk length: the lanes' bins (and log splits) fall in 32 different
    // shared-memory banks
    const int64_t cs = ((nbins + 31) >> 5) | 1;
    const int64_t i0 = (int64_t)lane * cs;
    const int64_t i1 = i0 + cs < nbins ? i0 + cs : nbins;
    int64_t sc = 0;
    for (int64_t i = i0; i < i1; ++i) sc += (int64_t)dense[i];
    const int64_t incC = warp_scan_i64(sc, lane);
    int64_t C = incC - sc;
    float Fh = 0.0f, Fl = 0.0f;
    if (i0 > 0 && i0 < nbins) {
      const float af = u64_to_f32(xmin + (uint64_t)i0);
      if (af >= 10.0f + 1.5f * f.a_hi) {
        two_sum(1.0f, -survival_em_f32(af, lnT_hi[i0], lnT_lo[i0], f), Fh, Fl);
      } else {
        for (int64_t i = 0; i < i0; ++i)
          ff_add(Fh, Fl, exp_neg_prod(f.a_hi, f.a_lo, lnT_hi[i], lnT_lo[i]) * f.invZ, 0.0f);
      }
    }
    for (int64_t i = i0; i < i1; ++i) {
      ff_add(Fh, Fl, exp_neg_prod(f.a_hi, f.a_lo, lnT_hi[i], lnT_lo[i]) * f.invZ, 0.0f);
      C += (int64_t)dense[i];
      best = fmaxf(best, fabsf(Fh - (float)(uint32_t)C * inv_n));
    }
    int64_t carryC = __shfl_sync(0xffffffffu, incC, 31);
    for (int64_t k0 = 0; k0 < nsd; k0 += 32) {
      const int64_t k = k0 + lane;
      const bool ok = k < nsd;
      const uint64_t v = ok ? pairs[2 * k] : 0;
      const int64_t c = ok ? (int64_t)pairs[2 * k + 1] : 0;
      const int64_t Ca = carryC + warp_scan_i64(c, lane);
      if (ok) best = fmaxf(best, spill_point_f32(v, Ca, Ca - c, inv_n, f));
      carryC = __shfl_sync(0xffffffffu, Ca, 31);
    }
    return (double)warp_maxf(best);
  }
}

// ===========================================================================
// Stable LSD radix sort of s uint64 keys by one warp, 8-bit digits of
// (key - smallest key), only as many digits as the key range needs.  Keys
// move between a and b (global memory, s entries each) and end in a; cnt is
// 256 words of the warp's shared memory.  A pass: digit counts (shared
// atomics), exclusive scan, then a stable scatter of 32 keys at a time (equal
// digits ranked among the warp's lanes with match.any).
__device__ void warp_radix_sort(uint64_t *a, uint64_t *b, int64_t s, uint32_t *cnt, int lane) {
  uint64_t lo = ~0ull, hi = 0;
  for (int64_t i = lane; i < s; i += 32) {
    const uint64_t x = a[i];
    lo = x < lo ? x : lo;
    hi = x > hi ? x : hi;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t l2 = __shfl_xor_sync(0xffffffffu, lo, o), h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = l2 < lo ? l2 : lo;
    hi = h2 > hi ? h2 : hi;
  }
  const uint64_t span = hi - lo;
  const int passes = span ? (71 - __clzll((long long)span)) / 8 : 0;  // ceil(bits / 8)
  uint64_t *src = a, *dst = b;
  for (int p = 0; p < passes; ++p) {
    const int sh = 8 * p;
    for (int d = lane; d < 256; d += 32) cnt[d] = 0;
    __syncwarp();
    for (int64_t i = lane; i < s; i += 32) atomicAdd(&cnt[(uint32_t)((src[i] - lo) >> sh) & 255u], 1u);
    __syncwarp();
    uint32_t v[8], t = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      v[k] = cnt[lane * 8 + k];
      t += v[k];
    }
    uint32_t incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    uint32_t run = incl - t;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      cnt[lane * 8 + k] = run;
      run += v[k];
    }
    __syncwarp();
    for (int64_t i0 = 0; i0 < s; i0 += 32) {
      const int64_t i = i0 + lane;
      const bool ok = i < s;
      const uint64_t x = ok ? src[i] : 0;
      const uint32_t d = ok ? ((uint32_t)((x - lo) >> sh) & 255u) : 256u + (uint32_t)lane;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const int rank = __popc(peers & ((1u << lane) - 1u));
      const uint32_t base = ok ? cnt[d] : 0u;
      __syncwarp();
      if (ok) {
        dst[base + rank] = x;
        if (rank == 0) cnt[d] = base + __popc(peers);
      }
      __syncwarp();
    }
    uint64_t *t2 = src;
    src = dst;
    dst = t2;
  }
  if (src != a) {
    for (int64_t i = lane; i < s; i += 32) a[i] = src[i];
    __syncwarp();
  }
}

// Bitonic sort of 32 < s <= 64 values in place: lane l holds elements 2l and
// 2l + 1 in registers (padding with the largest key); stride 1 is an exchange
// within a lane, larger strides exchanges with lane l ^ (stride / 2).
__device__ __forceinline__ void warp_bitonic_sort64(uint64_t *a, int64_t s, int lane) {
  uint64_t v[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) v[k] = 2 * lane + k < s ? a[2 * lane + k] : ~0ull;
#pragma unroll
  for (int size = 2; size <= 64; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride == 1) {
        const bool up = ((2 * lane) & size) == 0;
        const uint64_t mn = v[0] < v[1] ? v[0] : v[1], mx = v[0] < v[1] ? v[1] : v[0];
        v[0] = up ? mn : mx;
        v[1] = up ? mx : mn;
      } else {
        const int ls = stride >> 1;
        const bool lower = (lane & ls) == 0, up = ((2 * lane) & size) == 0;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const uint64_t y = __shfl_xor_sync(0xffffffffu, v[k], ls);
          const uint64_t mn = v[k] < y ? v[k] : y, mx = v[k] < y ? y : v[k];
          v[k] = (lower == up) ? mn : mx;
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 2; ++k)
    if (2 * lane + k < s) a[2 * lane + k] = v[k];
  __syncwarp();
}

// Sort the s spill values of one replicate, in place (up to 32: a bitonic
// network across the lanes' registers; up to 64: the same with two values per
// lane; more: the warp radix sort with `pairs` as the second buffer) and
// run-length encode them into interleaved (value, count) pairs at `pairs`
// (room for 2 s entries).  Returns the number of distinct values.
__device__ int64_t spill_compact(uint64_t *spill, uint32_t *onchip, int64_t s, uint64_t *pairs,
                                 int lane, Counters *ctr) {
  if (s <= 0) return 0;
  if (s <= 32) {
    uint64_t x = lane < s ? spill[lane] : ~0ull;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        const uint64_t y = __shfl_xor_sync(0xffffffffu, x, j);
        const bool up = (lane & k) == 0, lower = (lane & j) == 0;
        x = (lower == up) ? (x < y ? x : y) : (x < y ? y : x);
      }
    }
    const uint64_t prev = __shfl_up_sync(0xffffffffu, x, 1);
    const bool start = lane < s && (lane == 0 || prev != x);
    const unsigned bal = __ballot_sync(0xffffffffu, start);
    const unsigned after = bal & ~((2u << lane) - 1u);  // run starts beyond this lane
    const int next = after ? __ffs((int)after) - 1 : (int)s;
    if (start) {
      const int rank = __popc(bal & ((1u << lane) - 1u));
      pairs[2 * rank] = x;
      pairs[2 * rank + 1] = (uint64_t)(next - lane);
    }
    __syncwarp();
    return __popc(bal);
  }
  if (s <= 64) {
    warp_bitonic_sort64(spill, s, lane);
  } else {
    if (s > kSortSmem && lane == 0) atomicAdd(&ctr->global_sorts, 1ull);
    warp_radix_sort(spill, pairs, s, onchip, lane);
  }
  const uint64_t *buf = spill;
  int64_t base = 0;
  for (int64_t i0 = 0; i0 < s; i0 += 32) {
    const int64_t i = i0 + lane;
    const bool ok = i < s;
    const uint64_t x = ok ? buf[i] : 0;
    const bool start = ok && (i == 0 || buf[i - 1] != x);
    const unsigned bal = __ballot_sync(0xffffffffu, start);
    const int rank = __popc(bal & ((1u << lane) - 1u));
    if (start) {
      pairs[2 * (base + rank)] = x;
      pairs[2 * (base + rank) + 1] = (uint64_t)i;  // start position; count below
    }
    base += __popc(bal);
  }
  __syncwarp();
  for (int64_t k0 = 0; k0 < base; k0 += 32) {
    const int64_t k = k0 + lane;
    uint64_t cnt = 0;
    if (k < base) {
      const uint64_t st = pairs[2 * k + 1];
      const uint64_t en = (k + 1 < base) ? pairs[2 * (k + 1) + 1] : (uint64_t)s;
      cnt = en - st;
    }
    __syncwarp();
    if (k < base) pairs[2 * k + 1] = cnt;
    __syncwarp();
  }
  return base;
}

// ===========================================================================
// The two kernels of a simulation wave.
//
// Sampler (many warps, few registers): a block takes a work item (one cell,
// kItemReps replicates) and stages the law's table in shared memory; each warp
// draws its replicates (Philox, table search), histograms values below
// xmin + H in shared memory (two 16-bit bins per word; values xmin..xmin+3 in
// per-lane register counters) and writes the replicate record: the dense
// counts, up to scap spilled values (those beyond the table tagged for the
// finisher), and (tmax, spill count).
//
// Finisher: each warp takes 32 replicates of an item:
//   phase 1 (warp per replicate): resolve tagged tail draws (binary64), the
//           log-sum, sort and run-length encode the spills into the warp's
//           arena; a replicate whose spill slot overflowed is drawn again here
//           with a global spill buffer (same Philox stream, same values);
//   phase 2 (lane per replicate): binary64 fit (interpolated start + polish);
//   phase 3 (warp per replicate): KS distance.
#ifndef PL_SAMPLER_WARPS
#define PL_SAMPLER_WARPS 32
#endif
// entries per lane of a warp's draw queue: 10 take the sampler block's shared
// memory to 229,528 of the 232,448 bytes a block may use, and a warp drains
// once a lane holds more than 6 (8 entries, drained after 4, ran 3 % slower
// on GB300)
#ifndef PL_SAMPLER_QCAP
#define PL_SAMPLER_QCAP 10
#endif
constexpr int kAWarps = PL_SAMPLER_WARPS;
constexpr int kARepsPerWarp = (kItemReps + kAWarps - 1) / kAWarps;
#ifndef PL_SAMPLER_BLOCKS
#define PL_SAMPLER_BLOCKS (PL_SAMPLER_WARPS >= 24 ? 1 : 2)
#endif
constexpr int kABlocksPerSM = PL_SAMPLER_BLOCKS;

struct TailQueue {
  uint64_t *pos;          // element index in the record spill buffer
  uint32_t *law;          // law of the draw
  unsigned int *count;
  uint32_t cap;
};

// Draws of one replicate into a histogram, one draw at a time (the
// finisher's redraw of a replicate whose record spill slot overflowed).
// PACKED: two 16-bit bins per word (hist holds H/2 words); otherwise one
// 32-bit bin per word.  Spills beyond the capacity are counted but not stored;
// draws beyond the threshold table are stored tagged (kTailTag | m).  Returns
// tmax (the largest bin index below H that was hit, -1 if none) and leaves
// the spill count in *s_count.  The same values as the samplers' draws.
template <bool PACKED>
__device__ __forceinline__ int64_t draw_replicate(const uint64_t *sT, const uint32_t *sG, const Law &law,
                                                  const Cell &cell, uint32_t rep, const RoundKeys &rk,
                                                  uint32_t *hist, int *s_count, uint64_t *spill,
                                                  int64_t spill_capacity, int lane) {
  const int64_t n = cell.n;
  const uint64_t xmin = cell.xmin;
  const uint32_t H = cell.H;
  const int words = PACKED ? (int)(H / 2) : (int)H;
  for (int i = lane; i < words; i += 32) hist[i] = 0;
  if (lane == 0) *s_count = 0;
  __syncwarp();
  // b: the draw's table index; m: its m, needed (and given) only beyond the table
  auto bin = [&](uint32_t b, uint64_t m) {
    if (b < H) {
      if (PACKED) atomicAdd(&hist[b >> 1], 1u << ((b & 1u) << 4));
      else atomicAdd(&hist[b], 1u);
    } else {
      const int slot = atomicAdd(s_count, 1);
      if (slot < spill_capacity) spill[slot] = b < law.L2 ? xmin + b : (kTailTag | m);
    }
  };
  auto m_of = [&](uint32_t h, uint64_t i) {
    return draw_m_full(h, i, rep, cell.cell_id, cell.purpose, rk.k[0], rk.k[1]);
  };
  auto draw = [&](uint32_t h, uint64_t i) {
    const uint32_t gw = sG[h >> (32 - kGuideBits)];
    if (gw & kGuideMulti) {
      uint64_t m = 0;
      const uint32_t b = lookup_index_hi(sT, sG, law.T, law.L2, law.xmin_f, law.tail_c, law.tail_e, h,
                                         [&] { return m_of(h, i); }, &m);
      bin(b, m);
    } else {
      bin(gw, gw >= law.L2 ? m_of(h, i) : 0ull);
    }
  };
  for (int64_t p = lane; 4 * p < n; p += 32) {
    const uint4 w = philox4x32_10_rk(make_uint4((uint32_t)p, rep, cell.cell_id, cell.purpose), rk);
    const int64_t i0 = 4 * p;
    if (i0 < n) draw(w.x, (uint64_t)i0);
    if (i0 + 1 < n) draw(w.y, (uint64_t)i0 + 1);
    if (i0 + 2 < n) draw(w.z, (uint64_t)i0 + 2);
    if (i0 + 3 < n) draw(w.w, (uint64_t)i0 + 3);
  }
  __syncwarp();
  // largest bin hit: highest nonzero word, then its upper half
  int tw = -1;
  for (int i = lane; i < words; i += 32)
    if (hist[i]) tw = i;
  tw = __reduce_max_sync(0xffffffffu, (unsigned)(tw + 1)) - 1;
  if (!PACKED || tw < 0) return tw;
  return 2 * (int64_t)tw + ((hist[tw] >> 16) ? 1 : 0);
}

// Draws of one replicate for the warp-form sampler.  Every draw looks up its
// high word in the increment table (the lane's own copy, so the warp's 32
// loads touch 32 banks) and adds the entry to the lane's register `acc`:
// draws of the first four values count in its four 7-bit fields, flushed to
// 32-bit counters every kFlushBlocks Philox blocks (at most 124 increments).
// Every other draw (a larger value, a bucket holding a threshold, a value
// beyond the table) is appended to the lane's queue in shared memory (column
// `lane`, kQCap entries) with no warp vote; once a lane's queue may not take
// another block's four draws the warp drains all queues: the word of the fine
// guide (2^13 buckets), a
// search of the shared level-1 table where the bucket holds several values
// (compacted across the warp; level 2 of the table in global memory), then a
// shared atomic below H or a spill.  A value beyond the table is spilled as
// kTailTag | m and resolved by the tail kernel (binary64 inversion).  Counts
// do not depend on the order draws are
// binned in, and spills are sorted later, so the record equals
// draw_replicate's.  Returns tmax and leaves the spill count in *s_count.
constexpr int kQCap = PL_SAMPLER_QCAP;
constexpr int kFlushBlocks = 31;

// The draws of one replicate that the calling warp takes: Philox blocks p0,
// p0 + stride, ... below n/4 (p0 the lane's first block, stride a multiple of
// 32), then one ragged round.  WIDE: one 32-bit bin per word of hist (block
// form); else two 16-bit bins per word.  The lane's counts of the first four
// values are left in c[0..3] (not reduced across lanes).
template <bool WIDE, bool INL>
__device__ __forceinline__ void draw_queued(const uint64_t *sT, const uint32_t *sG, const uint32_t *sInc,
                                            const Law &law, const Cell &cell, uint32_t rep, const RoundKeys &rk,
                                            uint32_t *hist, int *s_count, uint64_t *spill, int64_t spill_capacity,
                                            int lane, const TailQueue *tq, uint64_t spill_pos0, uint64_t *queue,
                                            int64_t p0, int64_t stride, uint32_t c[4]) {
  const int64_t n = cell.n;
  const uint64_t xmin = cell.xmin;
  const uint32_t H = cell.H;
  // a table index b < L2: a shared atomic below H, else a spill
  auto bin = [&](uint32_t b) {
    if (b < H) {
      if (WIDE) atomicAdd(&hist[b], 1u);
      else atomicAdd(&hist[b >> 1], 1u << ((b & 1u) << 4));
    } else {
      const int slot = atomicAdd(s_count, 1);
      if (slot < spill_capacity) spill[slot] = xmin + b;
    }
  };
  auto m_of = [&](uint32_t h, uint64_t i) {
    return draw_m_full(h, i, rep, cell.cell_id, cell.purpose, rk.k[0], rk.k[1]);
  };
  // a draw whose value lies beyond the table: spilled as kTailTag | m for the
  // tail kernel
  auto spill_tagged = [&](uint64_t m) {
    const int slot = atomicAdd(s_count, 1);
    if (slot < spill_capacity) {
      spill[slot] = kTailTag | m;
      const unsigned q = atomicAdd(tq->count, 1u);
      if (q < tq->cap) {
        tq->pos[q] = spill_pos0 + (uint64_t)slot;
        tq->law[q] = cell.law;
      }
    }
  };
  // a queued draw (i << 32 | h) whose bucket holds several values: search the
  // table at m_first(h); its low word only when a threshold may lie in the
  // draw's interval of m or the answer lies beyond the table
  auto search = [&](uint64_t e) {
    const uint32_t h = (uint32_t)e;
    const uint32_t i0 =
        lookup_index<kFineBits>(sT, sG, law.T, law.L2, law.xmin_f, law.tail_c, law.tail_e, m_first(h));
    if (i0 < law.L2 && (i0 == 0 || table_at(sT, law.T, i0 - 1) > m_last(h))) {
      bin(i0);
      return;
    }
    const uint64_t m = m_of(h, e >> 32);
    const uint32_t b = lookup_index<kFineBits>(sT, sG, law.T, law.L2, law.xmin_f, law.tail_c, law.tail_e, m);
    if (b < law.L2) bin(b);
    else spill_tagged(m);
  };
  // queue entries: (h, i) as two 32-bit words, lane's entry k at queue[32 k + lane]
  uint2 *queue2 = reinterpret_cast<uint2 *>(queue);
  const uint32_t q0 = (uint32_t)__cvta_generic_to_shared(queue2 + lane);  // the lane's first entry
  uint32_t qa = q0;  // shared address of the lane's next free entry (rows of 256 bytes)
  const uint32_t q_full = q0 + 256u * (uint32_t)(kQCap - 4);  // beyond this a block's four draws may not fit
  const unsigned lt = (1u << lane) - 1u;
  // Each lane bins its own entries of single-valued buckets; entries of
  // multi-valued buckets are compacted to the front of the queue (row k is
  // read before the ballot of step k, and at most 32 (k + 1) entries are
  // compacted by then, so writes only reach rows already read) and searched
  // 32 at a time with every lane busy.
  auto drain = [&]() {
    const uint32_t qk = (qa - q0) >> 8;
    const uint32_t kmax = __reduce_max_sync(0xffffffffu, qk);
    uint32_t ns = 0;
    for (uint32_t k = 0; k < kmax; ++k) {
      const bool act = k < qk;
      const uint2 e = act ? queue2[32 * k + lane] : make_uint2(0u, 0u);
      const uint32_t gw = act ? sG[e.x >> (32 - kFineBits)] : 0u;
      const bool multi = act && (gw & kGuideMulti);
      if (act && !multi) {
        const uint32_t b = gw & kGuideIndex;
        if (b < law.L2) bin(b);
        else spill_tagged(m_of(e.x, e.y));
      }
      const unsigned bm = __ballot_sync(0xffffffffu, multi);
      if (multi) queue2[ns + __popc(bm & lt)] = e;
      ns += __popc(bm);
    }
    __syncwarp();
    for (uint32_t t0 = 0; t0 < ns; t0 += 32)
      if (t0 + lane < ns) {
        const uint2 e = queue2[t0 + lane];
        search(((uint64_t)e.y << 32) | e.x);
      }
    __syncwarp();
    qa = q0;
  };
  uint32_t acc = 0, c0 = 0, c1 = 0, c2 = 0, c3 = 0;
  auto flush = [&]() {
    c0 += acc & 0x7fu;
    c1 += (acc >> 8) & 0x7fu;
    c2 += (acc >> 16) & 0x7fu;
    c3 += (acc >> 24) & 0x7fu;
    acc = 0;
  };
  // the lane's copy of the increment table: entry of bucket j at inc_lane + 128 j
  const uint32_t inc_lane = (uint32_t)__cvta_generic_to_shared(sInc + lane);
  const uint32_t hist_s = (uint32_t)__cvta_generic_to_shared(hist);
  auto step = [&](uint32_t h, uint32_t i) {
    uint32_t e;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(e) : "r"(inc_lane + ((h >> (32 - kIncBits)) << 7)));
    acc += e;
    if (INL) {
      // heavy tails: nearly every warp has a lane beyond the first four
      // values at each step, so the step takes no branch.  The fine-guide
      // word is read for every draw; a single-valued bucket below H is binned
      // by a predicated shared reduction, and every other draw beyond the
      // first four values (multi-valued bucket, spill, beyond the table) is
      // queued for the drain, which bins or searches it.
      const uint32_t gw = sG[h >> (32 - kFineBits)], b = gw & kGuideIndex;
      const bool beyond = (int32_t)e < 0;
      const uint32_t direct = beyond && !(gw & kGuideMulti) && b < H;
      const uint32_t queued = beyond && !direct;
      const uint32_t addr = WIDE ? hist_s + 4u * b : hist_s + 2u * (b & ~1u);
      const uint32_t v = WIDE ? 1u : 1u << ((b & 1u) << 4);
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %0, 0;\n\t@p red.shared.add.u32 [%1], %2;\n\t}" ::"r"(direct),
          "r"(addr), "r"(v)
          : "memory");
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %0, 0;\n\t@p st.shared.v2.u32 [%1], {%2, %3};\n\t}" ::"r"(queued),
          "r"(qa), "r"(h), "r"(i)
          : "memory");
      qa += queued << 8;
    } else if ((int32_t)e < 0) {
      asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(qa), "r"(h), "r"(i) : "memory");
      qa += 256u;
    }
  };
  // full rounds (every lane has four valid draws: blocks below a multiple of
  // stride that is at most n/4), then one ragged round for the blocks left;
  // the trip counts are the same for every lane of the warp (n < 2^30)
  const uint32_t nn = (uint32_t)n, st = (uint32_t)stride;
  const uint32_t full = (nn >> 2) / st * st;
  uint32_t p = (uint32_t)p0;
  while (p < full) {
    const uint32_t pend = min(full, p - (uint32_t)lane + st * (uint32_t)kFlushBlocks);
    for (; p < pend; p += st) {
      const uint4 w = philox4x32_10_rk(make_uint4(p, rep, cell.cell_id, cell.purpose), rk);
      const uint32_t i0 = 4u * p;
      step(w.x, i0);
      step(w.y, i0 + 1u);
      step(w.z, i0 + 2u);
      step(w.w, i0 + 3u);
      if (__any_sync(0xffffffffu, qa > q_full)) drain();
    }
    flush();
  }
  if (4u * (p - (uint32_t)lane) < nn) {  // warp-uniform
    const uint4 w = philox4x32_10_rk(make_uint4(p, rep, cell.cell_id, cell.purpose), rk);
    const uint32_t i0 = 4u * p;
    if (i0 < nn) step(w.x, i0);
    if (i0 + 1u < nn) step(w.y, i0 + 1u);
    if (i0 + 2u < nn) step(w.z, i0 + 2u);
    if (i0 + 3u < nn) step(w.w, i0 + 3u);
    flush();
  }
  drain();
  c[0] = c0;
  c[1] = c1;
  c[2] = c2;
  c[3] = c3;
}

template <bool INL>
__device__ __forceinline__ int64_t draw_replicate_q(const uint64_t *sT, const uint32_t *sG, const uint32_t *sInc,
                                                    const Law &law, const Cell &cell, uint32_t rep,
                                                    const RoundKeys &rk, uint32_t *hist, int *s_count,
                                                    uint64_t *spill, int64_t spill_capacity, int lane,
                                                    const TailQueue *tq, uint64_t spill_pos0, uint64_t *queue) {
  const int words = (int)(cell.H / 2);
  for (int i = lane; i < words; i += 32) hist[i] = 0;
  if (lane == 0) *s_count = 0;
  __syncwarp();
  uint32_t c[4];
  draw_queued<false, INL>(sT, sG, sInc, law, cell, rep, rk, hist, s_count, spill, spill_capacity, lane, tq,
                          spill_pos0, queue, lane, 32, c);
  __syncwarp();
  const unsigned s0 = __reduce_add_sync(0xffffffffu, c[0]), s1 = __reduce_add_sync(0xffffffffu, c[1]);
  const unsigned s2 = __reduce_add_sync(0xffffffffu, c[2]), s3 = __reduce_add_sync(0xffffffffu, c[3]);
  if (lane == 0) {
    hist[0] += s0 | (s1 << 16);
    hist[1] += s2 | (s3 << 16);
  }
  __syncwarp();
  // largest bin hit: highest nonzero word, then its upper half
  int tw = -1;
  for (int i = lane; i < words; i += 32)
    if (hist[i]) tw = i;
  tw = __reduce_max_sync(0xffffffffu, (unsigned)(tw + 1)) - 1;
  if (tw < 0) return tw;
  return 2 * (int64_t)tw + ((hist[tw] >> 16) ? 1 : 0);
}

// INL: the launch's cells all bin in the draw loop (Cell::inline_bins), or none
// do; one kernel per mode keeps each draw loop's code on its own.
template <bool INL>
__global__ void __launch_bounds__(kAWarps * 32, kABlocksPerSM) sample_hist_kernel(SampleLaunch a) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t *sT = reinterpret_cast<uint64_t *>(smem);
  uint32_t *sG = reinterpret_cast<uint32_t *>(smem + kL1 * 8);
  uint32_t *sInc = reinterpret_cast<uint32_t *>(smem + kL1 * 8 + kFine * 4);
  uint32_t *sH = sInc + kIncBuckets * 32;
  uint64_t *sQ = reinterpret_cast<uint64_t *>(sH + kAWarps * (kHMax / 2));
  int *s_spill = reinterpret_cast<int *>(sQ + kAWarps * kQCap * 32);
  uint32_t *s_item = reinterpret_cast<uint32_t *>(s_spill + kAWarps);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(s_item + 2);
  StagedLaw staged{sT, sG, mbar, sInc};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t *hist = sH + warp * (kHMax / 2);
  uint64_t *queue = sQ + warp * kQCap * 32;
  const TailQueue tq{a.tq_pos, a.tq_law, a.tq_count, a.tq_cap};
  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    mbar_init(mbar + 1, 1);  // never arrived at: the wait-timeout test hook's flag
  }
  __syncthreads();
  uint32_t phase = 0, loaded = 0xffffffffu;
  for (;;) {
    if (threadIdx.x == 0)  // no further items once a wait has run out: records may be incomplete
      *s_item = (*(volatile unsigned int *)&a.ctr->status & kErrTimeout) ? a.nitems : atomicAdd(&a.ctr->work_next, 1u);
    __syncthreads();
    const uint32_t item = *s_item;
    if (item >= a.nitems) break;
    const WorkItem wi = a.items[item];
    const Cell cell = a.cells[wi.cell];
    const Law law = a.laws[cell.law];
    if (cell.law != loaded) {
      if (!stage_law(staged, law, phase, a.ctr)) return;
      loaded = cell.law;
    }
    for (int jj = 0; jj < kARepsPerWarp; ++jj) {
      const uint32_t j = warp + jj * kAWarps;  // strided: small items still use every warp
      if (j >= wi.nrep) break;
      const uint64_t pos0 = wi.spill_off + (uint64_t)j * cell.scap;
      const int64_t tmax = draw_replicate_q<INL>(sT, sG, sInc, law, cell, wi.r0 + j, a.rk, hist, &s_spill[warp],
                                            a.rec.spill + pos0, cell.scap, lane, &tq, pos0, queue);
      uint32_t *dense = reinterpret_cast<uint32_t *>(a.rec.dense + wi.dense_off + (uint64_t)j * cell.H);
      for (int64_t i = lane; i <= (tmax >> 1); i += 32) dense[i] = hist[i];
      if (lane == 0) a.rec.meta[wi.meta_off + j] = make_int2((int)tmax, s_spill[warp]);
      __syncwarp();
    }
    __syncthreads();
  }
}

// Block form (large n): a block per replicate, kHWide 32-bit bins in shared
// memory, the draws through the same increment table, per-lane queues and
// drains as the warp form (each warp a stride of the replicate's Philox blocks).
constexpr int kBlkThreads = 1024;
constexpr int kBlkWarps = kBlkThreads / 32;

template <bool INL>
__global__ void __launch_bounds__(kBlkThreads, 1) sample_block_kernel(SampleLaunch a) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t *sT = reinterpret_cast<uint64_t *>(smem);
  uint32_t *sG = reinterpret_cast<uint32_t *>(smem + kL1 * 8);
  uint32_t *sInc = reinterpret_cast<uint32_t *>(smem + kL1 * 8 + kFine * 4);
  uint32_t *hist = sInc + kIncBuckets * 32;
  uint64_t *sQ = reinterpret_cast<uint64_t *>(hist + kHWide);
  int *s_spill = reinterpret_cast<int *>(sQ + kBlkWarps * kQCap * 32);
  uint32_t *s_item = reinterpret_cast<uint32_t *>(s_spill + 1);
  int *s_tmax = reinterpret_cast<int *>(s_item + 1);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(s_tmax + 2);
  StagedLaw staged{sT, sG, mbar, sInc};
  const int lane = threadIdx.x & 31;
  uint64_t *queue = sQ + (threadIdx.x >> 5) * kQCap * 32;
  const TailQueue tq{a.tq_pos, a.tq_law, a.tq_count, a.tq_cap};
  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    mbar_init(mbar + 1, 1);  // never arrived at: the wait-timeout test hook's flag
  }
  __syncthreads();
  uint32_t phase = 0, loaded = 0xffffffffu;
  for (;;) {
    if (threadIdx.x == 0)  // no further items once a wait has run out: records may be incomplete
      *s_item = (*(volatile unsigned int *)&a.ctr->status & kErrTimeout) ? a.nitems : atomicAdd(&a.ctr->work_next, 1u);
    __syncthreads();
    const uint32_t item = *s_item;
    if (item >= a.nitems) break;
    const WorkItem wi = a.items[item];
    const Cell cell = a.cells[wi.cell];
    const Law law = a.laws[cell.law];
    if (cell.law != loaded) {
      if (!stage_law(staged, law, phase, a.ctr)) return;
      loaded = cell.law;
    }
    const uint32_t H = cell.H;
    for (uint32_t j = 0; j < wi.nrep; ++j) {
      for (uint32_t i = threadIdx.x; i < H; i += kBlkThreads) hist[i] = 0;
      if (threadIdx.x == 0) {
        *s_spill = 0;
        *s_tmax = -1;
      }
      __syncthreads();
      const uint64_t pos0 = wi.spill_off + (uint64_t)j * cell.scap;
      uint32_t c[4];
      draw_queued<true, INL>(sT, sG, sInc, law, cell, wi.r0 + j, a.rk, hist, s_spill, a.rec.spill + pos0, cell.scap,
                             lane, &tq, pos0, queue, threadIdx.x, kBlkThreads, c);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const unsigned t = __reduce_add_sync(0xffffffffu, c[q]);
        if (lane == 0 && t) atomicAdd(&hist[q], t);
      }
      __syncthreads();
      int tm = -1;
      for (uint32_t i = threadIdx.x; i < H; i += kBlkThreads)
        if (hist[i]) tm = (int)i;
      tm = (int)__reduce_max_sync(0xffffffffu, (unsigned)(tm + 1)) - 1;
      if (lane == 0 && tm >= 0) atomicMax(s_tmax, tm);
      __syncthreads();
      const int tmax = *s_tmax;
      uint32_t *dense = reinterpret_cast<uint32_t *>(a.rec.dense + wi.dense_off + (uint64_t)j * 2 * H);
      for (int i = threadIdx.x; i <= tmax; i += kBlkThreads) dense[i] = hist[i];
      if (threadIdx.x == 0) a.rec.meta[wi.meta_off + j] = make_int2(tmax, *s_spill);
      __syncthreads();
    }
  }
}

size_t block_sampler_smem_bytes() {
  return (size_t)kL1 * 8 + kFine * 4 + kIncBytes + (size_t)kHWide * 4 + (size_t)kBlkWarps * kQCap * 32 * 8 + 16 +
         16;
}

int block_sampler_blocks_per_sm() {
  int nb = 0;
  const size_t smem = block_sampler_smem_bytes();
  cudaFuncSetAttribute(sample_block_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(sample_block_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sample_block_kernel<false>, kBlkThreads, smem);
  return nb;
}

cudaError_t launch_sample_block(const SampleLaunch &a, bool inl, cudaStream_t st) {
  if (inl) sample_block_kernel<true><<<a.blocks, kBlkThreads, block_sampler_smem_bytes(), st>>>(a);
  else sample_block_kernel<false><<<a.blocks, kBlkThreads, block_sampler_smem_bytes(), st>>>(a);
  return cudaGetLastError();
}

// Beyond-table draws queued by the sampler: one thread per draw (full lanes),
// binary64 inversion written back into the record.
__global__ void __launch_bounds__(256) tail_queue_kernel(const Law *laws, TailQueue tq, uint64_t *spill,
                                                         Counters *ctr) {
  const unsigned cnt = *tq.count;
  const unsigned nq = cnt < tq.cap ? cnt : tq.cap;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
    const uint64_t pos = tq.pos[i];
    const uint64_t x = spill[pos];
    if (x & kTailTag) {
      bool beyond;
      spill[pos] = resolve_tagged(laws[tq.law[i]], x & ~kTailTag, &beyond);
      if (beyond) atomicAdd(&ctr->tail_draws, 1ull);
    }
  }
}

cudaError_t launch_tail_queue_raw(const Law *laws, uint64_t *pos, uint32_t *law, unsigned int *count,
                                  uint32_t cap, uint64_t *spill, Counters *ctr, int num_sms, cudaStream_t st) {
  const TailQueue tq{pos, law, count, cap};
  tail_queue_kernel<<<num_sms * 4, 256, 0, st>>>(laws, tq, spill, ctr);
  return cudaGetLastError();
}

size_t sample_kernel_smem_bytes() {
  return (size_t)kL1 * 8 + kFine * 4 + kIncBytes + (size_t)kAWarps * (kHMax / 2) * 4 +
         (size_t)kAWarps * kQCap * 32 * 8 + kAWarps * 4 + 8 + 16;
}

int sample_kernel_blocks_per_sm() {
  int nb = 0;
  const size_t smem = sample_kernel_smem_bytes();
  cudaFuncSetAttribute(sample_hist_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(sample_hist_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sample_hist_kernel<false>, kAWarps * 32, smem);
  return nb;
}

cudaError_t launch_sample_hist(const SampleLaunch &a, bool inl, cudaStream_t st) {
  if (inl) sample_hist_kernel<true><<<a.blocks, kAWarps * 32, sample_kernel_smem_bytes(), st>>>(a);
  else sample_hist_kernel<false><<<a.blocks, kAWarps * 32, sample_kernel_smem_bytes(), st>>>(a);
  return cudaGetLastError();
}

// Lane form (warp-form cells of histograms of at most kLaneSampleBins bins:
// small n, or light tails with up to kLaneSampleNMax values): one thread per
// replicate of a work item draws all its values, with no warp-wide steps.  A
// value's high word takes the lane's copy of the increment table (the first
// four values count in four 7-bit register fields, flushed every kFlushBlocks
// Philox blocks); any other draw reads the fine guide and, where the bucket holds
// several values, searches the staged table (its low word only when a
// threshold lies in the draw's interval or the answer lies beyond the table).
// Bins below H go to the thread's own histogram in shared memory (word w of
// thread t at w * kLaneSampleThreads + t, so a warp's accesses never share a
// bank), values beyond H to the record's spill slot, draws beyond the table to
// the tail queue.  The record (dense counts up to tmax, spills, meta) is the
// one the warp form writes: the finisher cannot tell the two apart.
constexpr int kLaneSampleThreads = kItemReps;
constexpr int kLaneSampleWords = kLaneSampleBins / 2;

size_t sample_lane_smem_bytes() {
  return (size_t)kL1 * 8 + kFine * 4 + kIncBytes + (size_t)kLaneSampleWords * kLaneSampleThreads * 4 + 16 + 16;
}

__global__ void __launch_bounds__(kLaneSampleThreads) sample_lane_kernel(SampleLaunch a) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t *sT = reinterpret_cast<uint64_t *>(smem);
  uint32_t *sG = reinterpret_cast<uint32_t *>(smem + kL1 * 8);
  uint32_t *sInc = reinterpret_cast<uint32_t *>(smem + kL1 * 8 + kFine * 4);
  uint32_t *sH = sInc + kIncBuckets * 32;
  uint32_t *s_item = sH + kLaneSampleWords * kLaneSampleThreads;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(s_item + 4);
  StagedLaw staged{sT, sG, mbar, sInc};
  const int t = threadIdx.x, lane = t & 31;
  uint32_t *hist = sH + t;  // word w at hist[w * kLaneSampleThreads]
  for (int w = 0; w < kLaneSampleWords; ++w) hist[w * kLaneSampleThreads] = 0;
  const TailQueue tq{a.tq_pos, a.tq_law, a.tq_count, a.tq_cap};
  if (t == 0) {
    mbar_init(mbar, 1);
    mbar_init(mbar + 1, 1);  // never arrived at: the wait-timeout test hook's flag
  }
  __syncthreads();
  uint32_t phase = 0, loaded = 0xffffffffu;
  const uint32_t *inc = sInc + lane;  // the lane's copy: bucket j at inc[32 j]
  for (;;) {
    if (t == 0)  // no further items once a wait has run out: records may be incomplete
      *s_item = (*(volatile unsigned int *)&a.ctr->status & kErrTimeout) ? a.nitems : atomicAdd(&a.ctr->work_next, 1u);
    __syncthreads();
    const uint32_t item = *s_item;
    if (item >= a.nitems) break;
    const WorkItem wi = a.items[item];
    const Cell cell = a.cells[wi.cell];
    const Law law = a.laws[cell.law];
    if (cell.law != loaded) {
      if (!stage_law(staged, law, phase, a.ctr)) return;
      loaded = cell.law;
    }
    if ((uint32_t)t < wi.nrep) {
      const uint32_t j = (uint32_t)t, rep = wi.r0 + j;
      const uint32_t n = (uint32_t)cell.n, H = cell.H;
      const uint64_t pos0 = wi.spill_off + (uint64_t)j * cell.scap;
      uint64_t *spill = a.rec.spill + pos0;
      int s = 0;  // spills (all of them: a count beyond the slot makes the finisher draw again)
      uint32_t acc = 0;
      auto spill_value = [&](uint64_t v) {
        if (s < (int)cell.scap) spill[s] = v;
        ++s;
      };
      auto bin = [&](uint32_t b) {
        if (b < H) hist[(b >> 1) * kLaneSampleThreads] += 1u << ((b & 1u) << 4);
        else spill_value(cell.xmin + b);
      };
      auto tagged = [&](uint64_t m) {
        if (s < (int)cell.scap) {
          const unsigned q = atomicAdd(tq.count, 1u);
          if (q < tq.cap) {
            tq.pos[q] = pos0 + (uint64_t)s;
            tq.law[q] = cell.law;
          }
        }
        spill_value(kTailTag | m);
      };
      auto step = [&](uint32_t h, uint32_t i) {
        const uint32_t e = inc[(h >> (32 - kIncBits)) << 5];
        acc += e;
        if ((int32_t)e >= 0) return;
        const uint32_t gw = sG[h >> (32 - kFineBits)];
        uint32_t b = gw & kGuideIndex;
        if (gw & kGuideMulti) {
          b = lookup_index<kFineBits>(sT, sG, law.T, law.L2, law.xmin_f, law.tail_c, law.tail_e, m_first(h));
          if (b < law.L2 && (b == 0 || table_at(sT, law.T, b - 1) > m_last(h))) {
            bin(b);
            return;
          }
        } else if (b < law.L2) {
          bin(b);
          return;
        }
        const uint64_t m = draw_m_full(h, i, rep, cell.cell_id, cell.purpose, a.rk.k[0], a.rk.k[1]);
        b = lookup_index<kFineBits>(sT, sG, law.T, law.L2, law.xmin_f, law.tail_c, law.tail_e, m);
        if (b < law.L2) bin(b);
        else tagged(m);
      };
      // the first four values' counts (7-bit fields) into bins 0..3, every
      // kFlushBlocks Philox blocks (at most 124 increments)
      auto flush = [&]() {
        hist[0] += (acc & 0x7fu) | (((acc >> 8) & 0x7fu) << 16);
        hist[kLaneSampleThreads] += ((acc >> 16) & 0x7fu) | (((acc >> 24) & 0x7fu) << 16);
        acc = 0;
      };
      for (uint32_t p = 0; 4u * p < n; ++p) {
        const uint4 w = philox4x32_10_rk(make_uint4(p, rep, cell.cell_id, cell.purpose), a.rk);
        const uint32_t i0 = 4u * p;
        step(w.x, i0);
        if (i0 + 1u < n) step(w.y, i0 + 1u);
        if (i0 + 2u < n) step(w.z, i0 + 2u);
        if (i0 + 3u < n) step(w.w, i0 + 3u);
        if (p % kFlushBlocks == kFlushBlocks - 1) flush();
      }
      flush();
      int tw = (int)(H >> 1) - 1;
      while (tw >= 0 && hist[tw * kLaneSampleThreads] == 0u) --tw;
      const int tmax = tw < 0 ? -1 : 2 * tw + ((hist[tw * kLaneSampleThreads] >> 16) ? 1 : 0);
      uint32_t *dense = reinterpret_cast<uint32_t *>(a.rec.dense + wi.dense_off + (uint64_t)j * H);
      for (int w = 0; w <= tw; ++w) {
        dense[w] = hist[w * kLaneSampleThreads];
        hist[w * kLaneSampleThreads] = 0;
      }
      a.rec.meta[wi.meta_off + j] = make_int2(tmax, s);
    }
    __syncthreads();
  }
}

int sample_lane_blocks_per_sm() {
  int nb = 0;
  const size_t smem = sample_lane_smem_bytes();
  cudaFuncSetAttribute(sample_lane_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sample_lane_kernel, kLaneSampleThreads, smem);
  return nb;
}

cudaError_t launch_sample_lane(const SampleLaunch &a, cudaStream_t st) {
  sample_lane_kernel<<<a.blocks, kLaneSampleThreads, sample_lane_smem_bytes(), st>>>(a);
  return cudaGetLastError();
}

// Copy the dense counts 0..tmax of a warp-form record (16-byte aligned, H >= 32
// bins) to the warp's shared memory with 16-byte loads, so that the scans
// below read them on chip instead of one dependent global load per bin.
__device__ __forceinline__ const uint16_t *stage_dense(const uint16_t *src, int64_t tmax, uint32_t *onchip,
                                                       int lane) {
  uint16_t *dst = reinterpret_cast<uint16_t *>(onchip);
  const int64_t nvec = (tmax + 8) >> 3;
  for (int64_t v = lane; v < nvec; v += 32)
    reinterpret_cast<uint4 *>(dst)[v] = reinterpret_cast<const uint4 *>(src)[v];
  __syncwarp();
  return dst;
}

// Small replicates (warp form, largest bin below the cell's lane_bins, at
// most kLaneSpills spills that fit the record's slot) are finished by one lane
// each: the log-sum and the KS scan run serially over the replicate's dense
// counts and then its spills, sorted in place, with no warp reductions.  Same
// arithmetic as the warp-cooperative path, summed in bin order and value
// order.

// A lane's spills: draws left tagged beyond the table resolved, then sorted
// ascending in place (odd-even transposition network over kLaneSpills
// registers, unused ones padded with the largest key).
__device__ __forceinline__ void lane_sort_spills(uint64_t *sp, int s, const Law &law, Counters *ctr,
                                                 bool tags_left) {
  for (int k = 0; tags_left && k < s; ++k) {
    const uint64_t x = sp[k];
    if (x & kTailTag) {
      bool beyond;
      sp[k] = resolve_tagged(law, x & ~kTailTag, &beyond);
      if (beyond) atomicAdd(&ctr->tail_draws, 1ull);
    }
  }
  uint64_t v[kLaneSpills];
#pragma unroll
  for (int k = 0; k < kLaneSpills; ++k) v[k] = k < s ? sp[k] : ~0ull;
#pragma unroll
  for (int r = 0; r < kLaneSpills; ++r) {
#pragma unroll
    for (int k = r & 1; k + 1 < kLaneSpills; k += 2) {
      const uint64_t lo = v[k] < v[k + 1] ? v[k] : v[k + 1], hi = v[k] < v[k + 1] ? v[k + 1] : v[k];
      v[k] = lo;
      v[k + 1] = hi;
    }
  }
#pragma unroll
  for (int k = 0; k < kLaneSpills; ++k)
    if (k < s) sp[k] = v[k];
}

template <bool F32>
__device__ __forceinline__ double lane_logsum_spills(const uint64_t *sp, int s) {
  if (!F32) {
    double acc = 0.0;
    for (int k = 0; k < s; ++k) acc += log((double)sp[k]);
    return acc;
  }
  float Sh = 0.0f, Sl = 0.0f;
  for (int k = 0; k < s; ++k) {
    float vh, vl;
    ln_u64_ff(sp[k], vh, vl);
    ff_add(Sh, Sl, vh, vl);
  }
  return (double)Sh + (double)Sl;
}

// KS candidates of a lane's sorted spills (every value beyond the dense bins,
// n - s values below them), one per run of equal values.
template <bool F32>
__device__ __forceinline__ double lane_ks_spills(const uint64_t *sp, int s, int64_t n, const FitOut &f,
                                                 double best) {
  int64_t Cb = n - s;
  const double invZ = F32 ? 0.0 : 1.0 / f.Z, inv_n = F32 ? 0.0 : 1.0 / (double)n;
  const float inv_nf = 1.0f / (float)(uint32_t)n;
  for (int k = 0; k < s; ++k) {
    const uint64_t v = sp[k];
    if (k + 1 < s && sp[k + 1] == v) continue;
    const int64_t Ca = n - s + k + 1;
    if (F32) best = fmax(best, (double)spill_point_f32(v, Ca, Cb, inv_nf, f));
    else best = fmax(best, spill_point_f64(v, Ca, Cb, f.ahat, invZ, inv_n));
    Cb = Ca;
  }
  return best;
}

template <bool F32>
__device__ __forceinline__ double lane_logsum(const uint16_t *dense, int64_t tmax, const Law &law, const float *lnHi,
                                              const float *lnLo) {
  if (!F32) {
    double acc = 0.0;
    for (int64_t i = 0; i <= tmax; ++i) acc += (double)dense[i] * law.lnT[i];
    return acc;
  }
  float Lh = 0.0f, Ll = 0.0f;
#pragma unroll 4
  for (int64_t i = 0; i <= tmax; ++i) {
    const float c = (float)dense[i];
    const float ph = c * lnHi[i];
    const float pe = fmaf(c, lnHi[i], -ph) + c * lnLo[i];
    ff_add(Lh, Ll, ph, pe);
  }
  return (double)Lh + (double)Ll;
}

template <bool F32>
__device__ __forceinline__ double lane_ks(const uint16_t *dense, int64_t tmax, int64_t n, const FitOut &f,
                                          const Law &law, const float *lnHi, const float *lnLo) {
  if (!F32) {
    const double invZ = 1.0 / f.Z, inv_n = 1.0 / (double)n;
    double F = 0.0, best = 0.0;
    int64_t C = 0;
    for (int64_t i = 0; i <= tmax; ++i) {
      F += exp(-f.ahat * law.lnT[i]) * invZ;
      C += dense[i];
      best = fmax(best, fabs(F - (double)C * inv_n));
    }
    return best;
  }
  const float inv_n = 1.0f / (float)(uint32_t)n;
  float Fh = 0.0f, Fl = 0.0f, best = 0.0f;
  uint32_t C = 0;
#pragma unroll 4
  for (int64_t i = 0; i <= tmax; ++i) {
    ff_add(Fh, Fl, exp_neg_prod(f.a_hi, f.a_lo, lnHi[i], lnLo[i]) * f.invZ, 0.0f);
    C += dense[i];
    best = fmaxf(best, fabsf(Fh - (float)C * inv_n));
  }
  return (double)best;
}

template <bool F32>
__global__ void __launch_bounds__(kWarps * 32, F32 ? PL_FIN_MIN_BLOCKS_F32 : PL_FIN_MIN_BLOCKS_F64)
    finish_kernel(FinishLaunch a) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t *sT = reinterpret_cast<uint64_t *>(smem);
  uint32_t *sG = reinterpret_cast<uint32_t *>(smem + kL1 * 8);
  uint32_t *sH = reinterpret_cast<uint32_t *>(smem + kL1 * 8 + kGuide * 4);
  int *s_spill = reinterpret_cast<int *>(smem + kL1 * 8 + kGuide * 4 + kWarps * kHMax * 4);
  uint32_t *s_item = reinterpret_cast<uint32_t *>(s_spill + kWarps);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + kL1 * 8 + kGuide * 4 + kWarps * kHMax * 4 + 64);
  float *sLn = reinterpret_cast<float *>(smem + kL1 * 8 + kGuide * 4 + kWarps * kHMax * 4 + 128);
  StagedLaw staged{sT, sG, mbar, nullptr, F32 ? sLn : nullptr};

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t *hist = sH + warp * kHMax;
  const size_t slot = (size_t)blockIdx.x * kWarps + warp;
  uint64_t *spill = reinterpret_cast<uint64_t *>(a.scratch + slot * (a.spill_cap * 8 + a.arena_bytes));
  uint8_t *arena = reinterpret_cast<uint8_t *>(spill + a.spill_cap);

  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    mbar_init(mbar + 1, 1);  // never arrived at: the wait-timeout test hook's flag
  }
  __syncthreads();
  uint32_t phase = 0, loaded = 0xffffffffu;
  const bool tags_left = !a.tq_count || *a.tq_count > a.tq_cap;

  for (;;) {
    if (threadIdx.x == 0)  // no further items once a wait has run out: records may be incomplete
      *s_item = (*(volatile unsigned int *)&a.ctr->status & kErrTimeout) ? a.nitems : atomicAdd(&a.ctr->work_next, 1u);
    __syncthreads();
    const uint32_t item = *s_item;
    if (item >= a.nitems) break;
    const WorkItem wi = a.items[item];
    const Cell cell = a.cells[wi.cell];
    const CellConst cc = a.consts[wi.cell];
    const Law law = a.laws[cell.law];
    if (cell.law != loaded) {
      if (!stage_law(staged, law, phase, a.ctr)) return;
      loaded = cell.law;
    }
    // the item's replicates spread evenly over the warps (at most 32 each)
    // binary32 log splits: the staged copy for warp-form cells (bins < kHMax)
    const float *lnHi = cell.wide ? law.lnT_hi : sLn, *lnLo = cell.wide ? law.lnT_lo : sLn + kHMax;
    const int per_warp = (int)((wi.nrep + kWarps - 1) / kWarps);
    const int j0 = warp * per_warp;
    const int nb = (int)min((int64_t)per_warp, (int64_t)wi.nrep - j0);
    if (nb > 0) {
      const int64_t n = cell.n;
      const uint64_t xmin = cell.xmin;
      // per-lane record of replicate j0 + lane
      double myL = 0.0;
      int64_t my_tmax = -1, my_nsd = 0;
      size_t my_off = 0;
      size_t arena_off = 0;
      int done = 0;
      const FitTable &ft = a.fits[cell.fit];
#ifdef PL_PHASE_TIMING
      long long pt_ = clock64();
#endif
      const uint64_t dslot = (uint64_t)cell.H * (cell.wide ? 2 : 1);
      const uint16_t *my_dense = a.rec.dense + wi.dense_off + (uint64_t)(j0 + (lane < nb ? lane : 0)) * dslot;
      bool simple = false;
      int my_s = 0;
      const uint64_t *my_sp = a.rec.spill + wi.spill_off + (uint64_t)(j0 + (lane < nb ? lane : 0)) * cell.scap;
      if (!cell.wide && lane < nb) {
        const int2 m = a.rec.meta[wi.meta_off + j0 + lane];
        // (a slot holds at least min(n, kLaneSpills) entries, so these never overflow)
        simple = m.y >= 0 && m.y <= kLaneSpills && m.x >= 0 && (uint32_t)m.x < cell.lane_bins;
        if (simple) {
          my_tmax = m.x;
          my_s = m.y;
          myL = lane_logsum<F32>(my_dense, my_tmax, law, lnHi, lnLo);
          if (my_s > 0) {
            lane_sort_spills(const_cast<uint64_t *>(my_sp), my_s, law, a.ctr, tags_left);
            myL += lane_logsum_spills<F32>(my_sp, my_s);
          }
          if ((int64_t)my_dense[0] == n) myL += cc.ln_allmin;
        }
      }
      const unsigned smask = __ballot_sync(0xffffffffu, simple);
      auto finish = [&](int b0, int b1) {
        PL_PHASE(6);
        const bool mine = lane >= b0 && lane < b1;
        // lanes without a replicate fit a stand-in log-sum (mean log excess 1/2)
        const double Lfit = mine ? myL : (double)n * (cc.ln_xmin + 0.5);
        const FitOut fo = fit_lanes(Lfit, n, xmin, cc, ft, law.lnT, F32, a.ctr);
        PL_PHASE(3);
        double myD = 0.0;
        for (int r = b0; r < b1; ++r) {
          if ((smask >> r) & 1u) continue;
          const FitOut fr = shfl_fit(fo, r);
          const int64_t tm = __shfl_sync(0xffffffffu, my_tmax, r);
          const int64_t ns = __shfl_sync(0xffffffffu, my_nsd, r);
          const size_t off = __shfl_sync(0xffffffffu, my_off, r);
          const uint16_t *dense =
              a.rec.dense + wi.dense_off + (uint64_t)(j0 + r) * (uint64_t)cell.H * (cell.wide ? 2 : 1);
          const uint64_t *pr = reinterpret_cast<const uint64_t *>(arena + off);
          double D;
          if (cell.wide) {
            D = ks_warp<F32, uint32_t>(reinterpret_cast<const uint32_t *>(dense), tm, pr, ns, n, xmin, fr, law.lnT,
                                       lnHi, lnLo, lane);
          } else {
            const uint16_t *sd = stage_dense(dense, tm, hist, lane);
            D = ks_warp<F32, uint16_t>(sd, tm, pr, ns, n, xmin, fr, law.lnT, lnHi, lnLo, lane);
            __syncwarp();
          }
          if (lane == r) myD = D;
        }
        if (mine && simple) {
          myD = lane_ks<F32>(my_dense, my_tmax, n, fo, law, lnHi, lnLo);
          if (my_s > 0) myD = lane_ks_spills<F32>(my_sp, my_s, n, fo, myD);
        }
        PL_PHASE(4);
        if (mine) {
          const int64_t o = cell.out_off + wi.r0 + j0 + lane;
          if (F32) reinterpret_cast<float *>(a.D_out)[o] = (float)myD;
          else reinterpret_cast<double *>(a.D_out)[o] = myD;
          if (a.A_out) a.A_out[o] = fo.ahat;
        }
      };

      for (int r = 0; r < nb; ++r) {
        if ((smask >> r) & 1u) continue;  // finished by its lane
        const uint32_t j = (uint32_t)(j0 + r);
        const int2 meta = a.rec.meta[wi.meta_off + j];
        int64_t tmax = meta.x;
        const int64_t s = meta.y;
        uint16_t *dense = a.rec.dense + wi.dense_off + (uint64_t)j * dslot;
        uint32_t *dense32 = cell.wide ? reinterpret_cast<uint32_t *>(dense) : nullptr;
        uint64_t *sp = a.rec.spill + wi.spill_off + (uint64_t)j * cell.scap;
        bool tags = tags_left;
        if (s > (int64_t)cell.scap) {
          tags = true;
          // the record's spill slot overflowed: draw this replicate again with
          // the warp's global spill buffer (same stream, same values); the
          // block form's histogram is rebuilt in place in the record
          if (lane == 0) atomicAdd(&a.ctr->resampled, 1ull);
          if (cell.wide) {
            tmax = draw_replicate<false>(sT, sG, law, cell, wi.r0 + j, a.rk, dense32, &s_spill[warp], spill,
                                         (int64_t)a.spill_cap, lane);
          } else {
            tmax = draw_replicate<false>(sT, sG, law, cell, wi.r0 + j, a.rk, hist, &s_spill[warp], spill,
                                         (int64_t)a.spill_cap, lane);
            for (int64_t i = lane; i <= tmax; i += 32) dense[i] = (uint16_t)hist[i];
          }
          __syncwarp();
          sp = spill;
          if (s > (int64_t)a.spill_cap) {  // beyond every buffer: report, leave this batch
            if (lane == 0) atomicOr(&a.ctr->status, kErrArena);
            break;
          }
        }
        PL_PHASE(0);
        // resolve the draws that fell beyond the threshold table (binary64 inversion)
        for (int64_t k = lane; tags && k < s; k += 32) {
          const uint64_t x = sp[k];
          if (x & kTailTag) {
            bool beyond;
            sp[k] = resolve_tagged(law, x & ~kTailTag, &beyond);
            if (beyond) atomicAdd(&a.ctr->tail_draws, 1ull);
          }
        }
        __syncwarp();
        // log-sum  L = sum ln x_i  (+ ln((xmin+1)/xmin) if every x_i = xmin):
        // dense part here, spill part after sorting (so that the summation
        // order, and hence the rounding, never depends on the spill order)
        double L;
        float Lh = 0.0f, Ll = 0.0f;
        const uint16_t *dsrc = dense32 ? dense : stage_dense(dense, tmax, hist, lane);
        if (!F32) {
          double acc = 0.0;
          for (int64_t i = lane; i <= tmax; i += 32)
            acc += (double)(dense32 ? dense32[i] : (uint32_t)dsrc[i]) * law.lnT[i];
          L = warp_sum(acc);
        } else {
          for (int64_t i = lane; i <= tmax; i += 32) {
            const float c = (float)(dense32 ? dense32[i] : (uint32_t)dsrc[i]);
            const float ph = c * lnHi[i];
            const float pe = fmaf(c, lnHi[i], -ph) + c * lnLo[i];
            ff_add(Lh, Ll, ph, pe);
          }
          L = 0.0;
        }
        const bool allmin = tmax >= 0 && (int64_t)(dense32 ? dense32[0] : (uint32_t)dsrc[0]) == n;
        __syncwarp();  // the staged copy is overwritten by the spill sort below
        PL_PHASE(1);
        // arena space for this replicate's spill pairs; run phases 2-3 early if full
        const size_t need = (size_t)s * 16;
        if (arena_off + need > a.arena_bytes) {
          if (done < r) finish(done, r);
          done = r;
          arena_off = 0;
          if (need > a.arena_bytes) {  // unreachable: the host sizes the arena for one replicate
            if (lane == 0) atomicOr(&a.ctr->status, kErrArena);
            break;                     // leave this batch; the block barrier below still meets
          }
        }
        uint64_t *pairs = reinterpret_cast<uint64_t *>(arena + arena_off);
        const int64_t nsd = spill_compact(sp, hist, s, pairs, lane, a.ctr);
        if (!F32) {
          double acc = 0.0;
          for (int64_t k = lane; k < nsd; k += 32) acc += (double)pairs[2 * k + 1] * log((double)pairs[2 * k]);
          L += warp_sum(acc);
        } else {
          for (int64_t k = lane; k < nsd; k += 32) {
            float vh, vl;
            ln_u64_ff(pairs[2 * k], vh, vl);
            const float c = (float)(uint32_t)pairs[2 * k + 1];
            const float ph = c * vh;
            ff_add(Lh, Ll, ph, fmaf(c, vh, -ph) + c * vl);
          }
          warp_sum_ff(Lh, Ll);
          L = (double)Lh + (double)Ll;
        }
        if (allmin) L += cc.ln_allmin;
        if (lane == r) {
          myL = L;
          my_tmax = tmax;
          my_nsd = nsd;
          my_off = arena_off;
        }
        arena_off += (size_t)nsd * 16;
        __syncwarp();
        PL_PHASE(2);
      }
      if (done < nb) finish(done, nb);
    }
    __syncthreads();
  }
}

size_t finish_kernel_smem_bytes() {
  return (size_t)kL1 * 8 + kGuide * 4 + (size_t)kWarps * kHMax * 4 + 128 + 2 * (size_t)kLnBytes;
}

int finish_kernel_blocks_per_sm(bool f32) {
  int nb = 0;
  const size_t smem = finish_kernel_smem_bytes();
  if (f32) {
    cudaFuncSetAttribute(finish_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, finish_kernel<true>, kWarps * 32, smem);
  } else {
    cudaFuncSetAttribute(finish_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, finish_kernel<false>, kWarps * 32, smem);
  }
  return nb;
}

cudaError_t launch_finish(const FinishLaunch &a, bool f32, cudaStream_t st) {
  const size_t smem = finish_kernel_smem_bytes();
  if (f32) finish_kernel<true><<<a.blocks, kWarps * 32, smem, st>>>(a);
  else finish_kernel<false><<<a.blocks, kWarps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

// ===========================================================================
// One data set (pl_fit_mle, pl_ks_stat, the observed side of the bootstrap):
// one block; dense bins [xmin, xmin + kHData) in shared memory, larger values
// spilled to global memory and sorted there.
constexpr int kHData = 8192;

template <bool F32>
__global__ void __launch_bounds__(1024) dataset_kernel(const int32_t *x, int64_t n, uint64_t xmin,
                                                       bool fit, double alpha_in, const Law *lnlaw,
                                                       CellConst cc, uint64_t *spill,
                                                       uint64_t *pairs, double *out, Counters *ctr) {
  __shared__ uint32_t hist[kHData];
  __shared__ unsigned long long s_cnt;
  __shared__ int s_bad;
  __shared__ long long s_tmax;
  __shared__ double s_red[32];
  const Law law = *lnlaw;
  for (int i = threadIdx.x; i < kHData; i += blockDim.x) hist[i] = 0;
  if (threadIdx.x == 0) {
    s_cnt = 0;
    s_bad = 0;
    s_tmax = -1;
  }
  __syncthreads();
  long long lmax = -1;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int32_t v = x[i];
    if (v < 1 || (uint64_t)v < xmin) {
      s_bad = 1;
      continue;
    }
    const uint64_t b = (uint64_t)v - xmin;
    if (b < (uint64_t)kHData) {
      atomicAdd(&hist[b], 1u);
      if ((long long)b > lmax) lmax = (long long)b;
    } else {
      spill[atomicAdd(&s_cnt, 1ull)] = (uint64_t)v;
    }
  }
  atomicMax(&s_tmax, lmax);
  __syncthreads();
  if (s_bad) {
    if (threadIdx.x == 0) {
      atomicOr(&ctr->status, kErrData);
      out[0] = out[1] = out[2] = __longlong_as_double(0x7ff8000000000000ll);
    }
    return;
  }
  const int64_t s = (int64_t)s_cnt;
  const int64_t tmax = s_tmax;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // log-sum (binary64 here: one data set, no bulk)
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i <= tmax; i += blockDim.x) acc += (double)hist[i] * law.lnT[i];
  acc = warp_sum(acc);
  if (lane == 0) s_red[warp] = acc;
  // sort the spills in global memory (block bitonic), padded to a power of two
  uint32_t P = 1;
  while ((int64_t)P < s) P <<= 1;
  for (uint32_t i = (uint32_t)s + threadIdx.x; s > 0 && i < P; i += blockDim.x) spill[i] = ~0ull;
  __syncthreads();
  if (s > 1) {
    for (uint32_t k = 2; k <= P; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
          const uint32_t l = i ^ j;
          if (l > i) {
            const uint64_t u = spill[i], w = spill[l];
            if ((u > w) == ((i & k) == 0)) {
              spill[i] = w;
              spill[l] = u;
            }
          }
        }
        __syncthreads();
      }
    }
  }
  if (warp == 0) {
    double L = lane < (int)(blockDim.x / 32) ? s_red[lane] : 0.0;
    L = warp_sum(L);
    if (hist[0] == (uint64_t)n) L += cc.ln_allmin;
    // run-length encode the sorted spills (warp 0)
    int64_t base = 0;
    for (int64_t i0 = 0; i0 < s; i0 += 32) {
      const int64_t i = i0 + lane;
      const bool ok = i < s;
      const uint64_t v = ok ? spill[i] : 0;
      const bool start = ok && (i == 0 || spill[i - 1] != v);
      const unsigned bal = __ballot_sync(0xffffffffu, start);
      const int rank = __popc(bal & ((1u << lane) - 1u));
      if (start) {
        pairs[2 * (base + rank)] = v;
        pairs[2 * (base + rank) + 1] = (uint64_t)i;
      }
      base += __popc(bal);
    }
    __syncwarp();
    for (int64_t k0 = 0; k0 < base; k0 += 32) {
      const int64_t k = k0 + lane;
      uint64_t cnt = 0;
      if (k < base) {
        const uint64_t st = pairs[2 * k + 1];
        const uint64_t en = (k + 1 < base) ? pairs[2 * (k + 1) + 1] : (uint64_t)s;
        cnt = en - st;
      }
      __syncwarp();
      if (k < base) pairs[2 * k + 1] = cnt;
      __syncwarp();
    }
    {  // spill part of the log-sum, over the sorted distinct values
      double sacc = 0.0;
      for (int64_t k = lane; k < base; k += 32) sacc += (double)pairs[2 * k + 1] * log((double)pairs[2 * k]);
      L += warp_sum(sacc);
    }
    FitOut fo{};
    if (fit) {
      if (lane == 0) fo = fit_from_logsum(L, n, xmin, cc, law.lnT, F32, ctr);
      fo = shfl_fit(fo, 0);
    } else {
      fo.ahat = alpha_in;
      if (lane == 0) {
        double z0;
        hurwitz_em<0, false>(alpha_in, (double)xmin, &z0, law.lnT, (double)xmin, kLnTable);
        fo.Z = z0;
        fo.a_hi = (float)alpha_in;
        fo.a_lo = (float)(alpha_in - (double)fo.a_hi);
        fo.invZ = (float)(1.0 / z0);
        fo.lnZ = (float)log(z0);
        const double lncd = log((alpha_in - 1.0) * z0);
        fo.lnc = (float)lncd;
        fo.lnc_lo = (float)(lncd - (double)fo.lnc);
      }
      fo = shfl_fit(fo, 0);
    }
    const double D =
        ks_warp<F32, uint32_t>(hist, tmax, pairs, base, n, xmin, fo, law.lnT, law.lnT_hi, law.lnT_lo, lane);
    if (lane == 0) {
      out[0] = fo.ahat;
      out[1] = D;
      out[2] = fo.Z;
    }
  }
}

cudaError_t launch_dataset(const int32_t *x, int64_t n, uint64_t xmin, bool fit, double alpha,
                           const Law *lnlaw, CellConst cc, bool f32, uint64_t *spill,
                           uint64_t *pairs, double *out, Counters *ctr, cudaStream_t st) {
  if (f32) dataset_kernel<true><<<1, 1024, 0, st>>>(x, n, xmin, fit, alpha, lnlaw, cc, spill, pairs, out, ctr);
  else dataset_kernel<false><<<1, 1024, 0, st>>>(x, n, xmin, fit, alpha, lnlaw, cc, spill, pairs, out, ctr);
  return cudaGetLastError();
}

// ===========================================================================
// Radix select: exact order statistic of non-negative floating-point keys
// (their bit patterns order like the values), 8 bits per pass from the top.
template <typename K>
__global__ void __launch_bounds__(1024) select_kernel(const K *keys, const int64_t *off,
                                                      const int64_t *Rs, const int64_t *rank,
                                                      int nq, double *out) {
  __shared__ unsigned int h[256];
  __shared__ K s_prefix;
  __shared__ long long s_k;
  const int c = blockIdx.x, j = blockIdx.y;
  const K *x = keys + off[c];
  const int64_t R = Rs[c];
  if (threadIdx.x == 0) {
    s_prefix = 0;
    s_k = rank[c * nq + j];
  }
  K mask = 0;
  for (int shift = (int)sizeof(K) * 8 - 8; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const K prefix = s_prefix;
    for (int64_t i = threadIdx.x; i < R; i += blockDim.x) {
      const K v = x[i];
      if ((v & mask) == prefix) atomicAdd(&h[(unsigned)((v >> shift) & 0xff)], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long k = s_k;
      int d = 0;
      for (; d < 255; ++d) {
        if (k < (long long)h[d]) break;
        k -= h[d];
      }
      s_k = k;
      s_prefix = prefix | ((K)d << shift);
    }
    mask |= (K)0xff << shift;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const K v = s_prefix;
    double r;
    if (sizeof(K) == 8) r = __longlong_as_double((long long)v);
    else r = (double)__uint_as_float((unsigned)v);
    out[c * nq + j] = r;
  }
}

cudaError_t launch_select(const void *keys, bool f32, const int64_t *off, const int64_t *R,
                          const int64_t *rank, int ncells, int nq, double *out, cudaStream_t st) {
  const dim3 grid(ncells, nq);
  if (f32) select_kernel<uint32_t><<<grid, 1024, 0, st>>>((const uint32_t *)keys, off, R, rank, nq, out);
  else select_kernel<uint64_t><<<grid, 1024, 0, st>>>((const uint64_t *)keys, off, R, rank, nq, out);
  return cudaGetLastError();
}

// ===========================================================================
__global__ void count_ge_kernel(const void *D, bool f32, int64_t B, const double *D_obs, double *p) {
  __shared__ unsigned long long cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  const double d0 = *D_obs;
  unsigned long long local = 0;
  for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
    const double v = f32 ? (double)reinterpret_cast<const float *>(D)[b]
                         : reinterpret_cast<const double *>(D)[b];
    local += (f32 ? (float)v >= (float)d0 : v >= d0) ? 1ull : 0ull;
  }
  atomicAdd(&cnt, local);
  __syncthreads();
  if (threadIdx.x == 0) *p = (double)cnt / (double)B;
}

cudaError_t launch_count_ge(const void *D, bool f32, int64_t B, const double *D_obs, double *p,
                            cudaStream_t st) {
  count_ge_kernel<<<1, 1024, 0, st>>>(D, f32, B, D_obs, p);
  return cudaGetLastError();
}

}  // namespace pl
