// pl_device.cuh -- device building blocks of the sm_103a KS-cutoff kernels.
//
// Philox4x32-10 streams, the Hurwitz zeta by Euler-Maclaurin (binary64 with
// s-derivatives, binary32 for the bulk KS tail), the integer threshold table
// that inverts the CDF of the law p(k) = k^-alpha / zeta(alpha, xmin)
// (Eq. 1 with a lower end xmin), the FP64 tail inversion beyond the table,
// and warp-level scans and sorts.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pl {

// ---------------------------------------------------------------------------
// Sizes of the on-chip structures.
constexpr uint64_t kXCap = 1ull << 62;      // simulated values saturate here
#ifndef PL_L1_ENTRIES
#define PL_L1_ENTRIES 2048
#endif
// finisher blocks per SM the compiler must fit (binary32 form / binary64
// form): two (128 registers, few spills) ran faster than three (80
// registers, more spills) on GB300, heavy-tailed cells most
#ifndef PL_FIN_MIN_BLOCKS_F32
#define PL_FIN_MIN_BLOCKS_F32 2
#endif
#ifndef PL_FIN_MIN_BLOCKS_F64
#define PL_FIN_MIN_BLOCKS_F64 2
#endif
constexpr int kL1 = PL_L1_ENTRIES;          // thresholds staged in shared memory
constexpr int kGuideBits = 12;              // guide table: 2^12 buckets of m
constexpr int kGuide = 1 << kGuideBits;
constexpr int kFineBits = 13;               // the warp-form sampler's finer guide: 2^13 buckets
constexpr int kFine = 1 << kFineBits;
// A guide word holds the bucket's smallest answer index (low 31 bits) and, in
// bit 31, whether the bucket holds more than one answer (a search is needed).
constexpr uint32_t kGuideMulti = 0x80000000u, kGuideIndex = 0x7fffffffu;
// Increment table of the warp-form sampler: 2^8 buckets of a draw's high
// word.  A bucket whose draws all take one of the first four values holds
// 1 << (8 b) (b = value - xmin), an increment of a lane's four 7-bit counter
// fields; any other bucket holds kIncOther.  Stored with 32 copies of every
// entry (bucket j, lane l at j * 32 + l) so that a warp's lookups never
// share a shared-memory bank.
constexpr int kIncBits = 8;
constexpr int kIncBuckets = 1 << kIncBits;
constexpr uint32_t kIncOther = 0x80000000u;
constexpr int kHMax = 1024;                 // dense histogram bins per warp
// Warp-form replicates with at most this many spills are finished by one lane
// (the record's spill slot always holds at least min(n, kLaneSpills)).
#ifndef PL_LANE_SPILLS
#define PL_LANE_SPILLS 20
#endif
constexpr int kLaneSpills = PL_LANE_SPILLS;
constexpr uint32_t kLaneBinsLong = 256, kLaneBinsShort = 128;
constexpr int64_t kLaneLongMinReps = 32768;  // cells with at least this many replicates take the long lanes
// Warp-form cells whose dense histogram has at most this many bins (small n)
// are drawn by the lane-form sampler, one thread per replicate.
#ifndef PL_LANE_SAMPLE_BINS
#define PL_LANE_SAMPLE_BINS 64
#endif
constexpr uint32_t kLaneSampleBins = PL_LANE_SAMPLE_BINS;
// ... and at most this many values per replicate (a light-tailed cell of more
// values may have kLaneSampleBins bins too; it stays in the warp form).
#ifndef PL_LANE_SAMPLE_NMAX
#define PL_LANE_SAMPLE_NMAX 100
#endif
constexpr int64_t kLaneSampleNMax = PL_LANE_SAMPLE_NMAX;
// Expected values per replicate beyond the dense bins that a warp-form cell's
// shortened histogram may leave to the spills.
#ifndef PL_LIGHT_SPILLS
#define PL_LIGHT_SPILLS 14.0
#endif
constexpr double kLightSpills = PL_LIGHT_SPILLS;
constexpr int kHWide = 8192;                // dense histogram bins per block (block form)
#ifndef PL_FIN_WARPS
#define PL_FIN_WARPS 8
#endif
constexpr int kWarps = PL_FIN_WARPS;        // finisher warps per block
constexpr int kSortSmem = kHMax / 2;        // replicates with more spills count as large sorts
constexpr int kLnTable = 16384;             // ln(xmin + i) tables, i < kLnTable
constexpr int kNewtonCap = 200;             // Newton iteration cap

// Device status word bits (latched; read by pl_sync).
constexpr uint32_t kErrTimeout = 1u;        // a bounded mbarrier wait ran out
constexpr uint32_t kErrData = 2u;           // a data value below xmin
constexpr uint32_t kErrArena = 4u;          // a replicate's spills exceeded every buffer

struct Counters {
  unsigned long long newton_capped;
  unsigned long long tail_draws;
  unsigned long long global_sorts;
  unsigned long long fit_fallbacks;          // replicates fitted by the full Newton iteration
  unsigned long long resampled;              // replicates whose spill slot overflowed
  unsigned int status;
  unsigned int work_next;                   // persistent-kernel work counter
  unsigned long long wait_limit;            // test hook: the first staging wait runs out after this many cycles
#ifdef PL_PHASE_TIMING
  unsigned long long phase_cycles[8];       // diagnostic build only
#endif
};

// One distinct (alpha, xmin): its inverse-CDF thresholds and log tables.
struct Law {
  double alpha;
  double Z;               // zeta(alpha, xmin)
  uint64_t xmin;
  uint32_t L2;            // table length (>= kL1, multiple of kL1)
  uint32_t pad;
  float tail_c;           // (alpha - 1) Z 2^-32, binary32: continuous tail approximation
  float tail_e;           // -1 / (alpha - 1)
  float xmin_f;           // xmin + 1/2, binary32
  uint64_t *T;            // T[i] = floor(Q(xmin+i) 2^53) + 1, Q(k) = P(X > k)
  uint32_t *guide;        // guide[j] = min{i : T[i] <= (j+1) 2^(53-g)} (or L2) | kGuideMulti flag
  uint32_t *inc;          // increment table (kIncBuckets x 32 copies)
  uint32_t *fine;         // guide of kFine buckets (same form as guide)
  double *lnT;            // ln(xmin + i), i < kLnTable
  float *lnT_hi;          // float split of lnT: hi + lo
  float *lnT_lo;
};

struct Cell {
  double alpha;           // exponent of the simulated law
  uint64_t xmin;
  int64_t n;
  int64_t R;
  uint32_t cell_id;
  uint32_t law;           // index into the law array
  uint32_t H;             // dense histogram bins in use (<= kHMax)
  uint32_t purpose;
  int64_t out_off;        // offset of replicate 0 in the per-replicate outputs
  uint32_t fit;           // index into the fit-table array (one per xmin)
  uint32_t scap;          // spill slot capacity of a replicate record
  uint32_t wide;          // block form: 32-bit dense counts, H = kHWide
  uint32_t inline_bins;   // draw loop: bin single-valued draws beyond the first four values at once (heavy tails)
  uint32_t lane_bins;     // finisher: warp-form replicates with a largest bin below this (and at most
                          // kLaneSpills spills) are finished by one lane each
  uint32_t lane_sample;   // drawn by the lane-form sampler (warp form, H <= kLaneSampleBins)
};

// A block-sized batch of replicates of one cell, with the offsets of its
// replicate records (dense counts, spill values, meta) in the record buffers.
constexpr int kItemReps = 256;
static_assert(kItemReps <= 32 * kWarps, "a finisher warp takes at most 32 replicates of an item (a lane each)");
struct WorkItem {
  uint32_t cell;
  uint32_t r0;            // first replicate
  uint32_t nrep;          // replicates in this item (<= kItemReps)
  uint32_t pad;
  uint64_t dense_off;     // uint16 index of replicate r0's dense counts
  uint64_t spill_off;     // uint64 index of replicate r0's spill values
  uint64_t meta_off;      // index of replicate r0's (tmax, spill count)
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// The same generator with the ten round keys precomputed: rk[2r], rk[2r+1]
// = key + r * (0x9E3779B9, 0xBB67AE85).  The 32x32 -> 64-bit products are
// taken whole (high and low halves from one multiply).
struct RoundKeys {
  uint32_t k[20];
};

__host__ __device__ inline RoundKeys round_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk.k[2 * r] = k0;
    rk.k[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return rk;
}

__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const RoundKeys &rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one 32x32->64 multiply per product, its halves unpacked in place
    uint32_t h0, l0, h1, l1;
    asm("{\n\t.reg .b64 t;\n\tmul.wide.u32 t, %2, 0xD2511F53;\n\tmov.b64 {%0, %1}, t;\n\t}"
        : "=r"(l0), "=r"(h0)
        : "r"(c.x));
    asm("{\n\t.reg .b64 t;\n\tmul.wide.u32 t, %2, 0xCD9E8D57;\n\tmov.b64 {%0, %1}, t;\n\t}"
        : "=r"(l1), "=r"(h1)
        : "r"(c.z));
    c = make_uint4(h1 ^ c.y ^ rk.k[2 * r], l1, h0 ^ c.w ^ rk.k[2 * r + 1], l0);
  }
  return c;
}

// Draw i of the stream (rep, cell, purpose): its high word h is word i mod 4
// of the Philox block with counter (floor(i/4), rep, cell, purpose), its low
// word l the same word of the block with counter (floor(i/4), rep, cell,
// purpose | kLowStream); m = h 2^21 + floor(l / 2^11) + 1 in [1, 2^53].  Every
// m of the interval [h 2^21 + 1, (h + 1) 2^21] has the same answer unless a
// threshold lies inside it (at most one draw in 2^32 per threshold), so the
// samplers take the low word only then, or for a draw beyond the table, whose
// tail inversion needs m itself.
constexpr uint32_t kLowStream = 0x80000000u;

__device__ __forceinline__ uint32_t quad_word(const uint4 &w, uint32_t j) {
  return j == 0 ? w.x : (j == 1 ? w.y : (j == 2 ? w.z : w.w));
}

__device__ __forceinline__ uint64_t draw_m(uint32_t h, uint32_t l) {
  return (((uint64_t)h << 21) | (l >> 11)) + 1ull;
}

// m of draw i from its high word h (one Philox block of the low stream).  A
// call, not inlined: the samplers take it rarely, and inlined its rounds
// would claim registers in their draw loops.
static __device__ __noinline__ uint64_t draw_m_full(uint32_t h, uint64_t i, uint32_t rep, uint32_t cell,
                                                    uint32_t purpose, uint32_t key_lo, uint32_t key_hi) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)(i >> 2), rep, cell, purpose | kLowStream),
                                make_uint2(key_lo, key_hi));
  return draw_m(h, quad_word(w, (uint32_t)i & 3u));
}

// Smallest and largest m a high word allows.
__device__ __forceinline__ uint64_t m_first(uint32_t h) { return ((uint64_t)h << 21) + 1ull; }
__device__ __forceinline__ uint64_t m_last(uint32_t h) { return ((uint64_t)h + 1ull) << 21; }

// ---------------------------------------------------------------------------
// Euler-Maclaurin for the Hurwitz zeta (DLMF 2.10.1, 25.11):
//   zeta(s,a) = sum_{k<M} (a+k)^-s + N^(1-s)/(s-1) + N^-s/2
//             + sum_{j=1..8} B_2j/(2j)! s(s+1)..(s+2j-2) N^(-s-2j+1),  N = a+M,
// with M chosen so that N >= 10 + 1.5 s; the first omitted term is then
// below 2^-56 of the integral term for every s > 1.
__device__ __forceinline__ double bern_coef(int j) {
  // B_2j / (2j)!, j = 1..8
  switch (j) {
    case 1: return 1.0 / 12.0;
    case 2: return -1.0 / 720.0;
    case 3: return 1.0 / 30240.0;
    case 4: return -1.0 / 1209600.0;
    case 5: return 1.0 / 47900160.0;
    case 6: return -691.0 / 1307674368000.0;
    case 7: return 1.0 / 74724249600.0;
    default: return -3617.0 / 10670622842880000.0;
  }
}

__device__ __forceinline__ int em_shift(double s, double a) {
  const double nmin = 10.0 + 1.5 * s;
  return a < nmin ? (int)ceil(nmin - a) : 0;
}

// The Euler-Maclaurin part beyond the direct terms, from N on:
//   N^(1-s)/(s-1) + N^-s/2 + sum_{j=1..8} B_2j/(2j)! s(s+1)..(s+2j-2) N^(-s-2j+1)
// and its first/second s-derivatives into z[0..ND].
template <int ND, bool PRECISE>
__device__ __forceinline__ void hurwitz_em_tail(double s, double N, double *z) {
  const double L = log(N);
  const double Ns = PRECISE ? pow(N, -s) : exp(-s * L);
  const double u = 1.0 / (s - 1.0);
  const double N1s = N * Ns;
  double z0 = N1s * u + 0.5 * Ns;
  double z1 = -N1s * (L * u + u * u) - 0.5 * L * Ns;
  double z2 = N1s * (L * L * u + 2.0 * L * u * u + 2.0 * u * u * u) + 0.5 * L * L * Ns;
  const double inv_n2 = 1.0 / (N * N);
  double w = Ns / N;                           // N^(-s-1)
  double P = s, dP = 1.0, d2P = 0.0;           // s(s+1)..(s+2j-2) and derivatives
#pragma unroll
  for (int j = 1; j <= 8; ++j) {
    const double c = bern_coef(j) * w;
    z0 += c * P;
    if (ND >= 1) z1 += c * (dP - L * P);
    if (ND >= 2) z2 += c * (d2P - 2.0 * L * dP + L * L * P);
#pragma unroll
    for (int f = 2 * j - 1; f <= 2 * j; ++f) {
      const double g = s + (double)f;
      if (ND >= 2) d2P = d2P * g + 2.0 * dP;
      if (ND >= 1) dP = dP * g + P;
      P *= g;
    }
    w *= inv_n2;
  }
  z[0] = z0;
  if (ND >= 1) z[1] = z1;
  if (ND >= 2) z[2] = z2;
}

// zeta(s, a) and, for ND >= 1/2, its first/second s-derivatives into z[0..ND].
// PRECISE evaluates powers with pow(); otherwise with exp(-s ln x), the log
// taken from lnx_table when x - a0 < table_len (table of ln(a0 + i)).
template <int ND, bool PRECISE>
__device__ __forceinline__ void hurwitz_em(double s, double a, double *z,
                                           const double *lnx_table = nullptr,
                                           double a0 = 0.0, int table_len = 0) {
  double z0 = 0.0, z1 = 0.0, z2 = 0.0;
  const int M = em_shift(s, a);
  for (int k = 0; k < M; ++k) {
    const double x = a + (double)k;
    double lx, t;
    if (PRECISE) {
      lx = log(x);
      t = pow(x, -s);
    } else {
      const int idx = (int)(x - a0);
      lx = (lnx_table && idx >= 0 && idx < table_len) ? lnx_table[idx] : log(x);
      t = exp(-s * lx);
    }
    z0 += t;
    if (ND >= 1) z1 -= lx * t;
    if (ND >= 2) z2 += lx * lx * t;
  }
  double t[3];
  hurwitz_em_tail<ND, PRECISE>(s, a + (double)M, t);
  z[0] = z0 + t[0];
  if (ND >= 1) z[1] = z1 + t[1];
  if (ND >= 2) z[2] = z2 + t[2];
}

__device__ __forceinline__ double hurwitz_precise(double s, double a) {
  double z;
  hurwitz_em<0, true>(s, a, &z);
  return z;
}

// zeta(s, a) for large a (a >= 10 + 1.5 s and a >= 1024): Euler-Maclaurin with
// no direct terms and 4 Bernoulli terms, written around the integral term:
//   a^(1-s)/(s-1) [1 + (s-1)/(2a) + sum_j B2j/(2j)! s(s+1)..(s+2j-2)(s-1) a^-2j];
// the first omitted term is below 1e-16 relative for s <= 64.
__device__ __forceinline__ double hurwitz_large_a(double s, double a) {
  const double ia2 = 1.0 / (a * a);
  const double sm1 = s - 1.0;
  double P = s, w = ia2, br = 1.0 + 0.5 * sm1 / a;
#pragma unroll
  for (int j = 1; j <= 4; ++j) {
    br += bern_coef(j) * P * sm1 * w;
    P *= (s + (double)(2 * j - 1)) * (s + (double)(2 * j));
    w *= ia2;
  }
  return pow(a, -sm1) / sm1 * br;
}

// Survival of the law at k: Q(k) = zeta(alpha, k+1) / Z, argument formed as
// (double)k + 1 (rounded for k > 2^53).
__device__ __forceinline__ double survival(double alpha, double Z, uint64_t k) {
  const double a = (double)k + 1.0;
  if (a >= 1024.0 && a >= 10.0 + 1.5 * alpha) return hurwitz_large_a(alpha, a) / Z;
  return hurwitz_precise(alpha, a) / Z;
}


// ---------------------------------------------------------------------------
// Single-evaluation form used by the Newton polish: 12 Bernoulli terms and
// N = max(a, ceil(7 + 0.75 s)) (warp-uniform, passed in), which keeps the first
// omitted term below 2^-56 of the tail for every s > 1.  For a = 1 and
// N <= 16 the direct terms k^-s are formed from exp(-s ln p) at the primes
// p = 2, 3, 5, 7, 11, 13 and products for the composites.
static __constant__ double c_bern12[12] = {
    1.0 / 12.0, -1.0 / 720.0, 1.0 / 30240.0, -1.0 / 1209600.0, 1.0 / 47900160.0,
    -691.0 / 1307674368000.0, 1.0 / 74724249600.0, -3617.0 / 10670622842880000.0,
    8.586062056277845e-15, -2.174868698558062e-16, 5.5090028283602295e-18,
    -1.3954464685812522e-19};
static __constant__ double c_ln_small[17] = {
    0.0,
    0.0,
    0.6931471805599453,
    1.0986122886681098,
    1.3862943611198906,
    1.6094379124341003,
    1.791759469228055,
    1.9459101490553132,
    2.0794415416798357,
    2.1972245773362196,
    2.302585092994046,
    2.3978952727983707,
    2.4849066497880004,
    2.5649493574615367,
    2.6390573296152584,
    2.70805020110221,
    2.772588722239781};

__device__ __forceinline__ int polish_shift_n(double s, uint64_t a) {
  const int n = (int)ceil(7.0 + 0.75 * s);
  return (uint64_t)n > a ? n : (int)a;
}

__device__ __forceinline__ void polish_direct_term(double t, double lk, double &z0, double &z1,
                                                   double &z2) {
  z0 += t;
  z1 -= lk * t;
  z2 += lk * lk * t;
}

// zeta(s, a), zeta', zeta'' with the shift Nw >= polish_shift_n(s, a).
__device__ __forceinline__ void hurwitz_polish(double s, uint64_t a, int Nw, const double *lnT,
                                               double *z) {
  double z0 = 0.0, z1 = 0.0, z2 = 0.0;
  if (a == 1 && Nw <= 16) {
    const double t2 = exp(-s * c_ln_small[2]);
    const double t3 = exp(-s * c_ln_small[3]);
    const double t5 = exp(-s * c_ln_small[5]);
    const double t7 = exp(-s * c_ln_small[7]);
    z0 = 1.0;  // k = 1
    polish_direct_term(t2, c_ln_small[2], z0, z1, z2);
    if (Nw > 3) polish_direct_term(t3, c_ln_small[3], z0, z1, z2);
    if (Nw > 4) polish_direct_term(t2 * t2, c_ln_small[4], z0, z1, z2);
    if (Nw > 5) polish_direct_term(t5, c_ln_small[5], z0, z1, z2);
    if (Nw > 6) polish_direct_term(t2 * t3, c_ln_small[6], z0, z1, z2);
    if (Nw > 7) polish_direct_term(t7, c_ln_small[7], z0, z1, z2);
    if (Nw > 8) polish_direct_term(t2 * t2 * t2, c_ln_small[8], z0, z1, z2);
    if (Nw > 9) polish_direct_term(t3 * t3, c_ln_small[9], z0, z1, z2);
    if (Nw > 10) polish_direct_term(t2 * t5, c_ln_small[10], z0, z1, z2);
    if (Nw > 11) polish_direct_term(exp(-s * c_ln_small[11]), c_ln_small[11], z0, z1, z2);
    if (Nw > 12) polish_direct_term(t2 * t2 * t3, c_ln_small[12], z0, z1, z2);
    if (Nw > 13) polish_direct_term(exp(-s * c_ln_small[13]), c_ln_small[13], z0, z1, z2);
    if (Nw > 14) polish_direct_term(t2 * t7, c_ln_small[14], z0, z1, z2);
    if (Nw > 15) polish_direct_term(t3 * t5, c_ln_small[15], z0, z1, z2);
  } else {
    for (uint64_t k = a; k < (uint64_t)Nw; ++k) {
      const double lk = lnT[k - a];
      polish_direct_term(exp(-s * lk), lk, z0, z1, z2);
    }
  }
  const double N = (double)Nw;
  const uint64_t ni = (uint64_t)Nw - a;
  const double L = (a == 1 && Nw <= 16) ? c_ln_small[Nw] : lnT[ni];
  const double Ns = exp(-s * L);
  const double u = 1.0 / (s - 1.0);
  const double N1s = N * Ns;
  z0 += N1s * u + 0.5 * Ns;
  z1 += -N1s * (L * u + u * u) - 0.5 * L * Ns;
  z2 += N1s * (L * L * u + 2.0 * L * u * u + 2.0 * u * u * u) + 0.5 * L * L * Ns;
  const double inv_n2 = 1.0 / (N * N);
  double w = Ns / N;
  double P = s, dP = 1.0, d2P = 0.0;
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    const double c = c_bern12[j] * w;
    z0 += c * P;
    z1 += c * (dP - L * P);
    z2 += c * (d2P - 2.0 * L * dP + L * L * P);
#pragma unroll
    for (int f = 2 * j + 1; f <= 2 * j + 2; ++f) {
      const double g = s + (double)f;
      d2P = d2P * g + 2.0 * dP;
      dP = dP * g + P;
      P *= g;
    }
    w *= inv_n2;
  }
  z[0] = z0;
  z[1] = z1;
  z[2] = z2;
}

// Inverse of the MLE equation per lower end xmin, for the Newton start.
// Nodes at a uniform grid of t = ln(alpha - 1) (alpha from 60 down to
// 1.003), ordered by increasing u = ln(h), h = E[ln(X / xmin)] =
// -zeta'/zeta - ln xmin; each node holds (u, alpha, d alpha/du = -h/Var(ln X),
// 1/(u_next - u)) from one Euler-Maclaurin evaluation.  A guide table over a
// uniform u grid points to the node at or below each bin start.  Lookup:
// guide, a short forward scan, cubic Hermite interpolation in u.
// Node of the inverse of the MLE equation, at u = ln(mean ln x - ln xmin):
// alpha(u), its slope, ln zeta(alpha, xmin) and its slope in u.
struct FitNode {
  double u, alpha, dadu, inv_du, lnZ, dlnZdu;
};
// Below this exponent the fit table's interpolation is accurate to ~1e-11
// (alpha and zeta) for every xmin; the binary32 form takes it as the fit.
constexpr double kFitTableOnlyMax = 16.0;
struct FitTable {
  uint64_t xmin;
  int nodes;
  int guides;
  double ug0, inv_dug;     // guide grid: bin b starts at ug0 + b / inv_dug
  FitNode *node;
  int *guide;
  const double *lnx;       // ln(xmin + i), i < kLnTable: read while the table is built
};
constexpr int kFitNodes = 4096;
constexpr int kFitGuides = 4096;
constexpr double kFitAlphaHi = 60.0, kFitAlphaLo = 1.003;

// ---------------------------------------------------------------------------
// Inverse CDF.  X = min(2^62, min{k >= xmin : Q(k) < v}), v = m 2^-53.
// Table region: T[i] <= m  <=>  Q(xmin+i) < v (T[i] = floor(Q 2^53) + 1 and
// Q 2^53 is exact), so the search is on 64-bit integers only.  The guide
// bucket j = (m-1) >> (53-g) bounds the answer to [guide[j], guide[j-1]].

// Beyond the table: FP64 evaluation of Q, started from the continuous
// approximation zeta(s, k+1) ~ (k + 1/2)^(1-s) / (s-1), which is within one of
// the answer beyond a few dozen; the guess is confirmed with
// Q(k) < v <= Q(k-1) = Q(k) + k^-s / Z.  Otherwise exponential search and
// bisection (every loop bounded).
static __device__ __noinline__ uint64_t tail_invert(double alpha, double Z, uint64_t kstart,
                                             uint64_t m) {
  const double v = (double)m * 0x1p-53;
  const double s = alpha;
  double g = pow((s - 1.0) * Z * v, -1.0 / (s - 1.0)) - 0.5;
  uint64_t k;
  if (!(g < (double)kXCap)) k = kXCap;
  else if (g <= (double)kstart) k = kstart;
  else k = (uint64_t)ceil(g);
  if (k > kstart && k < kXCap) {
    const double qk = survival(s, Z, k);
    if (qk < v && qk + pow((double)k, -s) / Z >= v) return k;
  }
  uint64_t lo, hi;
  if (survival(s, Z, k) < v) {
    hi = k;
    uint64_t d = 1;
    for (int it = 0; it < 64; ++it) {
      if (hi == kstart) break;
      const uint64_t c = (hi - kstart > d) ? hi - d : kstart;
      if (survival(s, Z, c) < v) {
        hi = c;
        d <<= 1;
      } else {
        lo = c + 1;
        goto bisect;
      }
    }
    return hi;  // hi == kstart (or the loop bound; unreachable for hi < 2^63)
  } else {
    if (k >= kXCap) return kXCap;
    lo = k + 1;
    uint64_t d = 1;
    for (int it = 0; it < 64; ++it) {
      const uint64_t c = (kXCap - lo > d) ? lo + d - 1 : kXCap;
      if (survival(s, Z, c) < v) {
        hi = c;
        goto bisect;
      }
      if (c == kXCap) return kXCap;
      lo = c + 1;
      d <<= 1;
    }
    return kXCap;
  }
bisect:
  for (int it = 0; it < 70 && lo < hi; ++it) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (survival(s, Z, mid) < v) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Table search: sT / sG are the shared-memory copies of T[0..kL1) and guide.
// Returns xmin + i, or kTailTag | m when the answer lies beyond the table (the
// caller resolves those with tail_invert).  A wide guide bucket (heavy tail)
// is first narrowed around the continuous-approximation guess
// k + 1/2 ~ ((alpha - 1) Z v)^(-1/(alpha-1)) in binary32, then by galloping;
// the final answer always comes from exact integer comparisons with T.
constexpr uint64_t kTailTag = 1ull << 63;

__device__ __forceinline__ uint64_t table_at(const uint64_t *sT, const uint64_t *gT, uint32_t i) {
  return i < (uint32_t)kL1 ? sT[i] : __ldg(gT + i);
}

// Index form: returns i = X - xmin for answers inside the table, L2 beyond it.
// GB: the guide's bucket bits (2^GB buckets of m).
template <int GB = kGuideBits>
__device__ __forceinline__ uint32_t lookup_index(const uint64_t *sT, const uint32_t *sG,
                                                 const uint64_t *gT, uint32_t L2, float xmin_f,
                                                 float tail_c, float tail_e, uint64_t m) {
  const uint32_t j = (uint32_t)((m - 1ull) >> (53 - GB));
  uint32_t lo = sG[j] & kGuideIndex;
  uint32_t hi = j ? sG[j - 1] & kGuideIndex : L2;
  if (hi - lo > 8) {
    // v 2^32 from the top 32 of the 53 bits of m (tail_c carries the 2^-32)
    const float v32 = (float)(uint32_t)(m >> 21);
    const float kf = exp2f(tail_e * __log2f(tail_c * v32)) - xmin_f;
    uint32_t g = lo;
    if (kf >= (float)hi) g = hi - 1;
    else if (kf > (float)lo) g = (uint32_t)kf;
    if (table_at(sT, gT, g) <= m) {  // answer in [lo, g]: gallop down
      hi = g;
      for (uint32_t d = 1; d < 64u && hi > lo; d <<= 1) {
        const uint32_t c = hi - lo > d ? hi - d : lo;
        if (table_at(sT, gT, c) <= m) hi = c;
        else {
          lo = c + 1;
          break;
        }
      }
    } else {  // answer in [g + 1, hi]: gallop up
      lo = g + 1;
      for (uint32_t d = 1; d < 64u && lo < hi; d <<= 1) {
        const uint32_t c = hi - lo > d ? lo + d - 1 : hi - 1;
        if (table_at(sT, gT, c) <= m) {
          hi = c;
          break;
        }
        lo = c + 1;
      }
    }
  }
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (table_at(sT, gT, mid) <= m) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Index of a draw known by its high word h: the answer at m_first(h); the
// low word (m_full(), which returns m) is drawn only when the answer at
// m_last(h) may be smaller (T[i - 1] <= m_last) or the answer lies beyond the
// table, and then *m receives m.  The answer is nonincreasing in m, so the
// first case is exact.
template <class MFull>
__device__ __forceinline__ uint32_t lookup_index_hi(const uint64_t *sT, const uint32_t *sG, const uint64_t *gT,
                                                    uint32_t L2, float xmin_f, float tail_c, float tail_e,
                                                    uint32_t h, MFull m_full, uint64_t *m) {
  const uint32_t i0 = lookup_index(sT, sG, gT, L2, xmin_f, tail_c, tail_e, m_first(h));
  if (i0 < L2 && (i0 == 0 || table_at(sT, gT, i0 - 1) > m_last(h))) return i0;
  *m = m_full();
  return lookup_index(sT, sG, gT, L2, xmin_f, tail_c, tail_e, *m);
}

// Value of a draw that a sampler left tagged (kTailTag | m): the exact table
// search in global memory when the answer lies inside the table, else the
// binary64 inversion beyond it.
__device__ __forceinline__ uint64_t resolve_tagged(const Law &law, uint64_t m, bool *beyond) {
  const uint32_t i = lookup_index(law.T, law.guide, law.T, law.L2, law.xmin_f, law.tail_c, law.tail_e, m);
  *beyond = i >= law.L2;
  return i < law.L2 ? law.xmin + i : tail_invert(law.alpha, law.Z, law.xmin + law.L2, m);
}

__device__ __forceinline__ uint64_t lookup_fast(const uint64_t *sT, const uint32_t *sG,
                                                const uint64_t *gT, uint32_t L2, uint64_t xmin,
                                                float xmin_f, float tail_c, float tail_e, uint64_t m) {
  const uint32_t i = lookup_index(sT, sG, gT, L2, xmin_f, tail_c, tail_e, m);
  return i < L2 ? xmin + i : (kTailTag | m);
}

__device__ __forceinline__ uint64_t lookup(const uint64_t *sT, const uint32_t *sG,
                                           const uint64_t *gT, uint32_t L2, uint64_t xmin,
                                           double alpha, double Z, float xmin_f, float tail_c,
                                           float tail_e, uint64_t m, unsigned long long *tail_counter) {
  const uint64_t x = lookup_fast(sT, sG, gT, L2, xmin, xmin_f, tail_c, tail_e, m);
  if (!(x & kTailTag)) return x;
  atomicAdd(tail_counter, 1ull);
  return tail_invert(alpha, Z, xmin + L2, m);
}

// ---------------------------------------------------------------------------
// Warp helpers.
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}
__device__ __forceinline__ float warp_maxf(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}
__device__ __forceinline__ int64_t warp_sum_i64(int64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ int64_t warp_max_i64(int64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t y = __shfl_xor_sync(0xffffffffu, x, o);
    x = x > y ? x : y;
  }
  return x;
}
// inclusive scans
__device__ __forceinline__ double warp_scan(double x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}
__device__ __forceinline__ int64_t warp_scan_i64(int64_t x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Error-free sum of two floats (Knuth TwoSum): s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) float pairs: compensated addition.
__device__ __forceinline__ void ff_add(float &hi, float &lo, float bh, float bl) {
  float s, e;
  two_sum(hi, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(lo, bl));
  hi = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s));
}
// inclusive compensated scan of (hi, lo) pairs
__device__ __forceinline__ void warp_scan_ff(float &hi, float &lo, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float yh = __shfl_up_sync(0xffffffffu, hi, o);
    const float yl = __shfl_up_sync(0xffffffffu, lo, o);
    if (lane >= o) ff_add(hi, lo, yh, yl);
  }
}
__device__ __forceinline__ void warp_sum_ff(float &hi, float &lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float yh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float yl = __shfl_xor_sync(0xffffffffu, lo, o);
    ff_add(hi, lo, yh, yl);
  }
}

// ---------------------------------------------------------------------------
// Bounded mbarrier wait: gives up after ~2^31 clock cycles (about a second)
// and reports false.
// Waits give up after kWaitCycles SM cycles (about a second at 2 GHz).
constexpr long long kWaitCycles = 1ll << 31;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity, long long limit = kWaitCycles) {
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(mbar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(mbar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(mbar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared (TMA engine, no tensor map), completion
// signalled on mbar.  dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *mbar) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(mbar);
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
      "l"(src), "r"(bytes), "r"(b)
      : "memory");
}

}  // namespace pl
