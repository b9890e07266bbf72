// pl_truncated.cuh -- the truncated law on 1..K (Section 1's second version
// of the power law, Tables 2-6): p(k) = k^-gamma / zeta_K(gamma),
// zeta_K(gamma) = sum_{k=1}^{K} k^-gamma, any gamma > 0.
//
// Device structures and launch wrappers (host side).  The same method as for
// the untruncated law: inverse-CDF draws from integer thresholds, the MLE of
// Eq. 2 with the finite scaling factor (its root searched on the whole real
// line, bounded to [-64, 64]) and D of Eq. 3 over the support.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pl_device.cuh"

namespace pl {

constexpr uint32_t kTzKMax = 1024;          // largest support
constexpr int64_t kTzNMax = 65535;          // largest sample (16-bit histogram counts)
constexpr int kTzGuideBits = 11;            // guide: 2^11 buckets of m
constexpr int kTzGuide = 1 << kTzGuideBits;
#ifndef PL_TZ_WARPS
#define PL_TZ_WARPS 8
#endif
#ifndef PL_TZ_MIN_BLOCKS
#define PL_TZ_MIN_BLOCKS 4
#endif
constexpr int kTzWarps = PL_TZ_WARPS;       // warps per block of the replicate kernel
// Fit nodes: gamma_j = -64 + j / 32, j = 0..4096.  Around each node the
// scaling factor is a polynomial in delta = gamma - gamma_j:
//   zeta_K(gamma_j + delta) = a_0 sum_r b_r delta^r,
//   a_r = sum_k (-ln k)^r k^-gamma_j / r!,  b_r = a_r / a_0 (b_0 = 1),
// exact as a series; kTzTerms terms leave a relative error below
// (ln(1024) / 32)^14 / 14! < 1e-20 for delta in [0, 1/32], and below
// 3e-17 in the second derivative.  The normalised polynomial stays in
// [K^(-1/32), 1] on the interval, whatever the scale of a_0.
constexpr int kTzNodeInv = 32;              // nodes per unit of gamma
constexpr double kTzGammaLo = -64.0, kTzGammaHi = 64.0;
constexpr int kTzNodes = 128 * kTzNodeInv + 1;
constexpr int kTzTerms = 14;
// Node record (doubles): a_0, b_1..b_13, then E_j (mean of ln X at gamma_j),
// V_j (its variance), 1 / (E_j - E_{j+1}), (E_j - E_{j+1}) / V_j,
// (E_j - E_{j+1}) / V_{j+1} (the Hermite start on [gamma_j, gamma_{j+1}]),
// 1 / a_0.
constexpr int kTzNodeStride = 20;
constexpr int kTzE = 14, kTzV = 15, kTzInvDE = 16, kTzS0 = 17, kTzS1 = 18, kTzInvA0 = 19;
constexpr int kTzNewtonCap = 64;

// One distinct (gamma, K): thresholds T[k] = floor(Q(k) 2^53) + 1 for
// k = 0..K, Q(k) = P(X > k) (T[0] = 2^53 + 1, T[K] = 1), and the guide
// guide[j] = min{k : T[k] <= (j + 1) 2^42}.
struct TzLaw {
  double gamma;
  uint32_t K;
  uint32_t table;          // index of the table of this K
  uint64_t *T;             // K + 1 entries
  uint16_t *guide;         // kTzGuide entries
};

// One distinct K: logarithms and the fit nodes.
struct TzTable {
  uint32_t K;
  uint32_t pad;
  double lnK;
  double *lnk;             // ln k at index k (k = 1..K; index 0 unused)
  float *lnk_hi, *lnk_lo;  // float split of ln k
  float *lnq_hi, *lnq_lo;  // float split of ln(k / K) (<= 0)
  double *node;            // kTzNodes records of kTzNodeStride doubles
  double *E;               // E_j = E[ln X] at gamma_j (decreasing in j)
};

struct TzCell {
  double gamma;
  int64_t n;
  int64_t R;
  int64_t out_off;         // offset of replicate 0 in the per-replicate outputs
  uint32_t cell_id;
  uint32_t law;
  uint32_t purpose;
  uint32_t pad;
};

struct TzItem {
  uint32_t cell;
  uint32_t r0;
  uint32_t nrep;
  uint32_t pad;
};

cudaError_t launch_tz_setup(TzLaw *laws, int nlaws, TzTable *tables, int ntables, cudaStream_t st);

cudaError_t launch_tz_sample(const TzLaw *law, uint64_t seed, uint32_t cell_id, uint32_t purpose,
                             uint32_t rep0, int64_t nrep, int64_t n, uint64_t *out, cudaStream_t st);

struct TzLaunch {
  const TzCell *cells;
  const TzLaw *laws;
  const TzTable *tables;
  const TzItem *items;
  uint32_t nitems;
  RoundKeys rk;
  void *D_out;             // double or float per precision
  double *A_out;           // may be null
  Counters *ctr;
};
cudaError_t launch_tz_replicates(const TzLaunch &a, bool f32, cudaStream_t st);

// Fit (or the given exponent) and D of one data set (values 1..K, int32):
// out = (gamma, D, zeta_K(gamma)); a value outside 1..K latches the data
// error and writes NaN.
cudaError_t launch_tz_dataset(const int32_t *x, int64_t n, const TzTable *tab, bool fit, double gamma, bool f32,
                              double *out, Counters *ctr, cudaStream_t st);

}  // namespace pl
