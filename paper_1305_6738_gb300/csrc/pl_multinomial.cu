// pl_multinomial.cu -- the multinomial histogram sampler (a large-n variant of
// the sampler; not in the paper): a replicate's histogram drawn bin by bin by
// conditional binomials, the few values of the tail one by one, written as a
// block-form replicate record that the finisher fits and tests as usual.
//
// Law: the inverse-CDF sampler's, through its integer thresholds T (with
// T[-1] = 2^53 + 1, P(X = xmin + i) = (T[i-1] - T[i]) 2^-53).  Bin i gets
// Bin(n_rem, p_i), p_i = (T[i-1] - T[i]) / (T[i-1] - 1), of the n_rem values
// not yet placed, for i = 0, 1, ... while i < kMnBins and n_rem p_i >= 1; each
// value left is drawn conditional on X >= xmin + i as the inverse CDF of m'
// uniform on [1, T[i-1] - 1] (the multiply-high of a 64-bit random word).
// Random words: draw index 0, 1, 2, ... of the replicate's stream in that
// order (u = m 2^-53 for a binomial, all 64 bits for a single value).
//
// One thread per replicate: the binomial chain is sequential, and its work
// (binary64) grows with the number of occupied bins, not with n.
#include <cmath>

#include "pl_multinomial.cuh"

namespace pl {
namespace {

constexpr int kMnBins = 2048;

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

// x ln(x/M) + M - x, by its series in v = (x - M)/(x + M) near x = M.
__device__ double mn_deviance(double x, double M) {
  if (fabs(x - M) < 0.1 * (x + M)) {
    const double v = (x - M) / (x + M), v2 = v * v;
    double s = (x - M) * v, e = 2.0 * x * v;
    for (int j = 1; j < 1000; ++j) {
      e *= v2;
      const double s1 = s + e / (double)(2 * j + 1);
      if (s1 == s) return s1;
      s = s1;
    }
    return s;
  }
  return x * log(x / M) + M - x;
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

// Bin(n, p) from one uniform u by inversion along a fixed order of the
// outcomes: 0, 1, 2, ... for a mean below 30, else from the mode outward,
// each step to the neighbour of larger probability (the upper on ties).
__device__ int64_t mn_binomial(int64_t n, double p, double q, double u) {
  if (n <= 0 || !(p > 0.0)) return 0;
  if (!(q > 0.0)) return n;
  const double r = p / q;
  if ((double)n * p < 30.0) {
    double f = mn_binom_pmf(0, n, p, q), c = f;
    int64_t k = 0;
    while (c < u && k < n) {
      f *= (double)(n - k) / (double)(k + 1) * r;
      ++k;
      c += f;
      if (f == 0.0 && (double)k > (double)n * p) break;
    }
    return k;
  }
  int64_t M = (int64_t)floor((double)(n + 1) * p);
  if (M > n) M = n;
  const double fM = mn_binom_pmf(M, n, p, q);
  double rest = u - fM;
  if (rest <= 0.0) return M;
  int64_t lo = M - 1, hi = M + 1, last = M;
  double flo = lo >= 0 ? fM * (double)M / ((double)(n - M + 1) * r) : 0.0;
  double fhi = hi <= n ? fM * (double)(n - M) / (double)(M + 1) * r : 0.0;
  while (flo > 0.0 || fhi > 0.0) {
    if (fhi >= flo) {
      rest -= fhi;
      last = hi;
      if (rest <= 0.0) return hi;
      fhi = hi < n ? fhi * (double)(n - hi) / (double)(hi + 1) * r : 0.0;
      ++hi;
    } else {
      rest -= flo;
      last = lo;
      if (rest <= 0.0) return lo;
      flo = lo > 0 ? flo * (double)lo / ((double)(n - lo + 1) * r) : 0.0;
      --lo;
    }
  }
  return last;
}

// The 64-bit random word i of a replicate's stream (two words of Philox block
// i/2), one block cached.
struct MnStream {
  uint32_t rep, cell, purpose;
  uint64_t blk;
  uint4 w;
  __device__ uint64_t word(uint64_t i, const RoundKeys &rk) {
    if ((i >> 1) != blk) {
      blk = i >> 1;
      w = philox4x32_10_rk(make_uint4((uint32_t)blk, rep, cell, purpose), rk);
    }
    return (i & 1) ? ((uint64_t)w.w << 32) | w.z : ((uint64_t)w.y << 32) | w.x;
  }
};

__global__ void __launch_bounds__(128) mn_sample_kernel(MnLaunch a) {
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t it = t / kWideReps, j = t % kWideReps;
  if (it >= a.nitems) return;
  const WorkItem wi = a.items[it];
  if (j >= wi.nrep) return;
  const Cell &cell = a.cells[wi.cell];
  const Law &law = a.laws[cell.law];
  const uint32_t H = cell.H, L2 = law.L2;
  const int64_t n = cell.n;
  uint32_t *dense = reinterpret_cast<uint32_t *>(a.rec.dense + wi.dense_off + j * 2 * (uint64_t)H);
  uint64_t *spill = a.rec.spill + wi.spill_off + j * (uint64_t)cell.scap;
  MnStream s{wi.r0 + (uint32_t)j, cell.cell_id, cell.purpose, ~0ull, make_uint4(0, 0, 0, 0)};
  // head: conditional binomials
  uint64_t Tprev = (1ull << 53) + 1, idx = 0;
  int64_t left = n, tmax = -1;
  uint32_t b = 0;
  for (; b < (uint32_t)kMnBins && left > 0; ++b) {
    const uint64_t Tb = law.T[b];
    const double p = (double)(Tprev - Tb) / (double)(Tprev - 1);
    const double q = (double)(Tb - 1) / (double)(Tprev - 1);
    if ((double)left * p < 1.0) break;
    const uint64_t m = (s.word(idx++, a.rk) >> 11) + 1;
    const int64_t c = mn_binomial(left, p, q, (double)m * 0x1p-53);
    dense[b] = (uint32_t)c;
    if (c) tmax = b;
    left -= c;
    Tprev = Tb;
  }
  // the values left, conditional on X >= xmin + b: first the largest
  // histogram index they reach (to clear the bins from b to it), then counted
  const uint64_t span = Tprev - 1;
  auto index_of = [&](uint64_t w) {
    const uint64_t mp = __umul64hi(w, span) + 1;
    return lookup_index(law.T, law.guide, law.T, L2, law.xmin_f, law.tail_c, law.tail_e, mp);
  };
  int64_t top = -1;
  for (int64_t k = 0; k < left; ++k) {
    const uint32_t i = index_of(s.word(idx + (uint64_t)k, a.rk));
    if (i < H && (int64_t)i > top) top = i;
  }
  for (int64_t i = b; i <= top; ++i) dense[i] = 0u;
  int64_t ns = 0;
  for (int64_t k = 0; k < left; ++k) {
    const uint64_t w = s.word(idx + (uint64_t)k, a.rk);
    const uint32_t i = index_of(w);
    if (i < H) {
      dense[i] += 1u;
      if ((int64_t)i > tmax) tmax = i;
    } else {
      const uint64_t v = i < L2 ? cell.xmin + i : tail_invert(cell.alpha, law.Z, cell.xmin + L2,
                                                              __umul64hi(w, span) + 1);
      if (ns < (int64_t)cell.scap) spill[ns] = v;
      ++ns;
    }
  }
  if (ns > (int64_t)cell.scap) atomicOr(&a.ctr->status, kErrArena);  // the finisher must not redraw
  a.rec.meta[wi.meta_off + j] = make_int2((int)tmax, (int)ns);
}

}  // namespace

cudaError_t launch_mn_sample(const MnLaunch &a, cudaStream_t st) {
  const uint64_t threads = (uint64_t)a.nitems * kWideReps;
  if (threads == 0) return cudaSuccess;
  mn_sample_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace pl
