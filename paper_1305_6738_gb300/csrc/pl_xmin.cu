// pl_xmin.cu -- the lower end x_min by KS minimisation (the procedure of
// Clauset, Shalizi & Newman that the paper's tables are used with, Section 3):
// for every candidate among the sample's distinct values, the MLE of Eq. 2 on
// the tail {x >= x_min} and D (Eq. 3) of the tail at its fit; the estimate is
// the candidate of smallest D.
//
// xmin_hist_kernel (many blocks): a histogram of the values up to kXHist, the
// larger ones collected; xmin_prep_kernel (one block): the sorted distinct
// values with their counts (the collected ones sorted in global memory), then
// suffix sums of the counts and of c ln v.
// xmin_cand_kernel (a warp per candidate): the fit on lane 0 (safeguarded
// Newton on the Euler-Maclaurin Hurwitz zeta), then D over the tail's distinct
// values v and v - 1 on all lanes.  xmin_pick_kernel: the smallest D.
#include <cmath>

#include "pl_xmin.cuh"

namespace pl {
namespace {

constexpr int kXHist = kXHistBins;  // values 1..kXHist counted in shared memory
constexpr int kXWarps = 8;     // candidates per block of xmin_cand_kernel

// Histogram of the sample over many blocks: values 1..kXHist counted in a
// shared histogram per block and added to the global one (ghist, zeroed
// before), larger values appended to spill (counter *nspill, zeroed before);
// a value below 1 latches the data error.
__global__ void __launch_bounds__(256) xmin_hist_kernel(const int32_t *x, int64_t n, uint32_t *ghist,
                                                        uint64_t *spill, unsigned long long *nspill,
                                                        Counters *ctr) {
  __shared__ uint32_t hist[kXHist];
  for (int i = threadIdx.x; i < kXHist; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = x[i];
    if (v < 1)
      bad = true;
    else if (v <= kXHist)
      atomicAdd(&hist[v - 1], 1u);
    else
      spill[atomicAdd(nspill, 1ull)] = (uint64_t)v;
  }
  if (bad) atomicOr(&ctr->status, kErrData);
  __syncthreads();
  for (int i = threadIdx.x; i < kXHist; i += blockDim.x)
    if (hist[i]) atomicAdd(&ghist[i], hist[i]);
}

// One block of 1024 threads, after xmin_hist_kernel.  Writes the distinct
// values (ascending) and counts, S[j] = tail count from j on (S[d] = 0),
// Lt[j] = sum_{i >= j} c_i ln v_i, and d.  spill: scratch of a power of two
// >= n uint64 (the larger values, sorted here).
__global__ void __launch_bounds__(1024) xmin_prep_kernel(const uint32_t *ghist, uint64_t *spill,
                                                         const unsigned long long *nspill, uint64_t *vals,
                                                         uint32_t *cnts, int64_t *S, double *Lt, int64_t *d_out,
                                                         const Counters *ctr) {
  __shared__ uint32_t hist[kXHist];
  __shared__ int64_t s_part[33];
  __shared__ double s_dpart[33];
  if (ctr->status & kErrData) {
    if (threadIdx.x == 0) *d_out = 0;
    return;
  }
  for (int i = threadIdx.x; i < kXHist; i += blockDim.x) hist[i] = ghist[i];
  __syncthreads();
  const int64_t s = (int64_t)*nspill;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // sort the spills (block bitonic in global memory, padded to a power of two)
  uint32_t Q = 1;
  while ((int64_t)Q < s) Q <<= 1;
  for (uint32_t i = (uint32_t)s + threadIdx.x; s > 0 && i < Q; i += blockDim.x) spill[i] = ~0ull;
  __syncthreads();
  if (s > 1) {
    for (uint32_t k = 2; k <= Q; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t i = threadIdx.x; i < Q; i += blockDim.x) {
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
  // dense part: thread t owns bins [8t, 8t + 8); compact the nonzero bins in order
  constexpr int kPer = kXHist / 1024;
  int mine = 0;
  for (int b = 0; b < kPer; ++b) mine += hist[threadIdx.x * kPer + b] != 0;
  int incl = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_part[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int64_t w = s_part[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_part[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const int64_t d1 = s_part[31];
  int64_t pos = (warp ? s_part[warp - 1] : 0) + incl - mine;
  for (int b = 0; b < kPer; ++b) {
    const int bin = threadIdx.x * kPer + b;
    if (hist[bin]) {
      vals[pos] = (uint64_t)bin + 1;
      cnts[pos] = hist[bin];
      ++pos;
    }
  }
  __syncthreads();
  // spill part: run-length encode the sorted spills after the dense values
  // (warp 0): run starts first (their index kept in cnts), then the counts
  __shared__ int64_t s_d;
  if (warp == 0) {
    int64_t base = d1;
    for (int64_t i0 = 0; i0 < s; i0 += 32) {
      const int64_t i = i0 + lane;
      const bool ok = i < s;
      const uint64_t v = ok ? spill[i] : 0;
      const bool start = ok && (i == 0 || spill[i - 1] != v);
      const unsigned sb = __ballot_sync(0xffffffffu, start);
      const int rank = __popc(sb & ((1u << lane) - 1u));
      if (start) {
        vals[base + rank] = v;
        cnts[base + rank] = (uint32_t)i;
      }
      base += __popc(sb);
    }
    __syncwarp();
    for (int64_t k0 = d1; k0 < base; k0 += 32) {
      const int64_t k = k0 + lane;
      uint32_t c = 0;
      if (k < base) c = ((k + 1 < base) ? cnts[k + 1] : (uint32_t)s) - cnts[k];
      __syncwarp();
      if (k < base) cnts[k] = c;
      __syncwarp();
    }
    if (lane == 0) {
      *d_out = base;
      s_d = base;
    }
  }
  __syncthreads();
  const int64_t dd = s_d;
  // suffix sums from the end, 1024 entries per step (thread t holds entry end - 1 - t)
  int64_t carryS = 0;
  double carryL = 0.0;
  if (threadIdx.x == 0) S[dd] = 0;
  for (int64_t e = dd; e > 0; e -= blockDim.x) {
    const int64_t i = e - 1 - threadIdx.x;
    const bool ok = i >= 0;
    int64_t c = ok ? (int64_t)cnts[i] : 0;
    double l = ok ? (double)c * log((double)vals[i]) : 0.0;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t yc = __shfl_up_sync(0xffffffffu, c, o);
      const double yl = __shfl_up_sync(0xffffffffu, l, o);
      if (lane >= o) {
        c += yc;
        l += yl;
      }
    }
    if (lane == 31) {
      s_part[warp] = c;
      s_dpart[warp] = l;
    }
    __syncthreads();
    if (warp == 0) {
      int64_t w = s_part[lane];
      double wl = s_dpart[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t yc = __shfl_up_sync(0xffffffffu, w, o);
        const double yl = __shfl_up_sync(0xffffffffu, wl, o);
        if (lane >= o) {
          w += yc;
          wl += yl;
        }
      }
      s_part[lane] = w;
      s_dpart[lane] = wl;
    }
    __syncthreads();
    const int64_t cS = c + (warp ? s_part[warp - 1] : 0) + carryS;
    const double cL = l + (warp ? s_dpart[warp - 1] : 0.0) + carryL;
    if (ok) {
      S[i] = cS;
      Lt[i] = cL;
    }
    const int64_t totS = s_part[31];
    const double totL = s_dpart[31];
    __syncthreads();
    carryS += totS;
    carryL += totL;
  }
}

// Safeguarded Newton for the MLE of the tail above xmin (Eq. 2), binary64,
// pow-based Euler-Maclaurin: the root of zeta'/zeta + mbar on (1 + 2^-40, 64],
// started at the continuous-law estimate, stopped within 4 ulp.
__device__ int xmin_fit(double mbar, double xmin, double *alpha_hat, double *Z) {
  double lo = 1.0 + 0x1p-40, hi = 64.0;
  double a = 1.0 + 1.0 / (mbar - log(xmin - 0.5));
  if (!(a > lo && a < hi)) a = 0.5 * (lo + hi);
  int it = 1;
  for (; it <= kNewtonCap; ++it) {
    double z[3];
    hurwitz_em<2, true>(a, xmin, z);
    const double g = z[1] / z[0];
    const double f = g + mbar;
    const double fp = z[2] / z[0] - g * g;
    if (f > 0.0)
      hi = a;
    else
      lo = a;
    double next = a - f / fp;
    if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
    const double step = fabs(next - a);
    a = next;
    const double tol = 4.0 * ldexp(1.0, ilogb(a) - 52);
    if (step <= tol || hi - lo <= tol) break;
  }
  *alpha_hat = a;
  double z0;
  hurwitz_em<0, true>(a, xmin, &z0);
  *Z = z0;
  return it;
}

__global__ void __launch_bounds__(kXWarps * 32) xmin_cand_kernel(const uint64_t *vals, const uint32_t *cnts,
                                                                 const int64_t *S, const double *Lt,
                                                                 const int64_t *d_in, int64_t max_cand,
                                                                 int64_t min_tail, uint64_t *c_xmin,
                                                                 double *c_alpha, double *c_D, int64_t *c_nt,
                                                                 Counters *ctr) {
  const int64_t j = blockIdx.x * (int64_t)kXWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int64_t d = *d_in;
  if (j >= d || j >= max_cand) return;  // warp-uniform
  const uint64_t xm = vals[j];
  const int64_t nt = S[j];
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  if (lane == 0) {
    c_xmin[j] = xm;
    c_nt[j] = nt;
  }
  if (nt < min_tail) {
    if (lane == 0) c_alpha[j] = c_D[j] = nan;
    return;
  }
  double a = 0.0, Z = 0.0;
  if (lane == 0) {
    double L = Lt[j];
    if ((int64_t)cnts[j] == nt) L += log1p(1.0 / (double)xm);  // every tail value equals xmin
    const int it = xmin_fit(L / (double)nt, (double)xm, &a, &Z);
    if (it > kNewtonCap) atomicAdd(&ctr->newton_capped, 1ull);
  }
  a = __shfl_sync(0xffffffffu, a, 0);
  Z = __shfl_sync(0xffffffffu, Z, 0);
  const double inv_nt = 1.0 / (double)nt;
  double best = 0.0;
  for (int64_t i = j + lane; i < d; i += 32) {
    const uint64_t v = vals[i];
    const double F1 = 1.0 - survival(a, Z, v);
    best = fmax(best, fabs(F1 - (double)(nt - S[i + 1]) * inv_nt));
    // t = v - 1 matters only after a gap: when the previous distinct value is
    // v - 1 the check there is the previous value's own
    if (i > j && vals[i - 1] != v - 1) {
      const double F0 = 1.0 - survival(a, Z, v - 1);
      best = fmax(best, fabs(F0 - (double)(nt - S[i]) * inv_nt));
    }
  }
  best = warp_max(best);
  if (lane == 0) {
    c_alpha[j] = a;
    c_D[j] = best;
  }
}

// The smallest D over the candidates (the first on ties), one block.
__global__ void __launch_bounds__(1024) xmin_pick_kernel(const uint64_t *c_xmin, const double *c_alpha,
                                                         const double *c_D, const int64_t *c_nt,
                                                         const int64_t *d_in, int64_t max_cand, XminOut *out) {
  __shared__ double s_best[32];
  __shared__ int64_t s_idx[32];
  const int64_t m = *d_in < max_cand ? *d_in : max_cand;
  double best = INFINITY;
  int64_t idx = -1;
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x) {
    const double v = c_D[j];
    if (v == v && (v < best || (v == best && j < idx))) {  // skip NaN
      best = v;
      idx = j;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (oi >= 0 && (idx < 0 || ob < best || (ob == best && oi < idx))) {
      best = ob;
      idx = oi;
    }
  }
  if (lane == 0) {
    s_best[warp] = best;
    s_idx[warp] = idx;
  }
  __syncthreads();
  if (warp == 0) {
    best = lane < (int)(blockDim.x >> 5) ? s_best[lane] : INFINITY;
    idx = lane < (int)(blockDim.x >> 5) ? s_idx[lane] : -1;
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int64_t oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (oi >= 0 && (idx < 0 || ob < best || (ob == best && oi < idx))) {
        best = ob;
        idx = oi;
      }
    }
    if (lane == 0) {
      out->candidates = m;
      out->best = idx;
      out->xmin = idx >= 0 ? c_xmin[idx] : 0;
      out->alpha_hat = idx >= 0 ? c_alpha[idx] : __longlong_as_double(0x7ff8000000000000ll);
      out->D = idx >= 0 ? c_D[idx] : __longlong_as_double(0x7ff8000000000000ll);
      out->n_tail = idx >= 0 ? c_nt[idx] : 0;
    }
  }
}

}  // namespace

cudaError_t launch_xmin(const int32_t *x, int64_t n, uint32_t *ghist, unsigned long long *nspill, uint64_t *spill,
                        uint64_t *vals, uint32_t *cnts, int64_t *S, double *Lt, int64_t *d, int64_t max_cand,
                        int64_t min_tail, uint64_t *c_xmin, double *c_alpha, double *c_D, int64_t *c_nt,
                        XminOut *out, Counters *ctr, int num_sms, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ghist, 0, sizeof(uint32_t) * kXHist, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(nspill, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const int64_t want = (n + 256 * 16 - 1) / (256 * 16);
  const int hblocks = (int)(want < 4 * num_sms ? (want < 1 ? 1 : want) : 4 * num_sms);
  xmin_hist_kernel<<<hblocks, 256, 0, st>>>(x, n, ghist, spill, nspill, ctr);
  xmin_prep_kernel<<<1, 1024, 0, st>>>(ghist, spill, nspill, vals, cnts, S, Lt, d, ctr);
  xmin_cand_kernel<<<(unsigned)((max_cand + kXWarps - 1) / kXWarps), kXWarps * 32, 0, st>>>(
      vals, cnts, S, Lt, d, max_cand, min_tail, c_xmin, c_alpha, c_D, c_nt, ctr);
  xmin_pick_kernel<<<1, 1024, 0, st>>>(c_xmin, c_alpha, c_D, c_nt, d, max_cand, out);
  return cudaGetLastError();
}

}  // namespace pl
