// pl_tables.cu -- per-call tables of the KS-cutoff simulation (sm_103a).
//
// The law tables of the inverse CDF (Section 4 of the paper: draws from
// p(k) = k^-alpha / zeta(alpha, xmin), Eq. 1): zeta(alpha, xmin), the integer
// thresholds T, two guides and the increment table; and the fit tables that
// give the maximum-likelihood exponent (Eq. 2) as a function of the mean log.
#include "pl_kernels.cuh"

namespace pl {
// ===========================================================================
// Law tables.

// Z = zeta(alpha, xmin), one warp per law: the lanes share the direct terms.
__global__ void law_z_kernel(Law *laws, int nlaws) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= nlaws) return;  // warp-uniform
  const double a = laws[i].alpha, x0 = (double)laws[i].xmin;
  const int M = em_shift(a, x0);
  double z = 0.0;
  for (int k = lane; k < M; k += 32) z += pow(x0 + (double)k, -a);
  z = warp_sum(z);
  if (lane != 0) return;
  double t;
  hurwitz_em_tail<0, true>(a, x0 + (double)M, &t);
  const double Z = z + t;
  laws[i].Z = Z;
  laws[i].tail_c = (float)((a - 1.0) * Z * 0x1p-32);
  laws[i].tail_e = (float)(-1.0 / (a - 1.0));
  laws[i].xmin_f = (float)(x0 + 0.5);
}

// T[i] = floor(Q(xmin+i) 2^53) + 1 and the log tables of xmin + i.
// Entries whose survival needs Euler-Maclaurin direct terms (argument below
// 10 + 1.5 alpha, at most ~100 entries) are left to law_fill_em_block.
__device__ __forceinline__ bool survival_needs_terms(const Law &law, uint32_t i) {
  return (double)(law.xmin + i) + 1.0 < 10.0 + 1.5 * law.alpha;
}

// blocks b of nb (256 threads each) of one law
__device__ __forceinline__ void law_fill_blocks(const Law &law, uint32_t b, uint32_t nb) {
  const uint32_t stride = nb * blockDim.x;
  for (uint32_t i = b * blockDim.x + threadIdx.x; i < law.L2 || i < (uint32_t)kLnTable; i += stride) {
    if (i < law.L2 && !survival_needs_terms(law, i)) {
      const double Q = survival(law.alpha, law.Z, law.xmin + i);
      law.T[i] = (uint64_t)(Q * 0x1p53) + 1ull;
    }
    if (i < (uint32_t)kLnTable) {
      const double l = log((double)(law.xmin + i));
      const float hi = (float)l;
      law.lnT[i] = l;
      law.lnT_hi[i] = hi;
      law.lnT_lo[i] = (float)(l - (double)hi);
    }
  }
}

// The first thresholds (survival with direct terms): one warp per entry, the
// lanes share the terms, a fixed-shape warp reduction adds them.
constexpr int kFillEmWarps = 8;

__device__ __forceinline__ void law_fill_em_block(const Law &law, uint32_t b) {
  const uint32_t i = b * kFillEmWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= law.L2 || !survival_needs_terms(law, i)) return;  // warp-uniform
  const double a = (double)(law.xmin + i) + 1.0;
  const int M = em_shift(law.alpha, a);
  double z = 0.0;
  for (int k = lane; k < M; k += 32) z += pow(a + (double)k, -law.alpha);
  z = warp_sum(z);
  if (lane == 0) {
    double t;
    hurwitz_em_tail<0, true>(law.alpha, a + (double)M, &t);
    law.T[i] = (uint64_t)((z + t) / law.Z * 0x1p53) + 1ull;
  }
}

// Both fills in one launch (they depend only on Z): the first kFillEmBlocks
// blocks of a law take the entries with direct terms, the others the rest.
constexpr uint32_t kFillEmBlocks = 128 / kFillEmWarps;  // entries with direct terms: i < 105 for alpha <= 64
constexpr uint32_t kFillBlocks = 256;

__global__ void __launch_bounds__(kFillEmWarps * 32) law_fill_kernel(Law *laws) {
  const Law law = laws[blockIdx.y];
  if (blockIdx.x < kFillEmBlocks) law_fill_em_block(law, blockIdx.x);
  else law_fill_blocks(law, blockIdx.x - kFillEmBlocks, kFillBlocks);
}

// guide[j] = min{i < L2 : T[i] <= (j+1) 2^(53-g)}, or L2, with kGuideMulti
// set unless the bucket's answers [guide[j], guide[j-1]] (L2 above bucket 0)
// are a single index.
template <int GB>
__device__ __forceinline__ uint32_t guide_bound(const Law &law, uint32_t j) {
  const uint64_t bound = (uint64_t)(j + 1) << (53 - GB);
  uint32_t lo = 0, hi = law.L2;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (law.T[mid] <= bound) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

template <int GB>
__device__ __forceinline__ void law_guide_block(const Law &law, uint32_t b) {
  const uint32_t j = b * blockDim.x + threadIdx.x;
  if (j >= (1u << GB)) return;
  const uint32_t lo = guide_bound<GB>(law, j);
  const uint32_t hi = j ? guide_bound<GB>(law, j - 1) : law.L2;
  (GB == kGuideBits ? law.guide : law.fine)[j] = lo | (hi != lo ? kGuideMulti : 0u);
}

// Increment table: bucket j of the high word covers m in [j 2^45 + 1,
// (j + 1) 2^45]; the answer index is nonincreasing in m, so it is one index
// over the bucket exactly when the answers at the two ends agree.
__device__ __forceinline__ uint32_t answer_at(const Law &law, uint64_t m) {
  uint32_t lo = 0, hi = law.L2;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (law.T[mid] <= m) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ void law_inc_block(const Law &law, uint32_t blk) {
  const uint32_t j = blk * 8 + (threadIdx.x >> 5), l = threadIdx.x & 31;
  if (j >= (uint32_t)kIncBuckets) return;
  const uint64_t m_lo = ((uint64_t)j << (53 - kIncBits)) + 1ull, m_hi = (uint64_t)(j + 1) << (53 - kIncBits);
  const uint32_t a = answer_at(law, m_lo), b = answer_at(law, m_hi);
  law.inc[j * 32 + l] = (a == b && a < 4) ? 1u << (8 * a) : kIncOther;
}

// The guides and the increment table in one launch (they depend only on T):
// blocks [0, 16) the 2^12-bucket guide, [16, 48) the 2^13-bucket guide,
// [48, 80) the increment table, 256 threads each.
constexpr uint32_t kGuideBlocks = kGuide / 256, kFineBlocks = kFine / 256, kIncBlocks = kIncBuckets / 8;

__global__ void __launch_bounds__(256) law_index_kernel(Law *laws) {
  const Law law = laws[blockIdx.y];
  const uint32_t b = blockIdx.x;
  if (b < kGuideBlocks) law_guide_block<kGuideBits>(law, b);
  else if (b < kGuideBlocks + kFineBlocks) law_guide_block<kFineBits>(law, b - kGuideBlocks);
  else law_inc_block(law, b - kGuideBlocks - kFineBlocks);
}

cudaError_t launch_law_setup(Law *laws_dev, int nlaws, cudaStream_t st) {
  if (nlaws <= 0) return cudaSuccess;
  law_z_kernel<<<(nlaws + 1) / 2, 64, 0, st>>>(laws_dev, nlaws);
  law_fill_kernel<<<dim3(kFillEmBlocks + kFillBlocks, nlaws), kFillEmWarps * 32, 0, st>>>(laws_dev);
  law_index_kernel<<<dim3(kGuideBlocks + kFineBlocks + kIncBlocks, nlaws), 256, 0, st>>>(laws_dev);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Fit tables (one Euler-Maclaurin evaluation per node, pow-based).
// Fit-table nodes in two passes.  First one warp per node sums the
// Euler-Maclaurin direct terms (the largest exponents need ~100 of them; the
// lanes share them, a fixed-shape warp reduction adds them) into the node's
// storage; then one thread per node adds the tail and forms the node, so the
// binary64 tail work runs on full warps.
constexpr int kFitNodeWarps = 8;

__device__ __forceinline__ double fit_node_alpha(const FitTable &ft, int k) {
  const double t_hi = log(kFitAlphaHi - 1.0), t_lo = log(kFitAlphaLo - 1.0);
  return 1.0 + exp(t_hi - (t_hi - t_lo) * (double)k / (double)(ft.nodes - 1));
}

__global__ void __launch_bounds__(kFitNodeWarps * 32) fit_sums_kernel(FitTable *fts) {
  const FitTable ft = fts[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * kFitNodeWarps + (threadIdx.x >> 5);
  if (k >= ft.nodes) return;  // warp-uniform
  const double a = fit_node_alpha(ft, k);
  const int M = em_shift(a, (double)ft.xmin);  // <= 100 < kLnTable
  double z0 = 0.0, z1 = 0.0, z2 = 0.0;
  for (int i = lane; i < M; i += 32) {
    const double lx = ft.lnx[i];
    const double tt = exp(-a * lx);  // node accuracy needs ~1e-13, not pow's last bit
    z0 += tt;
    z1 -= lx * tt;
    z2 += lx * lx * tt;
  }
  z0 = warp_sum(z0);
  z1 = warp_sum(z1);
  z2 = warp_sum(z2);
  if (lane == 0) {  // partial sums parked in the node until the second pass
    FitNode &nd = ft.node[k];
    nd.u = z0;
    nd.alpha = z1;
    nd.dadu = z2;
  }
}

__global__ void fit_nodes_kernel(FitTable *fts) {
  const FitTable ft = fts[blockIdx.y];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ft.nodes) return;
  const double a = fit_node_alpha(ft, k);
  const double x0 = (double)ft.xmin;
  FitNode &nd = ft.node[k];
  double z[3];
  hurwitz_em_tail<2, false>(a, x0 + (double)em_shift(a, x0), z);
  z[0] += nd.u;
  z[1] += nd.alpha;
  z[2] += nd.dadu;
  const double g = z[1] / z[0];
  const double h = -g - log(x0);
  const double var = z[2] / z[0] - g * g;
  nd.u = log(h);
  nd.alpha = a;
  nd.dadu = -h / var;
  nd.lnZ = log(z[0]);
  nd.dlnZdu = g * nd.dadu;  // d ln zeta / d alpha = zeta'/zeta
}

// inv_du of each interval, and the guide: guide[b] = max{k : u_k <= ug0 + b du_g}.
__global__ void fit_guide_kernel(FitTable *fts) {
  FitTable &ftr = fts[blockIdx.y];
  const FitTable ft = ftr;
  const double u_first = ft.node[0].u, u_last = ft.node[ft.nodes - 1].u;
  const double dug = (u_last - u_first) / (double)ft.guides;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ftr.ug0 = u_first;
    ftr.inv_dug = 1.0 / dug;
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ft.nodes - 1) ft.node[i].inv_du = 1.0 / (ft.node[i + 1].u - ft.node[i].u);
  if (i < ft.guides) {
    const double ub = u_first + dug * (double)i;
    int lo = 0, hi = ft.nodes - 1;  // last k with u_k <= ub
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ft.node[mid].u <= ub) lo = mid;
      else hi = mid - 1;
    }
    ft.guide[i] = lo;
  }
}

cudaError_t launch_fit_tables(FitTable *fts_dev, int nfit, cudaStream_t st) {
  if (nfit <= 0) return cudaSuccess;
  fit_sums_kernel<<<dim3((kFitNodes + kFitNodeWarps - 1) / kFitNodeWarps, nfit), kFitNodeWarps * 32, 0, st>>>(
      fts_dev);
  fit_nodes_kernel<<<dim3((kFitNodes + 127) / 128, nfit), 128, 0, st>>>(fts_dev);
  const int n = kFitNodes > kFitGuides ? kFitNodes : kFitGuides;
  fit_guide_kernel<<<dim3((n + 127) / 128, nfit), 128, 0, st>>>(fts_dev);
  return cudaGetLastError();
}

}  // namespace pl
