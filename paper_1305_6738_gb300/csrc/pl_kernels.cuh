// pl_kernels.cuh -- launch wrappers of the sm_103a kernels (host side).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "pl_device.cuh"

namespace pl {

// Per-cell constants that the host computes once (binary64).
struct CellConst {
  double ln_xmin_half;  // ln(xmin - 1/2): start of the Newton iteration
  double ln_allmin;     // ln((xmin + 1) / xmin): the all-equal rule
  double ln_xmin;       // ln(xmin)
};

cudaError_t launch_fit_tables(FitTable *fts_dev, int nfit, cudaStream_t st);

cudaError_t launch_law_setup(Law *laws_dev, int nlaws, cudaStream_t st);
constexpr int kLawSetupLaunches = 3;  // kernels launch_law_setup enqueues

cudaError_t launch_sample(const Law *law_dev, uint64_t seed, uint32_t cell_id, uint32_t purpose,
                          uint32_t rep0, int64_t nrep, int64_t n, uint64_t *out, Counters *ctr,
                          int num_sms, cudaStream_t st);

// Records of one wave of work items, written by the sampler and read by the
// finisher: dense histogram counts (uint16, H per replicate), spill values
// (uint64, scap per replicate) and (tmax, spill count) per replicate.
struct Records {
  uint16_t *dense;
  uint64_t *spill;
  int2 *meta;
};

struct TailQueue;
struct SampleLaunch {
  const Cell *cells;
  const Law *laws;
  const WorkItem *items;
  uint32_t nitems;
  RoundKeys rk;
  Records rec;
  Counters *ctr;
  int blocks;
  // queue of beyond-table draws (see TailQueue in the kernels)
  uint64_t *tq_pos;
  uint32_t *tq_law;
  unsigned int *tq_count;
  uint32_t tq_cap;
};
int sample_kernel_blocks_per_sm();
size_t sample_kernel_smem_bytes();
cudaError_t launch_sample_hist(const SampleLaunch &a, bool inl, cudaStream_t st);
int sample_lane_blocks_per_sm();
cudaError_t launch_sample_lane(const SampleLaunch &a, cudaStream_t st);
int block_sampler_blocks_per_sm();
cudaError_t launch_sample_block(const SampleLaunch &a, bool inl, cudaStream_t st);
cudaError_t launch_tail_queue_raw(const Law *laws, uint64_t *pos, uint32_t *law, unsigned int *count,
                                  uint32_t cap, uint64_t *spill, Counters *ctr, int num_sms, cudaStream_t st);

struct FinishLaunch {
  const Cell *cells;
  const CellConst *consts;
  const Law *laws;
  const FitTable *fits;
  const WorkItem *items;
  uint32_t nitems;
  RoundKeys rk;
  Records rec;
  void *D_out;            // double or float per precision
  double *A_out;          // may be null
  uint8_t *scratch;
  size_t spill_cap;       // uint64 entries per warp
  size_t arena_bytes;     // per warp
  Counters *ctr;
  int blocks;             // persistent grid size
  // the wave's tail queue: when it did not overflow, the tail kernel has
  // resolved every draw a sampler left beyond the table, and only replicates
  // drawn again here can hold such draws; null: the records may hold them
  const unsigned int *tq_count;
  uint32_t tq_cap;
};
int finish_kernel_blocks_per_sm(bool f32);
size_t finish_kernel_smem_bytes();
cudaError_t launch_finish(const FinishLaunch &a, bool f32, cudaStream_t st);

// Fit and/or KS of one data set.  out[0] = alpha-hat (or the given alpha),
// out[1] = D, out[2] = Z.
cudaError_t launch_dataset(const int32_t *x, int64_t n, uint64_t xmin, bool fit, double alpha,
                           const Law *lnlaw, CellConst cc, bool f32, uint64_t *spill,
                           uint64_t *pairs, double *out, Counters *ctr, cudaStream_t st);

// Order statistics: for cell c and quantile j, out[c*nq + j] = the rank[c*nq+j]-th
// smallest of keys[off[c] .. off[c] + R[c]).
cudaError_t launch_select(const void *keys, bool f32, const int64_t *off, const int64_t *R,
                          const int64_t *rank, int ncells, int nq, double *out, cudaStream_t st);

// p = #{D[b] >= D_obs} / B
cudaError_t launch_count_ge(const void *D, bool f32, int64_t B, const double *D_obs, double *p,
                            cudaStream_t st);

}  // namespace pl
