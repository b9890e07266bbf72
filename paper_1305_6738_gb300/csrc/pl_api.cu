// pl_api.cu -- host runtime behind the C ABI of include/pl.h.
//
// A context owns one device workspace inside a byte budget and a block of
// device counters.  Each call plans its buffers, grows the workspace if the
// plan needs it (never past the budget), stages its small host tables, sets
// up the law tables on the device, launches the kernels and, for host
// outputs, copies back and synchronises.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "pl.h"
#include "pl_kernels.cuh"
#include "pl_truncated.cuh"
#include "pl_lookup.cuh"
#include "pl_xmin.cuh"
#include "pl_multinomial.cuh"
#include "pl_probe.cuh"

using namespace pl;

struct pl_ctx {
  int device = 0;
  size_t budget = 0;
  std::string err;
  uint8_t *ws = nullptr;
  size_t ws_size = 0;
  Counters *ctr = nullptr;
  int num_sms = 0;
  int finish_blocks_per_sm[2] = {0, 0};
  int sample_blocks_per_sm = 0;
  int block_sampler_per_sm = 0;
  int lane_sampler_per_sm = 0;
  int64_t warp_split = 16384;    // n above this: block form
  int item_reps = 0;             // warp-form replicates per work item (0: sized by the plan)
  int hist_shift = 0;            // dense bins of a warp-form replicate: the default times 2^hist_shift
  uint64_t launches = 0;
  // Capacity overrides for tests (environment, read at pl_create; 0 = off):
  // they only shrink buffers so that the overflow fallbacks run.
  // PL_TEST_WAIT_CYCLES (cycles of the first shared-memory staging wait, in
  // the device counters) makes the bounded waits run out.
  uint32_t dbg_spill_cap = 0;    // PL_TEST_SPILL_SLOT: record spill slot entries
  uint32_t dbg_tail_cap = 0;     // PL_TEST_TAIL_QUEUE: tail-queue entries
  size_t dbg_arena = 0;          // PL_TEST_ARENA_BYTES: finisher arena bytes per warp
  bool tracing = false;
  bool traced = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> wave_ev;   // 4 per wave: sampler start/end, finisher start/end
  // Fit tables depend only on xmin: the context keeps those of the first
  // kFitCacheMax values of xmin it meets (nodes, guide and the finished
  // FitTable in one device allocation each, outside the byte budget).
  static constexpr size_t kFitCacheMax = 16;
  std::map<uint64_t, FitTable *> fit_cache;  // xmin -> the cached FitTable (device)
  std::vector<void *> fit_mem;
  uint32_t traced_waves = 0;
  uint32_t traced_sample_launches = 0;
  uint64_t traced_draws = 0;
  // pinned staging of the host-written tables and the event of its last copy
  void *staging = nullptr;
  size_t staging_size = 0;
  cudaEvent_t staging_ev = nullptr;
  bool staged = false;
  // side streams for independent small kernels inside one call (joined back
  // to the call's stream by events before the call continues)
  static constexpr int kAux = 8;
  cudaStream_t aux[kAux] = {};
  cudaEvent_t aux_ev[kAux + 1] = {};
};

namespace {

constexpr uint32_t kPurposeMultinomial = 3;  // stream tag of the multinomial sampler
constexpr int64_t kWarpNMax = 65535;     // warp form: n up to this (16-bit dense record counts)
constexpr int64_t kWideNMax = 1 << 21;   // block form: n up to this (16-bit lane counters)
constexpr uint32_t kWideItemReps = 8;    // block form: replicates per work item
#ifndef PL_INLINE_ALPHA
#define PL_INLINE_ALPHA 2.1
#endif
constexpr double kInlineAlpha = PL_INLINE_ALPHA;  // laws below this exponent bin in the draw loop
static_assert(kWideItemReps == kWideReps, "block-form items as the multinomial sampler reads them");

pl_status fail(pl_ctx *ctx, pl_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  return s;
}

#define PL_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(ctx, PL_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Workspace carving: the same sequence of take() calls sizes the plan (base
// null) and then hands out pointers.
struct Carver {
  uint8_t *base = nullptr;
  size_t off = 0;
  template <typename T>
  T *take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T *p = reinterpret_cast<T *>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

pl_status ensure_ws(pl_ctx *ctx, size_t bytes) {
  if (bytes > ctx->budget)
    return fail(ctx, PL_ENOMEM, "workspace of %zu bytes exceeds the budget of %zu", bytes, ctx->budget);
  if (bytes <= ctx->ws_size) return PL_OK;
  size_t want = std::min(ctx->budget, std::max(bytes, ctx->ws_size + ctx->ws_size / 2));
  PL_CUDA(cudaDeviceSynchronize());
  if (ctx->ws) PL_CUDA(cudaFree(ctx->ws));
  ctx->ws = nullptr;
  ctx->ws_size = 0;
  PL_CUDA(cudaMalloc(&ctx->ws, want));
  ctx->ws_size = want;
  return PL_OK;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Length of the inverse-CDF table: the smallest kL1 * 2^k (at most 2^20) at
// which the binary64 tail inversions it leaves (draws * P(X beyond), each about
// four times the cost of building one table entry) cost no more than the
// table itself.  Sizing only: uses the continuous tail approximation.
uint32_t table_length(double alpha, uint64_t xmin, double draws) {
  const double x = (double)xmin;
  const double Zapprox = std::pow(x, -alpha) + std::pow(x + 0.5, 1.0 - alpha) / (alpha - 1.0);
  uint32_t L = kL1;
  while (L < (1u << 20)) {
    const double Q = std::pow(x + L - 0.5, 1.0 - alpha) / ((alpha - 1.0) * Zapprox);
    if (4.0 * draws * Q <= (double)L) break;
    L <<= 1;
  }
  return L;
}

struct LawPlan {
  double alpha;
  uint64_t xmin;
  uint32_t L2;
};

// Allocate (or size, with a null carver base) one law's tables.
Law carve_law(Carver &cv, const LawPlan &lp) {
  Law l{};
  l.alpha = lp.alpha;
  l.xmin = lp.xmin;
  l.L2 = lp.L2;
  l.T = cv.take<uint64_t>(lp.L2);
  l.guide = cv.take<uint32_t>(kGuide);
  l.fine = cv.take<uint32_t>(kFine);
  l.inc = cv.take<uint32_t>((size_t)kIncBuckets * 32);
  l.lnT = cv.take<double>(kLnTable);
  l.lnT_hi = cv.take<float>(kLnTable);
  l.lnT_lo = cv.take<float>(kLnTable);
  return l;
}

CellConst cell_const(uint64_t xmin) {
  CellConst c;
  c.ln_xmin_half = std::log((double)xmin - 0.5);
  c.ln_allmin = std::log1p(1.0 / (double)xmin);
  c.ln_xmin = std::log((double)xmin);
  return c;
}

FitTable make_fit_table(Carver &cv, uint64_t xmin) {
  FitTable f{};
  f.xmin = xmin;
  f.nodes = kFitNodes;
  f.guides = kFitGuides;
  f.node = cv.take<FitNode>(kFitNodes);
  f.guide = cv.take<int>(kFitGuides);
  return f;
}

// Dense bins of a warp-form replicate: the smallest power of two >= 2n
// (32 .. kHMax), scaled by 2^shift within those bounds.
uint32_t hist_bins(int64_t n, int shift = 0) {
  int64_t H = 32;
  while (H < 2 * n && H < kHMax) H <<= 1;
  H = shift >= 0 ? H << shift : H >> -shift;
  return (uint32_t)std::min<int64_t>(kHMax, std::max<int64_t>(32, H));
}

// P(X >= xmin + H) by the continuous tail approximation.
double tail_beyond(double alpha, uint64_t xmin, uint32_t H) {
  const double x = (double)xmin;
  const double Zapprox = std::pow(x, -alpha) + std::pow(x + 0.5, 1.0 - alpha) / (alpha - 1.0);
  return std::min(1.0, std::pow(x + H - 0.5, 1.0 - alpha) / ((alpha - 1.0) * Zapprox));
}

// Spill slot of a replicate record: about twice the expected number of draws
// at or beyond xmin + H plus ten standard deviations (continuous tail
// approximation); a replicate that overflows it is drawn again by the finisher.
uint32_t spill_capacity(double alpha, uint64_t xmin, int64_t n, uint32_t H) {
  const double mu = (double)n * tail_beyond(alpha, xmin, H);
  const double cap = std::ceil(2.0 * mu + 10.0 * std::sqrt(mu) + 32.0);
  return (uint32_t)std::max<double>(1.0, std::min<double>((double)n, cap));
}

uint64_t next_pow2(uint64_t v) {
  uint64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Everything one batch of replicate cells needs on the device.
struct Wave {
  size_t first, count;             // items [first, first + count)
  size_t wide;                     // the first `wide` items are block-form cells
  size_t wide_inl, warp_inl;       // of the block-form and of the warp-form items, the first so many bin inline
  size_t lane;                     // the next `lane` items (after the block form) are drawn in the lane form
};

struct SimPlan {
  uint32_t tail_cap = 0;           // tail-queue entries (largest wave)
  std::vector<uint64_t> fit_xmins;
  std::vector<LawPlan> laws;
  std::vector<Cell> cells;
  std::vector<CellConst> consts;
  std::vector<WorkItem> items;
  std::vector<Wave> waves;
  size_t dense_elems = 0, spill_elems = 0, meta_elems = 0;  // largest wave
  int64_t total_R = 0;
  int64_t n_max = 0;
  int64_t finisher_spill = 0;      // spills one finisher warp must hold for one replicate
};

pl_status plan_cells(pl_ctx *ctx, const pl_cell *in, int ncells, uint32_t purpose, SimPlan &sp,
                     bool all_wide = false) {
  std::map<std::pair<double, uint64_t>, uint32_t> law_of;
  std::map<uint64_t, uint32_t> fit_of;
  std::vector<double> law_draws;
  sp.cells.resize(ncells);
  sp.consts.resize(ncells);
  for (int c = 0; c < ncells; ++c) {
    const pl_cell &x = in[c];
    if (!(x.alpha > 1.0) || !std::isfinite(x.alpha) || x.alpha > 64.0)
      return fail(ctx, PL_EINVAL, "cell %d: alpha must be in (1, 64]", c);
    if (x.xmin < 1 || x.xmin > (1ull << 40)) return fail(ctx, PL_EINVAL, "cell %d: xmin out of range", c);
    if (x.n < 1) return fail(ctx, PL_EINVAL, "cell %d: n < 1", c);
    if (x.n > kWideNMax)
      return fail(ctx, PL_EINVAL, "cell %d: n = %lld exceeds %lld", c, (long long)x.n, (long long)kWideNMax);
    if (x.replicates < 1 || x.replicates > (1ll << 31)) return fail(ctx, PL_EINVAL, "cell %d: replicates", c);
    if (x.cell_id >= (1ull << 32)) return fail(ctx, PL_EINVAL, "cell %d: cell_id >= 2^32", c);
    const auto key = std::make_pair(x.alpha, x.xmin);
    auto it = law_of.find(key);
    uint32_t li;
    if (it == law_of.end()) {
      li = (uint32_t)sp.laws.size();
      law_of[key] = li;
      sp.laws.push_back({x.alpha, x.xmin, 0});
      law_draws.push_back(0.0);
    } else {
      li = it->second;
    }
    law_draws[li] += (double)x.n * (double)x.replicates;
    Cell &cd = sp.cells[c];
    cd.alpha = x.alpha;
    cd.xmin = x.xmin;
    cd.n = x.n;
    cd.R = x.replicates;
    cd.cell_id = (uint32_t)x.cell_id;
    cd.law = li;
    cd.wide = (all_wide || x.n > std::min(kWarpNMax, ctx->warp_split)) ? 1u : 0u;
    cd.H = cd.wide ? (uint32_t)kHWide : hist_bins(x.n, ctx->hist_shift);
    // heavy tails (a third of the draws beyond the first four values at alpha
    // 1.5): their single-valued draws are binned in the draw loop instead of
    // queued; lighter tails queue them all (measured crossover on GB300)
    cd.inline_bins = x.alpha < kInlineAlpha ? 1u : 0u;
    // longer lane-serial finishing pays off in throughput (many replicates
    // per finisher warp); a small cell keeps the shorter lanes, whose latency
    // is lower.  Decided per cell, so a cell's results never depend on what
    // it is simulated with.
    cd.lane_bins = x.replicates >= kLaneLongMinReps ? kLaneBinsLong : kLaneBinsShort;
    // the fewest dense bins (64, 128 or 256) beyond which at most
    // kLightSpills values per replicate are expected (those become spills), so
    // that records are short and almost every replicate is finished by a lane
    if (!cd.wide)
      for (uint32_t h = kLaneSampleBins; h < cd.H && h <= kLaneBinsLong; h <<= 1)
        if ((double)x.n * tail_beyond(x.alpha, x.xmin, h) <= kLightSpills) {
          cd.H = h;
          break;
        }
    // small histograms of small samples: one thread per replicate draws the
    // whole sample (a shortened histogram only in a cell of many replicates:
    // a small simulation keeps the warp form's parallelism)
    cd.lane_sample = (!cd.wide && cd.H <= kLaneSampleBins && x.n <= kLaneSampleNMax &&
                      (hist_bins(x.n, ctx->hist_shift) <= kLaneSampleBins || x.replicates >= kLaneLongMinReps))
                         ? 1u
                         : 0u;
    cd.purpose = purpose;
    cd.out_off = sp.total_R;
    auto fi = fit_of.find(x.xmin);
    if (fi == fit_of.end()) {
      fi = fit_of.emplace(x.xmin, (uint32_t)sp.fit_xmins.size()).first;
      sp.fit_xmins.push_back(x.xmin);
    }
    cd.fit = fi->second;
    cd.scap = spill_capacity(x.alpha, x.xmin, x.n, cd.H);
    if (ctx->dbg_spill_cap) cd.scap = std::min(cd.scap, ctx->dbg_spill_cap);
    // never below what a lane-finished replicate may hold, so that whether a
    // replicate is finished by a lane does not depend on the slot size
    cd.scap = std::max<uint32_t>(cd.scap, (uint32_t)std::min<int64_t>(x.n, kLaneSpills));
    sp.finisher_spill = std::max<int64_t>(sp.finisher_spill, cd.wide ? 2 * (int64_t)cd.scap : x.n);
    sp.total_R += x.replicates;
    sp.n_max = std::max(sp.n_max, x.n);
    sp.consts[c] = cell_const(x.xmin);
  }
  // The samplers histogram table indices below H and treat index L2 as
  // "beyond the table", so every law's table must reach past H.
  std::vector<uint32_t> law_hmax(sp.laws.size(), 0);
  for (const Cell &cd : sp.cells) law_hmax[cd.law] = std::max(law_hmax[cd.law], cd.H);
  for (size_t l = 0; l < sp.laws.size(); ++l)
    sp.laws[l].L2 = std::max<uint32_t>(table_length(sp.laws[l].alpha, sp.laws[l].xmin, law_draws[l]),
                                       (uint32_t)next_pow2(2 * (uint64_t)law_hmax[l]));
  // work items: block form first, then inline binning first (one launch per
  // form and mode), cells grouped by law (the block keeps a law's table
  // staged), larger n first within a law
  std::vector<int> order(ncells);
  for (int c = 0; c < ncells; ++c) order[c] = c;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (sp.cells[a].wide != sp.cells[b].wide) return sp.cells[a].wide > sp.cells[b].wide;
    if (sp.cells[a].lane_sample != sp.cells[b].lane_sample) return sp.cells[a].lane_sample > sp.cells[b].lane_sample;
    if (sp.cells[a].inline_bins != sp.cells[b].inline_bins) return sp.cells[a].inline_bins > sp.cells[b].inline_bins;
    if (sp.cells[a].law != sp.cells[b].law) return sp.cells[a].law < sp.cells[b].law;
    return sp.cells[a].n > sp.cells[b].n;
  });
  // items, and waves whose replicate records fit the wave byte budget
  const size_t wave_budget = std::min<size_t>(ctx->budget / 4, (size_t)16 << 30);
  // Warp-form items hold up to kItemReps replicates; a small simulation gets
  // smaller items (down to 32) so that there are at least two per resident
  // sampler block.  Results do not depend on the item size.
  int64_t warp_R = 0;
  for (const Cell &cd : sp.cells)
    if (!cd.wide) warp_R += cd.R;
  const int64_t fill = 2 * (int64_t)ctx->num_sms * std::max(1, ctx->sample_blocks_per_sm);
  int64_t warp_item = kItemReps;
  while (warp_item > 32 && warp_R / warp_item < fill) warp_item /= 2;
  if (ctx->item_reps) warp_item = ctx->item_reps;
  size_t wd = 0, ws = 0, wm = 0, first = 0, nwide = 0, nwide_inl = 0, nwarp_inl = 0, nlane = 0;
  double wt = 0.0;  // expected beyond-table draws of the wave
  auto close_tail = [&]() {
    const double cap = std::ceil(2.0 * wt + 10.0 * std::sqrt(wt) + 1024.0);
    sp.tail_cap = std::max<uint32_t>(sp.tail_cap, (uint32_t)std::min(cap, 268435456.0));
  };
  for (int c : order) {
    const Cell &cd = sp.cells[c];
    const LawPlan &lp = sp.laws[cd.law];
    const double xq = (double)lp.xmin;
    const double Zq = std::pow(xq, -lp.alpha) + std::pow(xq + 0.5, 1.0 - lp.alpha) / (lp.alpha - 1.0);
    const double q_tail = std::min(1.0, std::pow(xq + lp.L2 - 0.5, 1.0 - lp.alpha) / ((lp.alpha - 1.0) * Zq));
    const int64_t per_item = cd.wide ? (int64_t)kWideItemReps : warp_item;
    for (int64_t r0 = 0; r0 < cd.R; r0 += per_item) {
      WorkItem it{};
      it.cell = (uint32_t)c;
      it.r0 = (uint32_t)r0;
      it.nrep = (uint32_t)std::min<int64_t>(per_item, cd.R - r0);
      const size_t d = (size_t)it.nrep * cd.H * (cd.wide ? 2 : 1), sp_ = (size_t)it.nrep * cd.scap, m = it.nrep;
      const size_t bytes_after = (wd + d) * 2 + (ws + sp_) * 8 + (wm + m) * 8;
      if (sp.items.size() > first && bytes_after > wave_budget) {
        sp.waves.push_back({first, sp.items.size() - first, nwide, nwide_inl, nwarp_inl, nlane});
        close_tail();
        first = sp.items.size();
        wd = ws = wm = 0;
        nwide = nwide_inl = nwarp_inl = nlane = 0;
        wt = 0.0;
      }
      if (cd.wide) ++nwide;
      if (cd.lane_sample) ++nlane;
      else if (cd.inline_bins) ++(cd.wide ? nwide_inl : nwarp_inl);
      wt += (double)it.nrep * (double)cd.n * q_tail;
      it.dense_off = wd;
      it.spill_off = ws;
      it.meta_off = wm;
      wd += d;
      ws += sp_;
      wm += m;
      sp.dense_elems = std::max(sp.dense_elems, wd);
      sp.spill_elems = std::max(sp.spill_elems, ws);
      sp.meta_elems = std::max(sp.meta_elems, wm);
      sp.items.push_back(it);
    }
  }
  sp.waves.push_back({first, sp.items.size() - first, nwide, nwide_inl, nwarp_inl, nlane});
  close_tail();
  if (ctx->dbg_tail_cap) sp.tail_cap = std::min(sp.tail_cap, ctx->dbg_tail_cap);
  return PL_OK;
}

struct SimBuffers {
  size_t host_bytes;      // laws_dev .. end of items: the host-written block
  FitTable *fits_dev;
  std::vector<FitTable> fits_host;
  Law *laws_dev;
  std::vector<Law> laws_host;
  Cell *cells;
  CellConst *consts;
  WorkItem *items;
  Records rec;
  uint64_t *tq_pos;
  uint32_t *tq_law;
  unsigned int *tq_count;
  uint8_t *scratch;
  size_t spill_cap, arena_bytes;
  int blocks, sample_blocks, block_sampler_blocks;
};

// Lay out (or size) the device buffers of a simulation plan.
void carve_sim(Carver &cv, const SimPlan &sp, int blocks, int sample_blocks, SimBuffers &b, size_t arena_override,
               int block_sampler_blocks) {
  // the small tables written from the host, contiguous: one copy uploads them
  b.laws_dev = cv.take<Law>(sp.laws.size());
  b.fits_dev = cv.take<FitTable>(sp.fit_xmins.size());
  b.cells = cv.take<Cell>(sp.cells.size());
  b.consts = cv.take<CellConst>(sp.consts.size());
  b.items = cv.take<WorkItem>(sp.items.size());
  b.host_bytes = (size_t)(reinterpret_cast<uint8_t *>(b.items + sp.items.size()) -
                          reinterpret_cast<uint8_t *>(b.laws_dev));
  b.fits_host.clear();
  for (uint64_t xm : sp.fit_xmins) b.fits_host.push_back(make_fit_table(cv, xm));
  b.laws_host.clear();
  for (const auto &lp : sp.laws) b.laws_host.push_back(carve_law(cv, lp));
  b.rec.dense = cv.take<uint16_t>(sp.dense_elems);
  b.rec.spill = cv.take<uint64_t>(sp.spill_elems);
  b.rec.meta = cv.take<int2>(sp.meta_elems);
  b.tq_pos = cv.take<uint64_t>(sp.tail_cap);
  b.tq_law = cv.take<uint32_t>(sp.tail_cap);
  b.tq_count = cv.take<unsigned int>(1);
  b.spill_cap = next_pow2((uint64_t)std::max<int64_t>(sp.finisher_spill, kSortSmem));
  b.arena_bytes = ((16 * (size_t)sp.finisher_spill + 16) + (size_t)32 * 2048 + 255) & ~(size_t)255;
  if (arena_override) b.arena_bytes = std::max<size_t>(16 * (size_t)sp.finisher_spill + 16, arena_override);
  // finisher grid: no more blocks than the largest wave has items (each
  // block's warps own a scratch slot)
  size_t max_items = 1;
  for (const Wave &w : sp.waves) max_items = std::max(max_items, w.count);
  b.blocks = (int)std::min<size_t>((size_t)blocks, max_items);
  b.sample_blocks = sample_blocks;
  b.block_sampler_blocks = block_sampler_blocks;
  b.scratch = cv.take<uint8_t>((size_t)b.blocks * kWarps * (b.spill_cap * 8 + b.arena_bytes));
}

// Pinned staging of the host-written tables, reused across calls; the copy
// of the previous call must have left it before it is rewritten.
pl_status staging(pl_ctx *ctx, size_t bytes, uint8_t **out) {
  if (ctx->staged) PL_CUDA(cudaEventSynchronize(ctx->staging_ev));
  if (bytes > ctx->staging_size) {
    if (ctx->staging) PL_CUDA(cudaFreeHost(ctx->staging));
    ctx->staging = nullptr;
    ctx->staging_size = 0;
    PL_CUDA(cudaMallocHost(&ctx->staging, std::max<size_t>(bytes, 1 << 16)));
    ctx->staging_size = std::max<size_t>(bytes, 1 << 16);
  }
  if (!ctx->staging_ev) PL_CUDA(cudaEventCreateWithFlags(&ctx->staging_ev, cudaEventDisableTiming));
  *out = static_cast<uint8_t *>(ctx->staging);
  return PL_OK;
}

pl_status upload_sim(pl_ctx *ctx, const SimPlan &sp, SimBuffers &b, cudaStream_t st) {
  std::vector<size_t> fresh;                             // fit tables to build
  std::vector<std::pair<size_t, FitTable *>> from, to;  // copies from / into the cache
  for (size_t i = 0; i < b.fits_host.size(); ++i) {
    const uint64_t xm = b.fits_host[i].xmin;
    auto it = ctx->fit_cache.find(xm);
    if (it != ctx->fit_cache.end()) {
      from.push_back({i, it->second});
      continue;
    }
    if (ctx->fit_cache.size() < pl_ctx::kFitCacheMax) {
      void *mem = nullptr;
      const size_t tab = sizeof(FitNode) * kFitNodes + sizeof(int) * kFitGuides;
      PL_CUDA(cudaMalloc(&mem, tab + sizeof(FitTable)));
      ctx->fit_mem.push_back(mem);
      b.fits_host[i].node = reinterpret_cast<FitNode *>(mem);
      b.fits_host[i].guide = reinterpret_cast<int *>(reinterpret_cast<FitNode *>(mem) + kFitNodes);
      to.push_back({i, reinterpret_cast<FitTable *>(static_cast<uint8_t *>(mem) + tab)});
    }
    fresh.push_back(i);
  }
  // fresh fit tables read ln(xmin + i) from a law of the same xmin (filled by
  // the law set-up, which runs first)
  for (size_t i : fresh) {
    b.fits_host[i].lnx = nullptr;
    for (const Law &l : b.laws_host)
      if (l.xmin == b.fits_host[i].xmin) {
        b.fits_host[i].lnx = l.lnT;
        break;
      }
    if (!b.fits_host[i].lnx) return fail(ctx, PL_ECUDA, "internal: no law for fit table xmin %llu",
                                         (unsigned long long)b.fits_host[i].xmin);
  }
  uint8_t *img = nullptr;
  if (pl_status e = staging(ctx, b.host_bytes, &img)) return e;
  const uint8_t *base = reinterpret_cast<const uint8_t *>(b.laws_dev);
  auto put = [&](const void *dev, const void *src, size_t bytes) {
    if (bytes) std::memcpy(img + (reinterpret_cast<const uint8_t *>(dev) - base), src, bytes);
  };
  put(b.laws_dev, b.laws_host.data(), sizeof(Law) * b.laws_host.size());
  put(b.fits_dev, b.fits_host.data(), sizeof(FitTable) * b.fits_host.size());
  put(b.cells, sp.cells.data(), sizeof(Cell) * sp.cells.size());
  put(b.consts, sp.consts.data(), sizeof(CellConst) * sp.consts.size());
  put(b.items, sp.items.data(), sizeof(WorkItem) * sp.items.size());
  PL_CUDA(cudaMemcpyAsync(b.laws_dev, img, b.host_bytes, cudaMemcpyHostToDevice, st));
  PL_CUDA(cudaEventRecord(ctx->staging_ev, st));
  ctx->staged = true;
  PL_CUDA(launch_law_setup(b.laws_dev, (int)b.laws_host.size(), st));
  ctx->launches += b.laws_host.empty() ? 0 : kLawSetupLaunches;
  if (fresh.size() == b.fits_host.size()) {
    PL_CUDA(launch_fit_tables(b.fits_dev, (int)b.fits_host.size(), st));
    ctx->launches += b.fits_host.empty() ? 0 : 3;
  } else {
    for (size_t i : fresh) PL_CUDA(launch_fit_tables(b.fits_dev + i, 1, st));
    ctx->launches += 3 * fresh.size();
  }
  // stream-ordered device copies of the finished FitTable (its guide origin
  // is set on the device): into the cache after a build, out of it for the
  // tables built by an earlier call (after this call's upload overwrote them)
  for (const auto &c : to) {
    PL_CUDA(cudaMemcpyAsync(c.second, b.fits_dev + c.first, sizeof(FitTable), cudaMemcpyDeviceToDevice, st));
    ctx->fit_cache[b.fits_host[c.first].xmin] = c.second;
  }
  for (const auto &c : from)
    PL_CUDA(cudaMemcpyAsync(b.fits_dev + c.first, c.second, sizeof(FitTable), cudaMemcpyDeviceToDevice, st));
  return PL_OK;
}

pl_status run_sim(pl_ctx *ctx, const SimPlan &sp, SimBuffers &b, uint64_t seed, bool f32, void *D,
                  double *A, cudaStream_t st, bool trace = true) {
  const RoundKeys rk = round_keys(seed);
  trace = trace && ctx->tracing;
  if (trace) {
    while (ctx->wave_ev.size() < 4 * sp.waves.size()) {
      cudaEvent_t e;
      PL_CUDA(cudaEventCreate(&e));
      ctx->wave_ev.push_back(e);
    }
    ctx->traced_waves = (uint32_t)sp.waves.size();
    ctx->traced_sample_launches = 0;
    ctx->traced_draws = 0;
    for (const Cell &c : sp.cells) ctx->traced_draws += (uint64_t)c.n * (uint64_t)c.R;
  }
  size_t wi_ = 0;
  for (const Wave &w : sp.waves) {
    cudaEvent_t *wev = trace ? &ctx->wave_ev[4 * wi_] : nullptr;
    ++wi_;
    SampleLaunch sl{};
    sl.cells = b.cells;
    sl.laws = b.laws_dev;
    sl.rk = rk;
    sl.rec = b.rec;
    sl.ctr = ctx->ctr;
    sl.tq_pos = b.tq_pos;
    sl.tq_law = b.tq_law;
    sl.tq_count = b.tq_count;
    sl.tq_cap = sp.tail_cap;
    PL_CUDA(cudaMemsetAsync(&ctx->ctr->work_next, 0, sizeof(unsigned int), st));
    PL_CUDA(cudaMemsetAsync(b.tq_count, 0, sizeof(unsigned int), st));
    if (wev) PL_CUDA(cudaEventRecord(wev[0], st));
    // the wave's items in five runs: block form (inline binning, then not),
    // lane form, warp form (inline binning, then not); a launch per nonempty
    // run, each with its own count
    const size_t wl = w.first + w.wide + w.lane;  // the first warp-form item
    const size_t run_first[5] = {w.first, w.first + w.wide_inl, w.first + w.wide, wl, wl + w.warp_inl};
    const size_t run_count[5] = {w.wide_inl, w.wide - w.wide_inl, w.lane, w.warp_inl,
                                 w.count - w.wide - w.lane - w.warp_inl};
    bool counter_used = false;
    for (int r = 0; r < 5; ++r) {
      if (!run_count[r]) continue;
      if (counter_used) PL_CUDA(cudaMemsetAsync(&ctx->ctr->work_next, 0, sizeof(unsigned int), st));
      counter_used = true;
      sl.items = b.items + run_first[r];
      sl.nitems = (uint32_t)run_count[r];
      if (r < 2) {
        sl.blocks = (int)std::min<size_t>((size_t)b.block_sampler_blocks, run_count[r]);
        PL_CUDA(launch_sample_block(sl, r == 0, st));
      } else if (r == 2) {
        sl.blocks = (int)std::min<size_t>((size_t)ctx->num_sms * std::max(1, ctx->lane_sampler_per_sm), run_count[r]);
        PL_CUDA(launch_sample_lane(sl, st));
      } else {
        sl.blocks = (int)std::min<size_t>((size_t)b.sample_blocks, run_count[r]);
        PL_CUDA(launch_sample_hist(sl, r == 3, st));
      }
      ctx->launches += 1;
      if (trace) ++ctx->traced_sample_launches;
    }
    if (wev) PL_CUDA(cudaEventRecord(wev[1], st));
    PL_CUDA(launch_tail_queue_raw(b.laws_dev, b.tq_pos, b.tq_law, b.tq_count, sp.tail_cap, b.rec.spill, ctx->ctr,
                                  ctx->num_sms, st));
    FinishLaunch fl{};
    fl.cells = b.cells;
    fl.consts = b.consts;
    fl.laws = b.laws_dev;
    fl.fits = b.fits_dev;
    fl.items = b.items + w.first;
    fl.nitems = (uint32_t)w.count;
    fl.rk = rk;
    fl.rec = b.rec;
    fl.D_out = D;
    fl.A_out = A;
    fl.scratch = b.scratch;
    fl.spill_cap = b.spill_cap;
    fl.arena_bytes = b.arena_bytes;
    fl.ctr = ctx->ctr;
    fl.blocks = (int)std::min<size_t>((size_t)b.blocks, w.count);
    fl.tq_count = b.tq_count;  // the sampler's beyond-table draws were queued and resolved
    fl.tq_cap = sp.tail_cap;
    PL_CUDA(cudaMemsetAsync(&ctx->ctr->work_next, 0, sizeof(unsigned int), st));
    if (wev) PL_CUDA(cudaEventRecord(wev[2], st));
    PL_CUDA(launch_finish(fl, f32, st));
    if (wev) PL_CUDA(cudaEventRecord(wev[3], st));
    ctx->launches += 2;
  }
  return PL_OK;
}

// The same waves with the multinomial sampler in place of the samplers (every
// cell in the block form, so each record has 32-bit counts for 8,192 values).
pl_status run_sim_mn(pl_ctx *ctx, const SimPlan &sp, SimBuffers &b, uint64_t seed, bool f32, void *D, double *A,
                     cudaStream_t st) {
  const RoundKeys rk = round_keys(seed);
  const bool trace = ctx->tracing;
  if (trace) {
    while (ctx->wave_ev.size() < 4 * sp.waves.size()) {
      cudaEvent_t e;
      PL_CUDA(cudaEventCreate(&e));
      ctx->wave_ev.push_back(e);
    }
    ctx->traced_waves = (uint32_t)sp.waves.size();
    ctx->traced_sample_launches = (uint32_t)sp.waves.size();
    ctx->traced_draws = 0;
    for (const Cell &c : sp.cells) ctx->traced_draws += (uint64_t)c.n * (uint64_t)c.R;
  }
  size_t wi_ = 0;
  for (const Wave &w : sp.waves) {
    cudaEvent_t *wev = trace ? &ctx->wave_ev[4 * wi_] : nullptr;
    ++wi_;
    MnLaunch ml{};
    ml.cells = b.cells;
    ml.laws = b.laws_dev;
    ml.items = b.items + w.first;
    ml.nitems = (uint32_t)w.count;
    ml.rk = rk;
    ml.rec = b.rec;
    ml.ctr = ctx->ctr;
    if (wev) PL_CUDA(cudaEventRecord(wev[0], st));
    PL_CUDA(launch_mn_sample(ml, st));
    if (wev) PL_CUDA(cudaEventRecord(wev[1], st));
    FinishLaunch fl{};
    fl.cells = b.cells;
    fl.consts = b.consts;
    fl.laws = b.laws_dev;
    fl.fits = b.fits_dev;
    fl.items = b.items + w.first;
    fl.nitems = (uint32_t)w.count;
    fl.rk = rk;
    fl.rec = b.rec;
    fl.D_out = D;
    fl.A_out = A;
    fl.scratch = b.scratch;
    fl.spill_cap = b.spill_cap;
    fl.arena_bytes = b.arena_bytes;
    fl.ctr = ctx->ctr;
    fl.blocks = (int)std::min<size_t>((size_t)b.blocks, w.count);
    PL_CUDA(cudaMemsetAsync(&ctx->ctr->work_next, 0, sizeof(unsigned int), st));
    if (wev) PL_CUDA(cudaEventRecord(wev[2], st));
    PL_CUDA(launch_finish(fl, f32, st));
    if (wev) PL_CUDA(cudaEventRecord(wev[3], st));
    ctx->launches += 2;
  }
  return PL_OK;
}

int sim_blocks(pl_ctx *ctx, bool f32) {
  return ctx->num_sms * std::max(1, ctx->finish_blocks_per_sm[f32 ? 1 : 0]);
}

int sample_blocks(pl_ctx *ctx) { return ctx->num_sms * std::max(1, ctx->sample_blocks_per_sm); }

pl_status mark(pl_ctx *ctx, int i, cudaStream_t st) {
  if (!ctx->tracing) return PL_OK;
  PL_CUDA(cudaEventRecord(ctx->ev[i], st));
  if (i == 3) ctx->traced = true;
  return PL_OK;
}

pl_status check_ctx(pl_ctx *ctx) {
  if (!ctx) return PL_EINVAL;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, PL_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  return PL_OK;
}

pl_status read_status(pl_ctx *ctx, cudaStream_t st) {
  PL_CUDA(cudaStreamSynchronize(st));
  unsigned int status = 0;
  PL_CUDA(cudaMemcpy(&status, &ctx->ctr->status, sizeof status, cudaMemcpyDeviceToHost));
  if (status) {
    PL_CUDA(cudaMemset(&ctx->ctr->status, 0, sizeof status));
    if (status & kErrTimeout) return fail(ctx, PL_ETIMEOUT, "a bounded device wait ran out");
    if (status & kErrData) return fail(ctx, PL_EINVAL, "a data value is below xmin (or below 1)");
    if (status & kErrArena) return fail(ctx, PL_ECUDA, "internal: replicate arena too small");
  }
  return PL_OK;
}

}  // namespace

// Hooks for the serving engine (pl_server.cu).
namespace pl {
uint64_t ctx_launches(const pl_ctx *ctx) { return ctx->launches; }

// Device bytes a bootstrap request of n values and B replicates plans (the
// data-set pass and the simulation), sized at exponent 1.4: the spill slots,
// tail queue and tables grow as the fitted exponent falls, and 1.4 covers
// power-law data with alpha >= 1.5 and the rounded-lognormal alternative.
size_t ctx_bootstrap_bytes(pl_ctx *ctx, int64_t n, uint64_t xmin, int64_t B) {
  pl_cell cell{1.4, xmin, n, B, 0};
  SimPlan sp;
  if (plan_cells(ctx, &cell, 1, 1u, sp) != PL_OK) return 0;
  const int blocks = sim_blocks(ctx, true), sblocks = sample_blocks(ctx),
            bsblocks = ctx->num_sms * std::max(1, ctx->block_sampler_per_sm);
  Carver cv;
  SimBuffers b;
  carve_sim(cv, sp, blocks, sblocks, b, ctx->dbg_arena, bsblocks);
  cv.take<uint8_t>((size_t)B * 8);  // as run_bootstrap lays out its buffers
  cv.take<double>(1);
  cv.take<double>(1);
  cv.take<int64_t>(3);
  cv.take<double>(1);
  const size_t sim = cv.off;
  const size_t data = (size_t)next_pow2((uint64_t)n) * 8 + (size_t)n * 16 + (1u << 20);
  return std::max(sim, data);
}
}  // namespace pl

// ===========================================================================
extern "C" {

pl_status pl_create(pl_ctx **out, int device, size_t mem_budget_bytes) {
  if (!out) return PL_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return PL_EINVAL;
  pl_ctx *ctx = new pl_ctx();
  ctx->device = device;
  ctx->budget = mem_budget_bytes ? mem_budget_bytes : (size_t)40 << 30;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&ctx->ctr, sizeof(Counters)) != cudaSuccess ||
      cudaMemset(ctx->ctr, 0, sizeof(Counters)) != cudaSuccess) {
    if (ctx->ctr) cudaFree(ctx->ctr);
    delete ctx;
    return PL_ECUDA;
  }
  if (const char *e = getenv("PL_TEST_SPILL_SLOT")) ctx->dbg_spill_cap = (uint32_t)strtoul(e, nullptr, 10);
  if (const char *e = getenv("PL_TEST_TAIL_QUEUE")) ctx->dbg_tail_cap = (uint32_t)strtoul(e, nullptr, 10);
  if (const char *e = getenv("PL_TEST_ARENA_BYTES")) ctx->dbg_arena = (size_t)strtoull(e, nullptr, 10);
  if (const char *e = getenv("PL_TEST_WAIT_CYCLES")) {
    const unsigned long long w = strtoull(e, nullptr, 10);
    if (cudaMemcpy(&ctx->ctr->wait_limit, &w, sizeof w, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(ctx->ctr);
      delete ctx;
      return PL_ECUDA;
    }
  }
  ctx->finish_blocks_per_sm[0] = finish_kernel_blocks_per_sm(false);
  ctx->finish_blocks_per_sm[1] = finish_kernel_blocks_per_sm(true);
  ctx->sample_blocks_per_sm = sample_kernel_blocks_per_sm();
  ctx->block_sampler_per_sm = block_sampler_blocks_per_sm();
  ctx->lane_sampler_per_sm = sample_lane_blocks_per_sm();
  cudaGetLastError();
  *out = ctx;
  return PL_OK;
}

void pl_destroy(pl_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto &e : ctx->ev)
    if (e) cudaEventDestroy(e);
  for (auto &e : ctx->wave_ev) cudaEventDestroy(e);
  if (ctx->staging_ev) cudaEventDestroy(ctx->staging_ev);
  if (ctx->staging) cudaFreeHost(ctx->staging);
  for (void *m : ctx->fit_mem) cudaFree(m);
  for (auto &x : ctx->aux)
    if (x) cudaStreamDestroy(x);
  for (auto &e : ctx->aux_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->ctr) cudaFree(ctx->ctr);
  delete ctx;
}

const char *pl_last_error(const pl_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

pl_status pl_set_tracing(pl_ctx *ctx, int on) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (on && !ctx->ev[0])
    for (auto &e : ctx->ev) PL_CUDA(cudaEventCreate(&e));
  ctx->tracing = on != 0;
  ctx->traced = false;
  return PL_OK;
}

pl_status pl_trace(pl_ctx *ctx, void *stream, pl_trace_info *out) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!out) return fail(ctx, PL_EINVAL, "pl_trace: null output");
  PL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  *out = pl_trace_info{};
  out->launches = ctx->launches;
  if (ctx->traced) {
    PL_CUDA(cudaEventElapsedTime(&out->law_ms, ctx->ev[0], ctx->ev[1]));
    PL_CUDA(cudaEventElapsedTime(&out->replicate_ms, ctx->ev[1], ctx->ev[2]));
    PL_CUDA(cudaEventElapsedTime(&out->select_ms, ctx->ev[2], ctx->ev[3]));
    PL_CUDA(cudaEventElapsedTime(&out->total_ms, ctx->ev[0], ctx->ev[3]));
    for (uint32_t w = 0; w < ctx->traced_waves && 4 * w + 3 < ctx->wave_ev.size(); ++w) {
      float a = 0.0f, b = 0.0f;
      PL_CUDA(cudaEventElapsedTime(&a, ctx->wave_ev[4 * w], ctx->wave_ev[4 * w + 1]));
      PL_CUDA(cudaEventElapsedTime(&b, ctx->wave_ev[4 * w + 2], ctx->wave_ev[4 * w + 3]));
      out->sample_ms += a;
      out->finish_ms += b;
    }
    out->waves = ctx->traced_waves;
    out->draws = ctx->traced_draws;
    out->sample_launches = ctx->traced_sample_launches;
  }
  return PL_OK;
}

pl_status pl_sync(pl_ctx *ctx, void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  return read_status(ctx, (cudaStream_t)stream);
}

pl_status pl_probe_rates(pl_ctx *ctx, void *stream, pl_probe_info *out) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!out) return fail(ctx, PL_EINVAL, "pl_probe_rates: null output");
  cudaStream_t st = (cudaStream_t)stream;
  // one block of kProbeBlock threads per SM
  const int grid = ctx->num_sms;
  const size_t words = (size_t)grid * kProbeBlock;
  if (pl_status s = ensure_ws(ctx, words * sizeof(uint32_t) + 256)) return s;
  uint32_t *o = reinterpret_cast<uint32_t *>(ctx->ws);
  long long *cyc = reinterpret_cast<long long *>(ctx->ws + ((words * sizeof(uint32_t) + 255) & ~(size_t)255));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PL_CUDA(cudaEventCreate(&e0));
  PL_CUDA(cudaEventCreate(&e1));
  // kind, loop iterations, operations per thread and iteration
  const struct { int kind, iters; double ops; } runs[4] = {
      {kProbeMulWide, 4096, (double)kProbeChains}, {kProbeLop3, 8192, (double)kProbeChains},
      {kProbeDfma, 256, (double)kProbeChains}, {kProbePhilox, 1024, 20.0}};
  double rate[4], mhz = 0.0, philox_ms = 0.0;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
    e = launch_probe(runs[k].kind, o, cyc, grid, runs[k].iters / 8, 1u, st);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch_probe(runs[k].kind, o, cyc, grid, runs[k].iters, 2u, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    long long c = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaMemcpy(&c, cyc, sizeof c, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) break;
    const double ops = (double)words * runs[k].iters * runs[k].ops;
    rate[k] = c > 0 ? ops / ((double)ctx->num_sms * (double)c) : 0.0;
    if (k == 0) mhz = ms > 0.0f ? (double)c / ((double)ms * 1e3) : 0.0;
    if (k == 3) philox_ms = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(ctx, PL_ECUDA, "pl_probe_rates: %s", cudaGetErrorString(e));
  out->sm_clock_mhz = mhz;
  out->mul_wide_per_sm_clk = rate[0];
  out->lop3_per_sm_clk = rate[1];
  out->dfma_per_sm_clk = rate[2];
  out->philox_words_per_s = philox_ms > 0.0 ? 4.0 * (double)words * runs[3].iters / (philox_ms * 1e-3) : 0.0;
  out->sms = ctx->num_sms;
  out->pad = 0;
  return PL_OK;
}

pl_status pl_counters(pl_ctx *ctx, void *stream, pl_counter_info *out) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!out) return fail(ctx, PL_EINVAL, "pl_counters: null output");
  PL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  Counters c{};
  PL_CUDA(cudaMemcpy(&c, ctx->ctr, sizeof c, cudaMemcpyDeviceToHost));
  out->newton_capped = c.newton_capped;
  out->tail_draws = c.tail_draws;
  out->global_sorts = c.global_sorts;
  out->fit_fallbacks = c.fit_fallbacks;
  out->resampled = c.resampled;
  return PL_OK;
}

pl_status pl_sample(pl_ctx *ctx, double alpha, uint64_t xmin, uint64_t seed, uint64_t cell_id,
                    uint32_t purpose, uint64_t rep0, int64_t nrep, int64_t n, uint64_t *out_dev,
                    void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!(alpha > 1.0) || alpha > 64.0 || xmin < 1 || xmin > (1ull << 40) || n < 1 || nrep < 1 ||
      cell_id >= (1ull << 32) || rep0 + (uint64_t)nrep > (1ull << 32) || n > (1ll << 34) || purpose >= kLowStream ||
      !out_dev)
    return fail(ctx, PL_EINVAL, "pl_sample: argument out of range");
  cudaStream_t st = (cudaStream_t)stream;
  LawPlan lp{alpha, xmin, table_length(alpha, xmin, (double)n * (double)nrep)};
  Carver cv;
  Law lh = carve_law(cv, lp);
  Law *ld = cv.take<Law>(1);
  if (pl_status s = ensure_ws(ctx, cv.off)) return s;
  cv.base = ctx->ws;
  cv.off = 0;
  lh = carve_law(cv, lp);
  ld = cv.take<Law>(1);
  PL_CUDA(cudaMemcpyAsync(ld, &lh, sizeof lh, cudaMemcpyHostToDevice, st));
  PL_CUDA(launch_law_setup(ld, 1, st));
  ctx->launches += kLawSetupLaunches + 1;  // the law set-up and the sampler
  PL_CUDA(launch_sample(ld, seed, (uint32_t)cell_id, purpose, (uint32_t)rep0, nrep, n, out_dev, ctx->ctr,
                        ctx->num_sms, st));
  return PL_OK;
}

// ---------------------------------------------------------------------------
// Truncated law on 1..K (Tables 2-6).
namespace {

struct TzPlan {
  std::vector<TzCell> cells;
  std::vector<TzLaw> laws;      // one per distinct (gamma, K)
  std::vector<TzTable> tables;  // one per distinct K
  std::vector<TzItem> items;
  int64_t total_R = 0;
};

struct TzBuffers {
  TzLaw *laws = nullptr;
  TzTable *tables = nullptr;
  TzCell *cells = nullptr;
  TzItem *items = nullptr;
  size_t host_bytes = 0;  // laws .. items, written from the host in one copy
};

pl_status tz_check_law(pl_ctx *ctx, double gamma, uint64_t K, bool any_sign = false) {
  if (any_sign ? !(gamma >= -64.0 && gamma <= 64.0) : !(gamma > 0.0 && gamma <= 64.0))
    return fail(ctx, PL_EINVAL, "truncated law: gamma must be in %s", any_sign ? "[-64, 64]" : "(0, 64]");
  if (K < 2 || K > kTzKMax) return fail(ctx, PL_EINVAL, "truncated law: K must be in [2, %u]", kTzKMax);
  return PL_OK;
}

uint32_t tz_law_index(TzPlan &tp, double gamma, uint32_t K, std::map<std::pair<double, uint32_t>, uint32_t> &ids) {
  auto key = std::make_pair(gamma, K);
  auto it = ids.find(key);
  if (it != ids.end()) return it->second;
  uint32_t tab = 0;
  while (tab < tp.tables.size() && tp.tables[tab].K != K) ++tab;
  if (tab == tp.tables.size()) {
    TzTable t{};
    t.K = K;
    t.lnK = std::log((double)K);
    tp.tables.push_back(t);
  }
  TzLaw l{};
  l.gamma = gamma;
  l.K = K;
  l.table = tab;
  tp.laws.push_back(l);
  ids[key] = (uint32_t)tp.laws.size() - 1;
  return (uint32_t)tp.laws.size() - 1;
}

// Cells, laws, tables and work items.  A work item is a block of kTzWarps
// warps, each taking a run of replicates of one cell; runs are sized by a
// replicate's cost (draws, support points and the fit) so that items of
// different cells cost about the same, and shrink when the call is too small
// to give every SM four items.  Costlier cells' items come first.
pl_status tz_plan(pl_ctx *ctx, const pl_tcell *in, int ncells, uint32_t purpose, TzPlan &tp, bool any_sign = false) {
  std::map<std::pair<double, uint32_t>, uint32_t> ids;
  std::vector<double> cost(ncells);
  double work = 0.0;
  for (int i = 0; i < ncells; ++i) {
    const pl_tcell &c = in[i];
    if (pl_status s = tz_check_law(ctx, c.gamma, c.K, any_sign)) return s;
    if (c.n < 1 || c.n > kTzNMax || c.replicates < 1 || c.replicates > (1ll << 32) || c.cell_id >= (1ull << 32))
      return fail(ctx, PL_EINVAL, "truncated cell %d: n must be in [1, %lld], replicates in [1, 2^32], cell_id < 2^32",
                  i, (long long)kTzNMax);
    TzCell tc{};
    tc.gamma = c.gamma;
    tc.n = c.n;
    tc.R = c.replicates;
    tc.out_off = tp.total_R;
    tc.cell_id = (uint32_t)c.cell_id;
    tc.law = tz_law_index(tp, c.gamma, (uint32_t)c.K, ids);
    tc.purpose = purpose;
    tp.cells.push_back(tc);
    tp.total_R += c.replicates;
    cost[i] = (double)c.n + 16.0 * (double)c.K + 1024.0;
    work += cost[i] * (double)c.replicates;
  }
  std::vector<int> order(ncells);
  for (int i = 0; i < ncells; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  int64_t cap = 64;  // replicates per warp, at most
  const int64_t want = 4 * (int64_t)ctx->num_sms;
  while (cap > 1 && work / (32768.0 * kTzWarps) < (double)want) cap >>= 1;
  for (int i : order) {
    const TzCell &c = tp.cells[i];
    const int64_t rpw = std::max<int64_t>(1, std::min<int64_t>(cap, (int64_t)(32768.0 / cost[i])));
    const int64_t per = rpw * kTzWarps;
    for (int64_t r0 = 0; r0 < c.R; r0 += per)
      tp.items.push_back({(uint32_t)i, (uint32_t)r0, (uint32_t)std::min<int64_t>(per, c.R - r0), 0u});
  }
  if (tp.items.size() > 0x7fffffffull) return fail(ctx, PL_ENOMEM, "truncated cutoffs: too many work items");
  return PL_OK;
}

void carve_tz(Carver &cv, TzPlan &tp, TzBuffers &b) {
  b.laws = cv.take<TzLaw>(tp.laws.size());
  b.tables = cv.take<TzTable>(tp.tables.size());
  b.cells = cv.take<TzCell>(tp.cells.size());
  b.items = cv.take<TzItem>(tp.items.size());
  b.host_bytes = (size_t)(reinterpret_cast<uint8_t *>(b.items + tp.items.size()) - reinterpret_cast<uint8_t *>(b.laws));
  for (TzLaw &l : tp.laws) {
    l.T = cv.take<uint64_t>(l.K + 1);
    l.guide = cv.take<uint16_t>(kTzGuide);
  }
  for (TzTable &t : tp.tables) {
    t.lnk = cv.take<double>(t.K + 1);
    t.lnk_hi = cv.take<float>(t.K + 1);
    t.lnk_lo = cv.take<float>(t.K + 1);
    t.lnq_hi = cv.take<float>(t.K + 1);
    t.lnq_lo = cv.take<float>(t.K + 1);
    t.node = cv.take<double>((size_t)kTzNodes * kTzNodeStride);
    t.E = cv.take<double>(kTzNodes);
  }
}

// Stage the host-written structures in one copy, then build the laws' and
// tables' contents on the device.
pl_status upload_tz(pl_ctx *ctx, const TzPlan &tp, const TzBuffers &b, cudaStream_t st) {
  uint8_t *img = nullptr;
  if (pl_status e = staging(ctx, b.host_bytes, &img)) return e;
  const uint8_t *base = reinterpret_cast<const uint8_t *>(b.laws);
  auto put = [&](const void *dev, const void *src, size_t bytes) {
    if (bytes) std::memcpy(img + (reinterpret_cast<const uint8_t *>(dev) - base), src, bytes);
  };
  put(b.laws, tp.laws.data(), sizeof(TzLaw) * tp.laws.size());
  put(b.tables, tp.tables.data(), sizeof(TzTable) * tp.tables.size());
  put(b.cells, tp.cells.data(), sizeof(TzCell) * tp.cells.size());
  put(b.items, tp.items.data(), sizeof(TzItem) * tp.items.size());
  PL_CUDA(cudaMemcpyAsync(b.laws, img, b.host_bytes, cudaMemcpyHostToDevice, st));
  PL_CUDA(cudaEventRecord(ctx->staging_ev, st));
  ctx->staged = true;
  PL_CUDA(launch_tz_setup(b.laws, (int)tp.laws.size(), b.tables, (int)tp.tables.size(), st));
  ctx->launches += 3;
  return PL_OK;
}

}  // namespace

pl_status pl_sample_truncated(pl_ctx *ctx, double gamma, uint64_t K, uint64_t seed, uint64_t cell_id,
                              uint32_t purpose, uint64_t rep0, int64_t nrep, int64_t n, uint64_t *out_dev,
                              void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (pl_status s = tz_check_law(ctx, gamma, K)) return s;
  if (n < 1 || nrep < 1 || cell_id >= (1ull << 32) || rep0 + (uint64_t)nrep > (1ull << 32) || n > (1ll << 34) ||
      purpose >= kLowStream || !out_dev)
    return fail(ctx, PL_EINVAL, "pl_sample_truncated: argument out of range");
  cudaStream_t st = (cudaStream_t)stream;
  TzLaw lh{};
  lh.gamma = gamma;
  lh.K = (uint32_t)K;
  auto lay = [&](Carver &cv, TzLaw *&ld) {
    ld = cv.take<TzLaw>(1);
    lh.T = cv.take<uint64_t>(K + 1);
    lh.guide = cv.take<uint16_t>(kTzGuide);
  };
  Carver cv;
  TzLaw *ld = nullptr;
  lay(cv, ld);
  if (pl_status s = ensure_ws(ctx, cv.off)) return s;
  cv.base = ctx->ws;
  cv.off = 0;
  lay(cv, ld);
  PL_CUDA(cudaMemcpyAsync(ld, &lh, sizeof lh, cudaMemcpyHostToDevice, st));
  PL_CUDA(launch_tz_setup(ld, 1, nullptr, 0, st));
  PL_CUDA(launch_tz_sample(ld, seed, (uint32_t)cell_id, purpose, (uint32_t)rep0, nrep, n, out_dev, st));
  ctx->launches += 2;
  return PL_OK;
}

namespace {

// Simulation of truncated cells (purpose 0: cutoff tables; 1: bespoke
// cutoffs of a data set) and the order statistics of each cell's D; with
// D_obs (device) also p = #{D >= D_obs} / R of the single cell.
pl_status run_tz_cutoffs(pl_ctx *ctx, const pl_tcell *cells, int ncells, uint32_t purpose, bool any_sign,
                         uint64_t seed, const double *q, int nq, bool f32, double *cutoffs, void *D_dev_opt,
                         double *gamma_hat_dev_opt, const double *D_obs_host, double *p_host, cudaStream_t st) {
  TzPlan tp;
  if (pl_status s = tz_plan(ctx, cells, ncells, purpose, tp, any_sign)) return s;
  const bool host_out = !is_device_ptr(cutoffs);
  const size_t dsz = f32 ? 4 : 8;
  TzBuffers b;
  void *D = nullptr;
  int64_t *off = nullptr, *Rs = nullptr, *rank = nullptr;
  double *cut = nullptr, *dobs = nullptr, *pd = nullptr;
  auto lay = [&](Carver &cv) {
    carve_tz(cv, tp, b);
    D = D_dev_opt ? D_dev_opt : (void *)cv.take<uint8_t>((size_t)tp.total_R * dsz);
    off = cv.take<int64_t>(ncells);
    Rs = cv.take<int64_t>(ncells);
    rank = cv.take<int64_t>((size_t)ncells * nq);
    cut = host_out ? cv.take<double>((size_t)ncells * nq) : cutoffs;
    dobs = cv.take<double>(1);
    pd = cv.take<double>(1);
  };
  Carver cv;
  lay(cv);
  if (pl_status s = ensure_ws(ctx, cv.off)) return s;
  cv.base = ctx->ws;
  cv.off = 0;
  lay(cv);
  if (pl_status s = mark(ctx, 0, st)) return s;
  if (pl_status s = upload_tz(ctx, tp, b, st)) return s;
  std::vector<int64_t> h_off(ncells), h_R(ncells), h_rank((size_t)ncells * nq);
  for (int c = 0; c < ncells; ++c) {
    h_off[c] = tp.cells[c].out_off;
    h_R[c] = tp.cells[c].R;
    for (int j = 0; j < nq; ++j) {
      int64_t i = (int64_t)std::floor((double)h_R[c] * q[j]);
      h_rank[(size_t)c * nq + j] = std::min(std::max<int64_t>(i, 0), h_R[c] - 1);
    }
  }
  PL_CUDA(cudaMemcpyAsync(off, h_off.data(), sizeof(int64_t) * ncells, cudaMemcpyHostToDevice, st));
  PL_CUDA(cudaMemcpyAsync(Rs, h_R.data(), sizeof(int64_t) * ncells, cudaMemcpyHostToDevice, st));
  PL_CUDA(cudaMemcpyAsync(rank, h_rank.data(), sizeof(int64_t) * h_rank.size(), cudaMemcpyHostToDevice, st));
  if (D_obs_host) PL_CUDA(cudaMemcpyAsync(dobs, D_obs_host, sizeof(double), cudaMemcpyHostToDevice, st));
  if (pl_status s = mark(ctx, 1, st)) return s;
  TzLaunch tl{};
  tl.cells = b.cells;
  tl.laws = b.laws;
  tl.tables = b.tables;
  tl.items = b.items;
  tl.nitems = (uint32_t)tp.items.size();
  tl.rk = round_keys(seed);
  tl.D_out = D;
  tl.A_out = gamma_hat_dev_opt;
  tl.ctr = ctx->ctr;
  PL_CUDA(launch_tz_replicates(tl, f32, st));
  ctx->launches += 1;
  if (ctx->tracing) {
    ctx->traced_waves = 0;
    ctx->traced_sample_launches = 0;
    ctx->traced_draws = 0;
    for (const TzCell &c : tp.cells) ctx->traced_draws += (uint64_t)c.n * (uint64_t)c.R;
  }
  if (pl_status s = mark(ctx, 2, st)) return s;
  PL_CUDA(launch_select(D, f32, off, Rs, rank, ncells, nq, cut, st));
  ctx->launches += 1;
  if (D_obs_host) {
    PL_CUDA(launch_count_ge(D, f32, tp.total_R, dobs, pd, st));
    ctx->launches += 1;
  }
  if (pl_status s = mark(ctx, 3, st)) return s;
  if (host_out) PL_CUDA(cudaMemcpyAsync(cutoffs, cut, sizeof(double) * ncells * nq, cudaMemcpyDeviceToHost, st));
  if (p_host) PL_CUDA(cudaMemcpyAsync(p_host, pd, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (host_out || p_host) return read_status(ctx, st);
  return PL_OK;
}

// Fit and/or D of one truncated data set: out_host = (gamma, D, zeta_K(gamma)).
pl_status run_tz_dataset(pl_ctx *ctx, const int32_t *x, int64_t n, uint64_t K, bool fit, double gamma, bool f32,
                         double out_host[3], cudaStream_t st) {
  if (!x || n < 1 || n > INT32_MAX) return fail(ctx, PL_EINVAL, "truncated data set: bad arguments");
  if (pl_status s = tz_check_law(ctx, fit ? 1.0 : gamma, K, true)) return s;
  TzTable th{};
  th.K = (uint32_t)K;
  th.lnK = std::log((double)K);
  auto lay = [&](Carver &cv, TzTable *&td, double *&out) {
    td = cv.take<TzTable>(1);
    th.lnk = cv.take<double>(K + 1);
    th.lnk_hi = cv.take<float>(K + 1);
    th.lnk_lo = cv.take<float>(K + 1);
    th.lnq_hi = cv.take<float>(K + 1);
    th.lnq_lo = cv.take<float>(K + 1);
    th.node = cv.take<double>((size_t)kTzNodes * kTzNodeStride);
    th.E = cv.take<double>(kTzNodes);
    out = cv.take<double>(4);
  };
  Carver cv;
  TzTable *td = nullptr;
  double *out = nullptr;
  lay(cv, td, out);
  if (pl_status s = ensure_ws(ctx, cv.off)) return s;
  cv.base = ctx->ws;
  cv.off = 0;
  lay(cv, td, out);
  PL_CUDA(cudaMemcpyAsync(td, &th, sizeof th, cudaMemcpyHostToDevice, st));
  PL_CUDA(launch_tz_setup(nullptr, 0, td, 1, st));
  PL_CUDA(launch_tz_dataset(x, n, td, fit, gamma, f32, out, ctx->ctr, st));
  ctx->launches += 4;
  PL_CUDA(cudaMemcpyAsync(out_host, out, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  return read_status(ctx, st);
}

}  // namespace

pl_status pl_ks_cutoffs_truncated(pl_ctx *ctx, const pl_tcell *cells, int ncells, uint64_t seed, const double *q,
                                  int nq, pl_precision prec, double *cutoffs, void *D_dev_opt,
                                  double *gamma_hat_dev_opt, void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!cells || ncells < 1 || !q || nq < 1 || !cutoffs)
    return fail(ctx, PL_EINVAL, "pl_ks_cutoffs_truncated: bad arguments");
  if (prec != PL_FP64 && prec != PL_FP32_BULK) return fail(ctx, PL_EINVAL, "unknown precision form");
  for (int j = 0; j < nq; ++j)
    if (!(q[j] > 0.0 && q[j] < 1.0)) return fail(ctx, PL_EINVAL, "quantile %d outside (0, 1)", j);
  return run_tz_cutoffs(ctx, cells, ncells, 0u, false, seed, q, nq, prec == PL_FP32_BULK, cutoffs, D_dev_opt,
                        gamma_hat_dev_opt, nullptr, nullptr, (cudaStream_t)stream);
}

pl_status pl_fit_ks_truncated(pl_ctx *ctx, const int32_t *x_dev, int64_t n, uint64_t K, double gamma,
                              pl_precision prec, double *gamma_host, double *D_host, void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!gamma_host || !D_host) return fail(ctx, PL_EINVAL, "pl_fit_ks_truncated: null output");
  if (prec != PL_FP64 && prec != PL_FP32_BULK) return fail(ctx, PL_EINVAL, "unknown precision form");
  const bool fit = std::isnan(gamma);
  double o[3];
  if (pl_status s = run_tz_dataset(ctx, x_dev, n, K, fit, fit ? 0.0 : gamma, prec == PL_FP32_BULK, o,
                                   (cudaStream_t)stream))
    return s;
  *gamma_host = o[0];
  *D_host = o[1];
  return PL_OK;
}

pl_status pl_bespoke_cutoffs_truncated(pl_ctx *ctx, const int32_t *x_dev, int64_t n, uint64_t K, int64_t R,
                                       uint64_t seed, uint64_t request_id, const double *q, int nq,
                                       pl_precision prec, double *gamma_hat, double *D, double *p,
                                       double *cutoffs_host, void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (R < 1 || R > (1ll << 32) || request_id >= (1ull << 32) || !gamma_hat || !D || !p || !q || nq < 1 ||
      !cutoffs_host || n > kTzNMax)
    return fail(ctx, PL_EINVAL, "pl_bespoke_cutoffs_truncated: bad arguments");
  if (prec != PL_FP64 && prec != PL_FP32_BULK) return fail(ctx, PL_EINVAL, "unknown precision form");
  for (int j = 0; j < nq; ++j)
    if (!(q[j] > 0.0 && q[j] < 1.0)) return fail(ctx, PL_EINVAL, "quantile %d outside (0, 1)", j);
  cudaStream_t st = (cudaStream_t)stream;
  const bool f32 = prec == PL_FP32_BULK;
  double obs[3];
  if (pl_status s = run_tz_dataset(ctx, x_dev, n, K, true, 0.0, f32, obs, st)) return s;
  pl_tcell cell{obs[0], K, n, R, request_id};
  double ph = 0.0;
  if (pl_status s = run_tz_cutoffs(ctx, &cell, 1, 1u, true, seed, q, nq, f32, cutoffs_host, nullptr, nullptr,
                                   &obs[1], &ph, st))
    return s;
  *gamma_hat = obs[0];
  *D = obs[1];
  *p = ph;
  return PL_OK;
}

// ---------------------------------------------------------------------------
namespace {
pl_status run_dataset(pl_ctx *ctx, const int32_t *x, int64_t n, uint64_t xmin, bool fit, double alpha,
                      pl_precision prec, double out_host[3], cudaStream_t st, Carver *keep = nullptr) {
  if (!x || n < 1 || n > INT32_MAX || xmin < 1 || xmin > (1ull << 31))
    return fail(ctx, PL_EINVAL, "data set: bad arguments");
  if (!fit && (!(alpha > 1.0) || alpha > 64.0)) return fail(ctx, PL_EINVAL, "alpha must be in (1, 64]");
  LawPlan lp{fit ? 2.0 : alpha, xmin, kL1};
  const uint64_t cap = next_pow2((uint64_t)n);
  auto lay = [&](Carver &cv, Law &lh, Law *&ld, uint64_t *&spill, uint64_t *&pairs, double *&out) {
    lh = carve_law(cv, lp);
    ld = cv.take<Law>(1);
    spill = cv.take<uint64_t>(cap);
    pairs = cv.take<uint64_t>(2 * (size_t)n);
    out = cv.take<double>(4);
  };
  Carver cv;
  Law lh;
  Law *ld;
  uint64_t *spill, *pairs;
  double *out;
  lay(cv, lh, ld, spill, pairs, out);
  if (pl_status s = ensure_ws(ctx, cv.off)) return s;
  cv.base = ctx->ws;
  cv.off = 0;
  lay(cv, lh, ld, spill, pairs, out);
  PL_CUDA(cudaMemcpyAsync(ld, &lh, sizeof lh, cudaMemcpyHostToDevice, st));
  PL_CUDA(launch_law_setup(ld, 1, st));
  ctx->launches += kLawSetupLaunches + 1;  // the law set-up and the data-set kernel
  PL_CUDA(launch_dataset(x, n, xmin, fit, alpha, ld, cell_const(xmin), prec == PL_FP32_BULK, spill, pairs, out,
                         ctx->ctr, st));
  PL_CUDA(cudaMemcpyAsync(out_host, out, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (keep) *keep = cv;
  return read_status(ctx, st);
}
}  // namespace

pl_status pl_fit_mle(pl_ctx *ctx, const int32_t *x_dev, int64_t n, uint64_t xmin, double *alpha_hat_host,
                     void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!alpha_hat_host) return fail(ctx, PL_EINVAL, "pl_fit_mle: null output");
  double o[3];
  if (pl_status s = run_dataset(ctx, x_dev, n, xmin, true, 0.0, PL_FP64, o, (cudaStream_t)stream)) return s;
  *alpha_hat_host = o[0];
  return PL_OK;
}

pl_status pl_ks_stat(pl_ctx *ctx, const int32_t *x_dev, int64_t n, uint64_t xmin, double alpha,
                     pl_precision prec, double *D_host, void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!D_host) return fail(ctx, PL_EINVAL, "pl_ks_stat: null output");
  double o[3];
  if (pl_status s = run_dataset(ctx, x_dev, n, xmin, false, alpha, prec, o, (cudaStream_t)stream)) return s;
  *D_host = o[1];
  return PL_OK;
}

pl_status pl_ks_cutoffs(pl_ctx *ctx, const pl_cell *cells, int ncells, uint64_t seed, const double *q, int nq,
                        pl_precision prec, double *cutoffs, void *D_dev_opt, double *alpha_hat_dev_opt,
                        void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!cells || ncells < 1 || !q || nq < 1 || !cutoffs) return fail(ctx, PL_EINVAL, "pl_ks_cutoffs: bad arguments");
  if (prec != PL_FP64 && prec != PL_FP32_BULK) return fail(ctx, PL_EINVAL, "unknown precision form");
  for (int j = 0; j < nq; ++j)
    if (!(q[j] > 0.0 && q[j] < 1.0)) return fail(ctx, PL_EINVAL, "quantile %d outside (0, 1)", j);
  cudaStream_t st = (cudaStream_t)stream;
  const bool f32 = prec == PL_FP32_BULK;
  SimPlan sp;
  if (pl_status s = plan_cells(ctx, cells, ncells, 0u, sp)) return s;
  const bool host_out = !is_device_ptr(cutoffs);
  const size_t dsz = f32 ? 4 : 8;
  const int blocks = sim_blocks(ctx, f32), sblocks = sample_blocks(ctx),
            bsblocks = ctx->num_sms * std::max(1, ctx->block_sampler_per_sm);
  auto lay = [&](Carver &cv, SimBuffers &b, void *&D, int64_t *&off, int64_t *&Rs, int64_t *&rank, double *&cut) {
    carve_sim(cv, sp, blocks, sblocks, b, ctx->dbg_arena, bsblocks);
    D = D_dev_opt ? D_dev_opt : (void *)cv.take<uint8_t>((size_t)sp.total_R * dsz);
    off = cv.take<int64_t>(ncells);
    Rs = cv.take<int64_t>(ncells);
    rank = cv.take<int64_t>((size_t)ncells * nq);
    cut = host_out ? cv.take<double>((size_t)ncells * nq) : cutoffs;
  };
  Carver cv;
  SimBuffers b;
  void *D;
  int64_t *off, *Rs, *rank;
  double *cut;
  lay(cv, b, D, off, Rs, rank, cut);
  if (pl_status s = ensure_ws(ctx, cv.off)) return s;
  cv.base = ctx->ws;
  cv.off = 0;
  lay(cv, b, D, off, Rs, rank, cut);
  if (pl_status s = mark(ctx, 0, st)) return s;
  if (pl_status s = upload_sim(ctx, sp, b, st)) return s;
  std::vector<int64_t> h_off(ncells), h_R(ncells), h_rank((size_t)ncells * nq);
  for (int c = 0; c < ncells; ++c) {
    h_off[c] = sp.cells[c].out_off;
    h_R[c] = sp.cells[c].R;
    for (int j = 0; j < nq; ++j) {
      int64_t i = (int64_t)std::floor((double)h_R[c] * q[j]);
      h_rank[(size_t)c * nq + j] = std::min(std::max<int64_t>(i, 0), h_R[c] - 1);
    }
  }
  PL_CUDA(cudaMemcpyAsync(off, h_off.data(), sizeof(int64_t) * ncells, cudaMemcpyHostToDevice, st));
  PL_CUDA(cudaMemcpyAsync(Rs, h_R.data(), sizeof(int64_t) * ncells, cudaMemcpyHostToDevice, st));
  PL_CUDA(cudaMemcpyAsync(rank, h_rank.data(), sizeof(int64_t) * h_rank.size(), cudaMemcpyHostToDevice, st));
  if (pl_status s = mark(ctx, 1, st)) return s;
  if (pl_status s = run_sim(ctx, sp, b, seed, f32, D, alpha_hat_dev_opt, st)) return s;
  if (pl_status s = mark(ctx, 2, st)) return s;
  PL_CUDA(launch_select(D, f32, off, Rs, rank, ncells, nq, cut, st));
  ctx->launches += 1;
  if (pl_status s = mark(ctx, 3, st)) return s;
  if (host_out) {
    PL_CUDA(cudaMemcpyAsync(cutoffs, cut, sizeof(double) * ncells * nq, cudaMemcpyDeviceToHost, st));
    return read_status(ctx, st);
  }
  return PL_OK;
}

}  // extern "C"

extern "C" {

pl_status pl_ks_cutoffs_multinomial(pl_ctx *ctx, const pl_cell *cells, int ncells, uint64_t seed, const double *q,
                                    int nq, pl_precision prec, double *cutoffs, void *D_dev_opt,
                                    double *alpha_hat_dev_opt, void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!cells || ncells < 1 || !q || nq < 1 || !cutoffs)
    return fail(ctx, PL_EINVAL, "pl_ks_cutoffs_multinomial: bad arguments");
  if (prec != PL_FP64 && prec != PL_FP32_BULK) return fail(ctx, PL_EINVAL, "unknown precision form");
  for (int j = 0; j < nq; ++j)
    if (!(q[j] > 0.0 && q[j] < 1.0)) return fail(ctx, PL_EINVAL, "quantile %d outside (0, 1)", j);
  cudaStream_t st = (cudaStream_t)stream;
  const bool f32 = prec == PL_FP32_BULK;
  SimPlan sp;
  if (pl_status s = plan_cells(ctx, cells, ncells, kPurposeMultinomial, sp, true)) return s;
  const bool host_out = !is_device_ptr(cutoffs);
  const size_t dsz = f32 ? 4 : 8;
  const int blocks = sim_blocks(ctx, f32), sblocks = sample_blocks(ctx),
            bsblocks = ctx->num_sms * std::max(1, ctx->block_sampler_per_sm);
  auto lay = [&](Carver &cv, SimBuffers &b, void *&D, int64_t *&off, int64_t *&Rs, int64_t *&rank, double *&cut) {
    carve_sim(cv, sp, blocks, sblocks, b, ctx->dbg_arena, bsblocks);
    D = D_dev_opt ? D_dev_opt : (void *)cv.take<uint8_t>((size_t)sp.total_R * dsz);
    off = cv.take<int64_t>(ncells);
    Rs = cv.take<int64_t>(ncells);
    rank = cv.take<int64_t>((size_t)ncells * nq);
    cut = host_out ? cv.take<double>((size_t)ncells * nq) : cutoffs;
  };
  Carver cv;
  SimBuffers b;
  void *D;
  int64_t *off, *Rs, *rank;
  double *cut;
  lay(cv, b, D, off, Rs, rank, cut);
  if (pl_status s = ensure_ws(ctx, cv.off)) return s;
  cv.base = ctx->ws;
  cv.off = 0;
  lay(cv, b, D, off, Rs, rank, cut);
  if (pl_status s = mark(ctx, 0, st)) return s;
  if (pl_status s = upload_sim(ctx, sp, b, st)) return s;
  std::vector<int64_t> h_off(ncells), h_R(ncells), h_rank((size_t)ncells * nq);
  for (int c = 0; c < ncells; ++c) {
    h_off[c] = sp.cells[c].out_off;
    h_R[c] = sp.cells[c].R;
    for (int j = 0; j < nq; ++j) {
      int64_t i = (int64_t)std::floor((double)h_R[c] * q[j]);
      h_rank[(size_t)c * nq + j] = std::min(std::max<int64_t>(i, 0), h_R[c] - 1);
    }
  }
  PL_CUDA(cudaMemcpyAsync(off, h_off.data(), sizeof(int64_t) * ncells, cudaMemcpyHostToDevice, st));
  PL_CUDA(cudaMemcpyAsync(Rs, h_R.data(), sizeof(int64_t) * ncells, cudaMemcpyHostToDevice, st));
  PL_CUDA(cudaMemcpyAsync(rank, h_rank.data(), sizeof(int64_t) * h_rank.size(), cudaMemcpyHostToDevice, st));
  if (pl_status s = mark(ctx, 1, st)) return s;
  if (pl_status s = run_sim_mn(ctx, sp, b, seed, f32, D, alpha_hat_dev_opt, st)) return s;
  if (pl_status s = mark(ctx, 2, st)) return s;
  PL_CUDA(launch_select(D, f32, off, Rs, rank, ncells, nq, cut, st));
  ctx->launches += 1;
  if (pl_status s = mark(ctx, 3, st)) return s;
  if (host_out) {
    PL_CUDA(cudaMemcpyAsync(cutoffs, cut, sizeof(double) * ncells * nq, cudaMemcpyDeviceToHost, st));
    return read_status(ctx, st);
  }
  return PL_OK;
}

}  // extern "C"

struct pl_plan {
  pl_ctx *ctx = nullptr;
  SimPlan sp;
  SimBuffers b;
  uint8_t *mem = nullptr;
  void *D = nullptr;
  int64_t *off = nullptr, *Rs = nullptr, *rank = nullptr;
  int ncells = 0, nq = 0;
  bool f32 = false;
};

extern "C" {

pl_status pl_set_split(pl_ctx *ctx, int64_t split) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (split < 1 || split > kWarpNMax) return fail(ctx, PL_EINVAL, "split must be in [1, %lld]", (long long)kWarpNMax);
  ctx->warp_split = split;
  return PL_OK;
}

pl_status pl_autotune(pl_ctx *ctx, void *stream, int64_t *split_out) {
  if (pl_status s = check_ctx(ctx)) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t saved = ctx->warp_split;
  const bool saved_tracing = ctx->tracing;
  if (pl_status s = pl_set_tracing(ctx, 1)) return s;
  const double q = 0.9;
  double cut = 0.0;
  int64_t best = 256;  // the warp form is kept below the smallest bucket tried
  pl_status st_all = PL_OK;
  for (int64_t n = 512; n <= 65536; n *= 2) {
    const int64_t nn = std::min(n, kWarpNMax);
    pl_cell cell{2.0, 1, nn, 65536, 0};
    float t[2] = {0.0f, 0.0f};
    for (int form = 0; form < 2 && !st_all; ++form) {  // 0: warp, 1: block
      ctx->warp_split = form == 0 ? kWarpNMax : 1;
      for (int rep = 0; rep < 2 && !st_all; ++rep) {  // second run timed
        st_all = pl_ks_cutoffs(ctx, &cell, 1, 1, &q, 1, PL_FP32_BULK, &cut, nullptr, nullptr, stream);
        if (!st_all) {
          pl_trace_info ti;
          st_all = pl_trace(ctx, stream, &ti);
          t[form] = ti.replicate_ms;
        }
      }
    }
    if (st_all) break;
    if (t[0] <= t[1]) best = nn;
    else break;
  }
  ctx->warp_split = st_all ? saved : best;
  pl_set_tracing(ctx, saved_tracing ? 1 : 0);
  PL_CUDA(cudaStreamSynchronize(st));
  if (split_out) *split_out = ctx->warp_split;
  return st_all;
}

pl_status pl_autotune_cells(pl_ctx *ctx, const pl_cell *cells, int ncells, pl_precision prec,
                            int64_t sample_replicates, pl_tuning *out, void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!cells || ncells < 1 || sample_replicates < 1 || (prec != PL_FP64 && prec != PL_FP32_BULK))
    return fail(ctx, PL_EINVAL, "pl_autotune_cells: bad arguments");
  // the cell mix with at most sample_replicates replicates per cell
  std::vector<pl_cell> sub(cells, cells + ncells);
  for (pl_cell &c : sub) c.replicates = std::min<int64_t>(c.replicates, sample_replicates);
  const int64_t saved_split = ctx->warp_split;
  const int saved_item = ctx->item_reps, saved_shift = ctx->hist_shift;
  const bool saved_tracing = ctx->tracing;
  if (pl_status s = pl_set_tracing(ctx, 1)) return s;
  const double q = 0.9;
  std::vector<double> cut(ncells);
  // time of one call at the context's current settings (median of three, after one untimed)
  auto trial = [&](double *ms) -> pl_status {
    float t[3];
    for (int rep = 0; rep < 4; ++rep) {
      if (pl_status s = pl_ks_cutoffs(ctx, sub.data(), ncells, 1, &q, 1, prec, cut.data(), nullptr, nullptr, stream))
        return s;
      pl_trace_info ti;
      if (pl_status s = pl_trace(ctx, stream, &ti)) return s;
      if (rep) t[rep - 1] = ti.total_ms;
    }
    std::sort(t, t + 3);
    *ms = (double)t[1];
    return PL_OK;
  };
  pl_status st_all = PL_OK;
  double best = 0.0;
  st_all = trial(&best);
  // coordinate descent: warp/block split, then replicates per work item, then dense bins
  const int64_t splits[] = {256, 1024, 4096, 16384, kWarpNMax};
  int64_t best_split = ctx->warp_split;
  for (int64_t sp : splits) {
    if (st_all) break;
    ctx->warp_split = sp;
    double t;
    st_all = trial(&t);
    if (!st_all && t < best) best = t, best_split = sp;
  }
  ctx->warp_split = best_split;
  // the work-item size is tuned only on the whole workload: on a replicate
  // sample the plan's own sizing (items small enough to fill the GPU) is what
  // a sample of a larger workload would measure, not the full-size optimum
  bool whole = true;
  for (int c = 0; c < ncells; ++c) whole = whole && cells[c].replicates <= sample_replicates;
  const int items[] = {32, 64, 128, 256};
  int best_item = ctx->item_reps;
  for (int it : items) {
    if (st_all || !whole) break;
    ctx->item_reps = it;
    double t;
    st_all = trial(&t);
    if (!st_all && t < best) best = t, best_item = it;
  }
  ctx->item_reps = best_item;
  int best_shift = ctx->hist_shift;
  for (int sh = -1; sh <= 1; ++sh) {
    if (st_all) break;
    if (sh == best_shift) continue;
    ctx->hist_shift = sh;
    double t;
    st_all = trial(&t);
    if (!st_all && t < best) best = t, best_shift = sh;
  }
  ctx->hist_shift = best_shift;
  if (st_all) {
    ctx->warp_split = saved_split;
    ctx->item_reps = saved_item;
    ctx->hist_shift = saved_shift;
  }
  pl_set_tracing(ctx, saved_tracing ? 1 : 0);
  PL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (out && !st_all) {
    out->split = ctx->warp_split;
    out->item_reps = ctx->item_reps;
    out->hist_shift = ctx->hist_shift;
    out->best_ms = best;
  }
  return st_all;
}

pl_status pl_set_tuning(pl_ctx *ctx, const pl_tuning *t) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!t || t->split < 1 || t->split > kWarpNMax || (t->item_reps != 0 && (t->item_reps < 1 || t->item_reps > kItemReps)) ||
      t->hist_shift < -5 || t->hist_shift > 5)
    return fail(ctx, PL_EINVAL, "pl_set_tuning: setting out of range");
  ctx->warp_split = t->split;
  ctx->item_reps = t->item_reps;
  ctx->hist_shift = t->hist_shift;
  return PL_OK;
}

pl_status pl_plan_cutoffs(pl_ctx *ctx, const pl_cell *cells, int ncells, const double *q, int nq,
                          pl_precision prec, pl_plan **out, void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!out || !cells || ncells < 1 || !q || nq < 1) return fail(ctx, PL_EINVAL, "pl_plan_cutoffs: bad arguments");
  *out = nullptr;
  if (prec != PL_FP64 && prec != PL_FP32_BULK) return fail(ctx, PL_EINVAL, "unknown precision form");
  for (int j = 0; j < nq; ++j)
    if (!(q[j] > 0.0 && q[j] < 1.0)) return fail(ctx, PL_EINVAL, "quantile %d outside (0, 1)", j);
  cudaStream_t st = (cudaStream_t)stream;
  pl_plan *pp = new pl_plan();
  pp->ctx = ctx;
  pp->ncells = ncells;
  pp->nq = nq;
  pp->f32 = prec == PL_FP32_BULK;
  if (pl_status s = plan_cells(ctx, cells, ncells, 0u, pp->sp)) {
    delete pp;
    return s;
  }
  const SimPlan &sp = pp->sp;
  const int blocks = sim_blocks(ctx, pp->f32), sblocks = sample_blocks(ctx),
            bsblocks = ctx->num_sms * std::max(1, ctx->block_sampler_per_sm);
  auto lay = [&](Carver &cv) {
    carve_sim(cv, sp, blocks, sblocks, pp->b, ctx->dbg_arena, bsblocks);
    pp->D = cv.take<uint8_t>((size_t)sp.total_R * (pp->f32 ? 4 : 8));
    pp->off = cv.take<int64_t>(ncells);
    pp->Rs = cv.take<int64_t>(ncells);
    pp->rank = cv.take<int64_t>((size_t)ncells * nq);
  };
  Carver cv;
  lay(cv);
  if (cv.off > ctx->budget) {
    delete pp;
    return fail(ctx, PL_ENOMEM, "plan of %zu bytes exceeds the budget of %zu", cv.off, ctx->budget);
  }
  if (cudaMalloc(&pp->mem, cv.off) != cudaSuccess) {
    cudaGetLastError();
    delete pp;
    return fail(ctx, PL_ENOMEM, "plan allocation of %zu bytes failed", cv.off);
  }
  cv.base = pp->mem;
  cv.off = 0;
  lay(cv);
  pl_status s = upload_sim(ctx, sp, pp->b, st);
  std::vector<int64_t> h_off(ncells), h_R(ncells), h_rank((size_t)ncells * nq);
  for (int c = 0; c < ncells; ++c) {
    h_off[c] = sp.cells[c].out_off;
    h_R[c] = sp.cells[c].R;
    for (int j = 0; j < nq; ++j) {
      int64_t i = (int64_t)std::floor((double)h_R[c] * q[j]);
      h_rank[(size_t)c * nq + j] = std::min(std::max<int64_t>(i, 0), h_R[c] - 1);
    }
  }
  if (!s && (cudaMemcpyAsync(pp->off, h_off.data(), sizeof(int64_t) * ncells, cudaMemcpyHostToDevice, st) ||
             cudaMemcpyAsync(pp->Rs, h_R.data(), sizeof(int64_t) * ncells, cudaMemcpyHostToDevice, st) ||
             cudaMemcpyAsync(pp->rank, h_rank.data(), sizeof(int64_t) * h_rank.size(), cudaMemcpyHostToDevice,
                             st)))
    s = fail(ctx, PL_ECUDA, "plan upload failed");
  if (!s) s = read_status(ctx, st);
  if (s) {
    cudaFree(pp->mem);
    delete pp;
    return s;
  }
  *out = pp;
  return PL_OK;
}

pl_status pl_plan_run(pl_plan *plan, uint64_t seed, double *cutoffs_dev, void *D_dev_opt,
                      double *alpha_hat_dev_opt, void *stream) {
  if (!plan) return PL_EINVAL;
  pl_ctx *ctx = plan->ctx;
  if (pl_status s = check_ctx(ctx)) return s;
  if (!cutoffs_dev) return fail(ctx, PL_EINVAL, "pl_plan_run: null cutoffs");
  cudaStream_t st = (cudaStream_t)stream;
  void *D = D_dev_opt ? D_dev_opt : plan->D;
  if (pl_status s = run_sim(ctx, plan->sp, plan->b, seed, plan->f32, D, alpha_hat_dev_opt, st, false)) return s;
  PL_CUDA(launch_select(D, plan->f32, plan->off, plan->Rs, plan->rank, plan->ncells, plan->nq, cutoffs_dev, st));
  ctx->launches += 1;
  return PL_OK;
}

void pl_plan_destroy(pl_plan *plan) {
  if (!plan) return;
  cudaSetDevice(plan->ctx->device);
  cudaDeviceSynchronize();
  cudaFree(plan->mem);
  delete plan;
}

namespace {
// The parametric bootstrap of one data set: fit (Eq. 2) and D (Eq. 3), then B
// data sets of the same n at alpha-hat (purpose 1, cell = request id), each
// refitted; p = #{D_b >= D} / B and, for nq > 0, the order statistics of the
// D_b at the quantiles q (the bespoke cutoffs).
pl_status run_bootstrap(pl_ctx *ctx, const int32_t *x_dev, int64_t n, uint64_t xmin, int64_t B, uint64_t seed,
                        uint64_t request_id, pl_precision prec, const double *q, int nq, double *alpha_hat,
                        double *D, double *p, double *cut_host, cudaStream_t st) {
  if (B < 1 || B > (1ll << 31) || request_id >= (1ull << 32) || !alpha_hat || !D || !p || nq < 0 ||
      (nq > 0 && (!q || !cut_host)))
    return fail(ctx, PL_EINVAL, "bootstrap: bad arguments");
  if (prec != PL_FP64 && prec != PL_FP32_BULK) return fail(ctx, PL_EINVAL, "unknown precision form");
  for (int j = 0; j < nq; ++j)
    if (!(q[j] > 0.0 && q[j] < 1.0)) return fail(ctx, PL_EINVAL, "quantile %d outside (0, 1)", j);
  const bool f32 = prec == PL_FP32_BULK;
  double obs[3];
  if (pl_status s = run_dataset(ctx, x_dev, n, xmin, true, 0.0, prec, obs, st)) return s;
  pl_cell cell{obs[0], xmin, n, B, request_id};
  SimPlan sp;
  if (pl_status s = plan_cells(ctx, &cell, 1, 1u, sp)) return s;
  const int blocks = sim_blocks(ctx, f32), sblocks = sample_blocks(ctx),
            bsblocks = ctx->num_sms * std::max(1, ctx->block_sampler_per_sm);
  const int nsel = std::max(nq, 1);
  auto lay = [&](Carver &cv, SimBuffers &b, void *&Db, double *&dobs, double *&pd, int64_t *&sel, double *&cut) {
    carve_sim(cv, sp, blocks, sblocks, b, ctx->dbg_arena, bsblocks);
    Db = cv.take<uint8_t>((size_t)B * (f32 ? 4 : 8));
    dobs = cv.take<double>(1);
    pd = cv.take<double>(1);
    sel = cv.take<int64_t>(2 + (size_t)nsel);  // offset 0, R, then the ranks
    cut = cv.take<double>(nsel);
  };
  Carver cv;
  SimBuffers b;
  void *Db;
  double *dobs, *pd, *cut;
  int64_t *sel;
  lay(cv, b, Db, dobs, pd, sel, cut);
  if (pl_status s = ensure_ws(ctx, cv.off)) return s;
  cv.base = ctx->ws;
  cv.off = 0;
  lay(cv, b, Db, dobs, pd, sel, cut);
  PL_CUDA(cudaMemcpyAsync(dobs, &obs[1], sizeof(double), cudaMemcpyHostToDevice, st));
  std::vector<int64_t> h_sel(2 + (size_t)nsel, 0);
  h_sel[1] = B;
  for (int j = 0; j < nq; ++j)
    h_sel[2 + j] = std::min(std::max<int64_t>((int64_t)std::floor((double)B * q[j]), 0), B - 1);
  if (nq > 0) PL_CUDA(cudaMemcpyAsync(sel, h_sel.data(), sizeof(int64_t) * h_sel.size(), cudaMemcpyHostToDevice, st));
  if (pl_status s = mark(ctx, 0, st)) return s;
  if (pl_status s = upload_sim(ctx, sp, b, st)) return s;
  if (pl_status s = mark(ctx, 1, st)) return s;
  if (pl_status s = run_sim(ctx, sp, b, seed, f32, Db, nullptr, st)) return s;
  if (pl_status s = mark(ctx, 2, st)) return s;
  PL_CUDA(launch_count_ge(Db, f32, B, dobs, pd, st));
  ctx->launches += 1;
  if (nq > 0) {
    PL_CUDA(launch_select(Db, f32, sel, sel + 1, sel + 2, 1, nq, cut, st));
    ctx->launches += 1;
  }
  if (pl_status s = mark(ctx, 3, st)) return s;
  double ph = 0.0;
  PL_CUDA(cudaMemcpyAsync(&ph, pd, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (nq > 0) PL_CUDA(cudaMemcpyAsync(cut_host, cut, sizeof(double) * nq, cudaMemcpyDeviceToHost, st));
  if (pl_status s = read_status(ctx, st)) return s;
  *alpha_hat = obs[0];
  *D = obs[1];
  *p = ph;
  return PL_OK;
}
}  // namespace

pl_status pl_bootstrap_pvalue(pl_ctx *ctx, const int32_t *x_dev, int64_t n, uint64_t xmin, int64_t B,
                              uint64_t seed, uint64_t request_id, pl_precision prec, double *alpha_hat,
                              double *D, double *p, void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  return run_bootstrap(ctx, x_dev, n, xmin, B, seed, request_id, prec, nullptr, 0, alpha_hat, D, p, nullptr,
                       (cudaStream_t)stream);
}

pl_status pl_bespoke_cutoffs(pl_ctx *ctx, const int32_t *x_dev, int64_t n, uint64_t xmin, int64_t R, uint64_t seed,
                             uint64_t request_id, const double *q, int nq, pl_precision prec, double *alpha_hat,
                             double *D, double *p, double *cutoffs_host, void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!q || nq < 1 || !cutoffs_host) return fail(ctx, PL_EINVAL, "pl_bespoke_cutoffs: bad arguments");
  return run_bootstrap(ctx, x_dev, n, xmin, R, seed, request_id, prec, q, nq, alpha_hat, D, p, cutoffs_host,
                       (cudaStream_t)stream);
}

pl_status pl_bespoke_cutoffs_batch(pl_ctx *ctx, int nsets, const int32_t *const *x_dev, const int64_t *n,
                                   const uint64_t *xmin, int64_t R, uint64_t seed, const uint64_t *request_id,
                                   const double *q, int nq, pl_precision prec, double *alpha_hat, double *D,
                                   double *p, double *cutoffs_host, void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (nsets < 1 || !x_dev || !n || !xmin || !request_id || !q || nq < 1 || !alpha_hat || !D || !p ||
      !cutoffs_host || R < 1 || R > (1ll << 31))
    return fail(ctx, PL_EINVAL, "pl_bespoke_cutoffs_batch: bad arguments");
  if (prec != PL_FP64 && prec != PL_FP32_BULK) return fail(ctx, PL_EINVAL, "unknown precision form");
  for (int j = 0; j < nq; ++j)
    if (!(q[j] > 0.0 && q[j] < 1.0)) return fail(ctx, PL_EINVAL, "quantile %d outside (0, 1)", j);
  for (int i = 0; i < nsets; ++i)
    if (!x_dev[i] || n[i] < 1 || n[i] > INT32_MAX || xmin[i] < 1 || xmin[i] > (1ull << 31) ||
        request_id[i] >= (1ull << 32))
      return fail(ctx, PL_EINVAL, "pl_bespoke_cutoffs_batch: data set %d: bad arguments", i);
  cudaStream_t st = (cudaStream_t)stream;
  const bool f32 = prec == PL_FP32_BULK;
  // 1. every data set's fit and D (the data-set kernel, one log table per lower end), one synchronisation
  std::map<uint64_t, int> law_of;
  std::vector<LawPlan> lps;
  for (int i = 0; i < nsets; ++i)
    if (law_of.emplace(xmin[i], (int)lps.size()).second) lps.push_back({2.0, xmin[i], kL1});
  std::vector<Law> lh(lps.size());
  std::vector<Law *> ld(lps.size());
  std::vector<uint64_t *> spill(nsets), pairs(nsets);
  double *outs = nullptr;
  auto lay_fit = [&](Carver &cv) {
    for (size_t k = 0; k < lps.size(); ++k) {
      lh[k] = carve_law(cv, lps[k]);
      ld[k] = cv.take<Law>(1);
    }
    for (int i = 0; i < nsets; ++i) {
      spill[i] = cv.take<uint64_t>(next_pow2((uint64_t)n[i]));
      pairs[i] = cv.take<uint64_t>(2 * (size_t)n[i]);
    }
    outs = cv.take<double>(4 * (size_t)nsets);
  };
  {
    Carver cv;
    lay_fit(cv);
    if (pl_status s = ensure_ws(ctx, cv.off)) return s;
    cv.base = ctx->ws;
    cv.off = 0;
    lay_fit(cv);
  }
  for (size_t k = 0; k < lps.size(); ++k) {
    PL_CUDA(cudaMemcpyAsync(ld[k], &lh[k], sizeof(Law), cudaMemcpyHostToDevice, st));
    PL_CUDA(launch_law_setup(ld[k], 1, st));
    ctx->launches += kLawSetupLaunches;
  }
  // the fits are independent one-block kernels: spread over the side streams
  const int naux = std::min(nsets, pl_ctx::kAux);
  for (int k = 0; k < naux; ++k)
    if (!ctx->aux[k]) PL_CUDA(cudaStreamCreateWithFlags(&ctx->aux[k], cudaStreamNonBlocking));
  for (auto &e : ctx->aux_ev)
    if (!e) PL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  PL_CUDA(cudaEventRecord(ctx->aux_ev[pl_ctx::kAux], st));
  for (int k = 0; k < naux; ++k) PL_CUDA(cudaStreamWaitEvent(ctx->aux[k], ctx->aux_ev[pl_ctx::kAux], 0));
  for (int i = 0; i < nsets; ++i) {
    PL_CUDA(launch_dataset(x_dev[i], n[i], xmin[i], true, 0.0, ld[law_of[xmin[i]]], cell_const(xmin[i]), f32,
                           spill[i], pairs[i], outs + 4 * (size_t)i, ctx->ctr, ctx->aux[i % naux]));
    ctx->launches += 1;
  }
  for (int k = 0; k < naux; ++k) {
    PL_CUDA(cudaEventRecord(ctx->aux_ev[k], ctx->aux[k]));
    PL_CUDA(cudaStreamWaitEvent(st, ctx->aux_ev[k], 0));
  }
  std::vector<double> obs(4 * (size_t)nsets);
  PL_CUDA(cudaMemcpyAsync(obs.data(), outs, sizeof(double) * obs.size(), cudaMemcpyDeviceToHost, st));
  if (pl_status s = read_status(ctx, st)) return s;
  // 2. one simulation of every data set's cell at its fit (purpose 1, cell = request id)
  std::vector<pl_cell> cells(nsets);
  for (int i = 0; i < nsets; ++i) cells[i] = pl_cell{obs[4 * (size_t)i], xmin[i], n[i], R, request_id[i]};
  SimPlan sp;
  if (pl_status s = plan_cells(ctx, cells.data(), nsets, 1u, sp)) return s;
  const size_t dsz = f32 ? 4 : 8;
  const int blocks = sim_blocks(ctx, f32), sblocks = sample_blocks(ctx),
            bsblocks = ctx->num_sms * std::max(1, ctx->block_sampler_per_sm);
  SimBuffers b;
  uint8_t *Db = nullptr;
  int64_t *off = nullptr, *Rs = nullptr, *rank = nullptr;
  double *dobs = nullptr, *pd = nullptr, *cut = nullptr;
  auto lay_sim = [&](Carver &cv) {
    carve_sim(cv, sp, blocks, sblocks, b, ctx->dbg_arena, bsblocks);
    Db = cv.take<uint8_t>((size_t)sp.total_R * dsz);
    off = cv.take<int64_t>(nsets);
    Rs = cv.take<int64_t>(nsets);
    rank = cv.take<int64_t>((size_t)nsets * nq);
    dobs = cv.take<double>(nsets);
    pd = cv.take<double>(nsets);
    cut = cv.take<double>((size_t)nsets * nq);
  };
  {
    Carver cv;
    lay_sim(cv);
    if (pl_status s = ensure_ws(ctx, cv.off)) return s;
    cv.base = ctx->ws;
    cv.off = 0;
    lay_sim(cv);
  }
  if (pl_status s = mark(ctx, 0, st)) return s;
  if (pl_status s = upload_sim(ctx, sp, b, st)) return s;
  std::vector<int64_t> h_off(nsets), h_R(nsets), h_rank((size_t)nsets * nq);
  std::vector<double> h_dobs(nsets);
  for (int c = 0; c < nsets; ++c) {
    h_off[c] = sp.cells[c].out_off;
    h_R[c] = sp.cells[c].R;
    h_dobs[c] = obs[4 * (size_t)c + 1];
    for (int j = 0; j < nq; ++j) {
      const int64_t i = (int64_t)std::floor((double)h_R[c] * q[j]);
      h_rank[(size_t)c * nq + j] = std::min(std::max<int64_t>(i, 0), h_R[c] - 1);
    }
  }
  PL_CUDA(cudaMemcpyAsync(off, h_off.data(), sizeof(int64_t) * nsets, cudaMemcpyHostToDevice, st));
  PL_CUDA(cudaMemcpyAsync(Rs, h_R.data(), sizeof(int64_t) * nsets, cudaMemcpyHostToDevice, st));
  PL_CUDA(cudaMemcpyAsync(rank, h_rank.data(), sizeof(int64_t) * h_rank.size(), cudaMemcpyHostToDevice, st));
  PL_CUDA(cudaMemcpyAsync(dobs, h_dobs.data(), sizeof(double) * nsets, cudaMemcpyHostToDevice, st));
  if (pl_status s = mark(ctx, 1, st)) return s;
  if (pl_status s = run_sim(ctx, sp, b, seed, f32, Db, nullptr, st)) return s;
  if (pl_status s = mark(ctx, 2, st)) return s;
  PL_CUDA(launch_select(Db, f32, off, Rs, rank, nsets, nq, cut, st));
  for (int c = 0; c < nsets; ++c)
    PL_CUDA(launch_count_ge(Db + (size_t)h_off[c] * dsz, f32, R, dobs + c, pd + c, st));
  ctx->launches += 1 + (uint64_t)nsets;
  if (pl_status s = mark(ctx, 3, st)) return s;
  PL_CUDA(cudaMemcpyAsync(p, pd, sizeof(double) * nsets, cudaMemcpyDeviceToHost, st));
  PL_CUDA(cudaMemcpyAsync(cutoffs_host, cut, sizeof(double) * nsets * nq, cudaMemcpyDeviceToHost, st));
  if (pl_status s = read_status(ctx, st)) return s;
  for (int i = 0; i < nsets; ++i) {
    alpha_hat[i] = obs[4 * (size_t)i];
    D[i] = obs[4 * (size_t)i + 1];
  }
  return PL_OK;
}

pl_status pl_cutoff_lookup(pl_ctx *ctx, const double *grid_alpha, int na, const int64_t *grid_n, int nn,
                           const double *table_dev, int nq, const double *alpha_dev, const int64_t *n_dev,
                           int64_t nquery, double *out_dev, void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!grid_alpha || !grid_n || na < 1 || nn < 1 || na > kLookupGridMax || nn > kLookupGridMax || nq < 1 ||
      nquery < 0 || !table_dev ||
      (nquery > 0 && (!alpha_dev || !n_dev || !out_dev)))
    return fail(ctx, PL_EINVAL, "pl_cutoff_lookup: bad arguments");
  for (int i = 0; i < na; ++i)
    if (!std::isfinite(grid_alpha[i]) || (i && !(grid_alpha[i] > grid_alpha[i - 1])))
      return fail(ctx, PL_EINVAL, "pl_cutoff_lookup: exponent grid not strictly increasing");
  for (int i = 0; i < nn; ++i)
    if (grid_n[i] < 1 || (i && !(grid_n[i] > grid_n[i - 1])))
      return fail(ctx, PL_EINVAL, "pl_cutoff_lookup: sample-size grid not strictly increasing from 1");
  cudaStream_t st = (cudaStream_t)stream;
  auto lay = [&](Carver &cv, double *&ga, int64_t *&gn) {
    ga = cv.take<double>(na);
    gn = cv.take<int64_t>(nn);
  };
  Carver cv;
  double *ga;
  int64_t *gn;
  lay(cv, ga, gn);
  if (pl_status s = ensure_ws(ctx, cv.off)) return s;
  cv.base = ctx->ws;
  cv.off = 0;
  lay(cv, ga, gn);
  PL_CUDA(cudaMemcpyAsync(ga, grid_alpha, sizeof(double) * na, cudaMemcpyHostToDevice, st));
  PL_CUDA(cudaMemcpyAsync(gn, grid_n, sizeof(int64_t) * nn, cudaMemcpyHostToDevice, st));
  PL_CUDA(launch_lookup(ga, na, gn, nn, table_dev, nq, alpha_dev, n_dev, nquery, out_dev, st));
  ctx->launches += nquery > 0 ? 1 : 0;
  return PL_OK;
}

pl_status pl_estimate_xmin(pl_ctx *ctx, const int32_t *x_dev, int64_t n, int64_t max_candidates, int64_t min_tail,
                           pl_xmin_result *out_host, uint64_t *cand_xmin_dev, double *cand_alpha_dev,
                           double *cand_D_dev, int64_t *cand_ntail_dev, void *stream) {
  if (pl_status s = check_ctx(ctx)) return s;
  if (!x_dev || n < 1 || n > INT32_MAX || max_candidates < 1 || max_candidates > (1ll << 24) || min_tail < 1 ||
      !out_host)
    return fail(ctx, PL_EINVAL, "pl_estimate_xmin: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t P = next_pow2((uint64_t)n);
  auto lay = [&](Carver &cv, uint32_t *&ghist, unsigned long long *&nsp, uint64_t *&spill, uint64_t *&vals,
                 uint32_t *&cnts, int64_t *&S, double *&Lt, int64_t *&d, uint64_t *&cx, double *&ca, double *&cD,
                 int64_t *&cn, XminOut *&out) {
    ghist = cv.take<uint32_t>(kXHistBins);
    nsp = cv.take<unsigned long long>(1);
    spill = cv.take<uint64_t>(P);
    vals = cv.take<uint64_t>(n);
    cnts = cv.take<uint32_t>(n);
    S = cv.take<int64_t>(n + 1);
    Lt = cv.take<double>(n);
    d = cv.take<int64_t>(1);
    cx = cand_xmin_dev ? cand_xmin_dev : cv.take<uint64_t>(max_candidates);
    ca = cand_alpha_dev ? cand_alpha_dev : cv.take<double>(max_candidates);
    cD = cand_D_dev ? cand_D_dev : cv.take<double>(max_candidates);
    cn = cand_ntail_dev ? cand_ntail_dev : cv.take<int64_t>(max_candidates);
    out = cv.take<XminOut>(1);
  };
  Carver cv;
  uint32_t *ghist;
  unsigned long long *nsp;
  uint64_t *spill, *vals, *cx;
  uint32_t *cnts;
  int64_t *S, *d, *cn;
  double *Lt, *ca, *cD;
  XminOut *out;
  lay(cv, ghist, nsp, spill, vals, cnts, S, Lt, d, cx, ca, cD, cn, out);
  if (pl_status s = ensure_ws(ctx, cv.off)) return s;
  cv.base = ctx->ws;
  cv.off = 0;
  lay(cv, ghist, nsp, spill, vals, cnts, S, Lt, d, cx, ca, cD, cn, out);
  PL_CUDA(launch_xmin(x_dev, n, ghist, nsp, spill, vals, cnts, S, Lt, d, max_candidates, min_tail, cx, ca, cD, cn,
                      out, ctx->ctr, ctx->num_sms, st));
  ctx->launches += 4;
  XminOut o{};
  PL_CUDA(cudaMemcpyAsync(&o, out, sizeof o, cudaMemcpyDeviceToHost, st));
  if (pl_status s = read_status(ctx, st)) return s;
  out_host->xmin = o.xmin;
  out_host->alpha_hat = o.alpha_hat;
  out_host->D = o.D;
  out_host->n_tail = o.n_tail;
  out_host->candidates = o.candidates;
  return PL_OK;
}

#ifdef PL_PHASE_TIMING
pl_status pl_debug_phase_cycles(pl_ctx *ctx, uint64_t out[8]) {
  if (pl_status s = check_ctx(ctx)) return s;
  PL_CUDA(cudaDeviceSynchronize());
  Counters c{};
  PL_CUDA(cudaMemcpy(&c, ctx->ctr, sizeof c, cudaMemcpyDeviceToHost));
  for (int i = 0; i < 8; ++i) out[i] = c.phase_cycles[i];
  return PL_OK;
}
#endif

}  // extern "C"
