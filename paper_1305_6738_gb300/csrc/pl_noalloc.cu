// pl_noalloc.cu -- fit and KS distance of one data set without any device
// allocation: the scratch of the data-set kernel lives in a fixed file-scope
// device array instead of a context workspace.
//
// Who needs this: callers that cannot let a library call cudaMalloc, e.g. a
// runtime that reserves all device memory up front for its own pool allocator
// (a library cudaMalloc would then fail or fragment that pool), or a
// latency-critical loop that must never reach the allocator, whose calls can
// synchronise the device.  They pass their own input and output buffers; the
// scratch below is allocated once, at module load, by the CUDA runtime.
//
// Every call shares the one array (per device), which keeps the last call's
// contents; the set-up kernel of each call clears what must start at zero.
// Calls that overlap on the GPU (two streams, or two host threads) race on
// the array and must be serialised by the caller.
#include <cmath>
#include <mutex>

#include "pl.h"
#include "pl_kernels.cuh"

namespace {

using namespace pl;

constexpr int64_t kNoAllocMaxN = 262144;  // largest data set (values)

constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t kOffLaw = 0;
constexpr size_t kOffCtr = align256(sizeof(Law));
constexpr size_t kOffLnT = align256(kOffCtr + sizeof(Counters));
constexpr size_t kOffLnHi = align256(kOffLnT + (size_t)kLnTable * sizeof(double));
constexpr size_t kOffLnLo = align256(kOffLnHi + (size_t)kLnTable * sizeof(float));
constexpr size_t kOffSpill = align256(kOffLnLo + (size_t)kLnTable * sizeof(float));
constexpr size_t kOffPairs = align256(kOffSpill + (size_t)kNoAllocMaxN * sizeof(uint64_t));
constexpr size_t kScratchBytes = align256(kOffPairs + 2 * (size_t)kNoAllocMaxN * sizeof(uint64_t));

}  // namespace

// The scratch: about 6.3 MB, held by every GPU that loads the library until
// the process exits.  Host code must not use this name as an address (in host
// code it is a host-side stand-in); it uses the pointer from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

// ln tables of x_min + i and the law record the data-set kernel reads; zero
// counters.  Device code may name the array directly.
__global__ void noalloc_setup_kernel(uint64_t xmin, double alpha) {
  unsigned char *base = g_noalloc_scratch;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double *lnT = reinterpret_cast<double *>(base + kOffLnT);
  float *lnHi = reinterpret_cast<float *>(base + kOffLnHi);
  float *lnLo = reinterpret_cast<float *>(base + kOffLnLo);
  if (i < kLnTable) {
    const double l = log((double)(xmin + (uint64_t)i));
    const float hi = (float)l;
    lnT[i] = l;
    lnHi[i] = hi;
    lnLo[i] = (float)(l - (double)hi);
  }
  if (i == 0) {
    Law *law = reinterpret_cast<Law *>(base + kOffLaw);
    *law = Law{};
    law->alpha = alpha;
    law->xmin = xmin;
    law->lnT = lnT;
    law->lnT_hi = lnHi;
    law->lnT_lo = lnLo;
    Counters *ctr = reinterpret_cast<Counters *>(base + kOffCtr);
    *ctr = Counters{};
  }
}

// Device address of the scratch, looked up once per device with that device
// current (the first call of the entry point on each device does it).
std::mutex g_mu;
unsigned char *g_base[64] = {};

pl_status scratch_address(unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PL_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_base[dev]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return PL_ECUDA;
    g_base[dev] = static_cast<unsigned char *>(ptr);
  }
  *out = g_base[dev];
  return PL_OK;
}

}  // namespace

extern "C" pl_status pl_fit_ks_noalloc(const int32_t *x_dev, int64_t n, uint64_t xmin, double alpha,
                                       pl_precision prec, double *out_dev, void *stream) {
  if (!x_dev || !out_dev || n < 1 || xmin < 1 || xmin > (1ull << 31)) return PL_EINVAL;
  if (n > kNoAllocMaxN) return PL_EINVAL;
  if (prec != PL_FP64 && prec != PL_FP32_BULK) return PL_EINVAL;
  const bool fit = !(alpha > 0.0);  // NaN or <= 0: fit the exponent
  if (!fit && (!(alpha > 1.0) || alpha > 64.0)) return PL_EINVAL;
  unsigned char *base = nullptr;
  if (pl_status s = scratch_address(&base)) return s;
  cudaStream_t st = (cudaStream_t)stream;
  noalloc_setup_kernel<<<(kLnTable + 255) / 256, 256, 0, st>>>(xmin, fit ? 2.0 : alpha);
  if (cudaGetLastError() != cudaSuccess) return PL_ECUDA;
  CellConst cc;
  cc.ln_xmin_half = std::log((double)xmin - 0.5);
  cc.ln_allmin = std::log1p(1.0 / (double)xmin);
  cc.ln_xmin = std::log((double)xmin);
  const cudaError_t e = launch_dataset(
      x_dev, n, xmin, fit, fit ? 0.0 : alpha, reinterpret_cast<const Law *>(base + kOffLaw), cc,
      prec == PL_FP32_BULK, reinterpret_cast<uint64_t *>(base + kOffSpill),
      reinterpret_cast<uint64_t *>(base + kOffPairs), out_dev, reinterpret_cast<Counters *>(base + kOffCtr), st);
  return e == cudaSuccess ? PL_OK : PL_ECUDA;
}
