// pl_probe.cu -- issue-rate probe of the units that bound the kernels.
//
// The samplers are bound by 32x32->64-bit multiplies (Philox4x32-10 takes 20
// per block of four 32-bit words) and by integer/logic issue; the fit and the
// binary64 KS are bound by the binary64 pipe.  Each probe kernel keeps every
// thread busy with eight independent dependency chains of one instruction
// (so the unit, not latency, limits it) and writes one word per thread so
// that nothing is optimised away.  One 1024-thread block per SM; thread 0 of
// every block reads clock64 around its loop and the largest count is kept:
// it is the kernel's length in SM cycles, and cycles over the CUDA-event time
// give the SM clock of the run.
#include <cstdint>

#include "pl_probe.cuh"

namespace pl {

namespace {

constexpr int kChains = kProbeChains;

__device__ __forceinline__ void probe_clock(long long *cyc, long long t0) {
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(reinterpret_cast<unsigned long long *>(cyc), (unsigned long long)(clock64() - t0));
}

__global__ void __launch_bounds__(kProbeBlock) probe_mul_wide(uint32_t *out, long long *cyc, int iters, uint32_t s) {
  const long long t0 = clock64();
  uint32_t a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = threadIdx.x * 7u + (uint32_t)c + s;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      uint32_t lo, hi;
      asm volatile("{\n\t.reg .b64 t;\n\tmul.wide.u32 t, %2, 0xD2511F53;\n\tmov.b64 {%0, %1}, t;\n\t}"
                   : "=r"(lo), "=r"(hi)
                   : "r"(a[c]));
      a[c] = lo ^ hi;
    }
  }
  uint32_t r = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) r ^= a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
  probe_clock(cyc, t0);
}

__global__ void __launch_bounds__(kProbeBlock) probe_lop3(uint32_t *out, long long *cyc, int iters, uint32_t s) {
  const long long t0 = clock64();
  uint32_t a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = threadIdx.x * 7u + (uint32_t)c + s;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      uint32_t r;
      asm volatile("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(r) : "r"(a[c]), "r"(a[(c + 1) % kChains]), "r"(s));
      a[c] = r;
    }
  }
  uint32_t r = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) r ^= a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
  probe_clock(cyc, t0);
}

__global__ void __launch_bounds__(kProbeBlock) probe_dfma(uint32_t *out, long long *cyc, int iters, uint32_t s) {
  const long long t0 = clock64();
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = (double)(threadIdx.x * 7u + (uint32_t)c + s);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      double r;
      asm volatile("fma.rn.f64 %0, %1, 0d3FEFFFFFFFFFFFFE, 0d3FF0000000000000;" : "=d"(r) : "d"(a[c]));
      a[c] = r;
    }
  }
  double r = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) r += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (uint32_t)__double2hiint(r) ^ (uint32_t)__double2loint(r);
  probe_clock(cyc, t0);
}

// Philox4x32-10 blocks with counters (it, thread, 7, 0): iters blocks per thread.
__global__ void __launch_bounds__(kProbeBlock) probe_philox(uint32_t *out, long long *cyc, int iters, uint32_t s) {
  const long long t0 = clock64();
  const uint32_t rep = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (int it = 0; it < iters; ++it) {
    uint32_t c0 = (uint32_t)it, c1 = rep, c2 = 7u, c3 = 0u, k0 = s, k1 = 0x1234u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      uint32_t h0, l0, h1, l1;
      asm("{\n\t.reg .b64 t;\n\tmul.wide.u32 t, %2, 0xD2511F53;\n\tmov.b64 {%0, %1}, t;\n\t}"
          : "=r"(l0), "=r"(h0)
          : "r"(c0));
      asm("{\n\t.reg .b64 t;\n\tmul.wide.u32 t, %2, 0xCD9E8D57;\n\tmov.b64 {%0, %1}, t;\n\t}"
          : "=r"(l1), "=r"(h1)
          : "r"(c2));
      const uint32_t n0 = h1 ^ c1 ^ k0, n2 = h0 ^ c3 ^ k1;
      c0 = n0;
      c1 = l1;
      c2 = n2;
      c3 = l0;
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    acc ^= c0 ^ c1 ^ c2 ^ c3;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  probe_clock(cyc, t0);
}

}  // namespace

cudaError_t launch_probe(int kind, uint32_t *out, long long *cyc, int grid, int iters, uint32_t seed,
                         cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(cyc, 0, sizeof(long long), st);
  if (e != cudaSuccess) return e;
  switch (kind) {
    case kProbeMulWide: probe_mul_wide<<<grid, kProbeBlock, 0, st>>>(out, cyc, iters, seed); break;
    case kProbeLop3: probe_lop3<<<grid, kProbeBlock, 0, st>>>(out, cyc, iters, seed); break;
    case kProbeDfma: probe_dfma<<<grid, kProbeBlock, 0, st>>>(out, cyc, iters, seed); break;
    case kProbePhilox: probe_philox<<<grid, kProbeBlock, 0, st>>>(out, cyc, iters, seed); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace pl
