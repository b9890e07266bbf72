// Test helper: Philox4x32-10 blocks from cuRAND's device generator, for
// pinning the oracle's generator at counters whose fourth word is nonzero
// (curand_init(seed, subsequence, offset): the block after the call has the
// counter (offset / 4 as two words, subsequence as two words)).
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void curand_blocks_kernel(unsigned long long seed, const unsigned long long *subseq,
                                     const unsigned long long *offset, int n, uint4 *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seed, subseq[i], offset[i], &st);
  out[i] = curand4(&st);
}

extern "C" int curand_philox_blocks(unsigned long long seed, const unsigned long long *subseq_host,
                                    const unsigned long long *offset_host, int n, unsigned int *out_host) {
  if (n < 1) return 0;
  unsigned long long *d_s = nullptr, *d_o = nullptr;
  uint4 *d_out = nullptr;
  cudaError_t e = cudaMalloc(&d_s, sizeof(unsigned long long) * n);
  if (e == cudaSuccess) e = cudaMalloc(&d_o, sizeof(unsigned long long) * n);
  if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(uint4) * n);
  if (e == cudaSuccess) e = cudaMemcpy(d_s, subseq_host, sizeof(unsigned long long) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_o, offset_host, sizeof(unsigned long long) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    curand_blocks_kernel<<<(n + 127) / 128, 128>>>(seed, d_s, d_o, n, d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out_host, d_out, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
  cudaFree(d_s);
  cudaFree(d_o);
  cudaFree(d_out);
  return (int)e;
}
