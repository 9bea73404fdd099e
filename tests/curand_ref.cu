// Test helper: cuRAND's Philox4_32_10 device generator (the library's own implementation), used
// only to check the project's Philox4x32-10 against it.  Built by test_gpu_rng.py into a temporary
// folder.  Output i is the first curand4() of a state initialised with (seed, subsequence[i],
// 4 * block[i]): Philox with key (seed low, seed high) and counter (block low, block high,
// subsequence low, subsequence high), per cuRAND's documented counter layout.
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void k_curand_ref(unsigned long long seed, const unsigned long long* sub, const unsigned long long* blk,
                             uint4* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t s;
  curand_init(seed, sub[i], 4ull * blk[i], &s);
  out[i] = curand4(&s);
}

extern "C" int curand_ref(unsigned long long seed, const unsigned long long* sub, const unsigned long long* blk,
                          unsigned int* out, int n) {
  unsigned long long *d_sub = nullptr, *d_blk = nullptr;
  uint4* d_out = nullptr;
  cudaError_t e = cudaMalloc(&d_sub, n * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&d_blk, n * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&d_out, n * sizeof(uint4));
  if (e == cudaSuccess) e = cudaMemcpy(d_sub, sub, n * sizeof(unsigned long long), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_blk, blk, n * sizeof(unsigned long long), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_curand_ref<<<(n + 127) / 128, 128>>>(seed, d_sub, d_blk, d_out, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, n * sizeof(uint4), cudaMemcpyDeviceToHost);
  cudaFree(d_sub);
  cudaFree(d_blk);
  cudaFree(d_out);
  return (int)e;
}
