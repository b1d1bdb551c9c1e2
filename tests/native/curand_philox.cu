// Test helper (not part of the library): draws cuRAND's Philox4_32_10 so a
// GPU test can compare the CPU oracle's Philox4x32-10 against NVIDIA's.
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void draw(unsigned long long seed, unsigned long long subseq, unsigned long long offset, int n,
                     uint4* out) {
  curandStatePhilox4_32_10_t st;
  curand_init(seed, subseq, offset, &st);
  for (int k = 0; k < n; ++k) out[k] = curand4(&st);
}

extern "C" int curand_philox_draw(unsigned long long seed, unsigned long long subseq, unsigned long long offset,
                                  int n, unsigned* host_out) {
  uint4* d = nullptr;
  if (cudaMalloc(&d, sizeof(uint4) * (size_t)n) != cudaSuccess) return 1;
  draw<<<1, 1>>>(seed, subseq, offset, n, d);
  cudaError_t e = cudaMemcpy(host_out, d, sizeof(uint4) * (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? 0 : 2;
}
