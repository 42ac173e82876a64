// Test-only reference for the Philox4x32-10 pin: evaluates cuRAND's device-side
// curand_Philox4x32_10(counter, key) on caller-given counters and keys.  Compiled by the test
// that uses it, never into the library.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <stdint.h>

__global__ void k_curand_philox(const uint4 *ctr, const uint2 *key, uint4 *out, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = curand_Philox4x32_10(ctr[t], key[t]);
}

// ctr: host [n][4], key: host [n][2], out: host [n][4].  Returns a cudaError_t value.
extern "C" int curand_philox_words(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int n) {
  if (n <= 0) return 0;
  uint4 *dc = nullptr, *dout = nullptr;
  uint2 *dk = nullptr;
  cudaError_t e = cudaMalloc(&dc, sizeof(uint4) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dk, sizeof(uint2) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(uint4) * n);
  if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dk, key, sizeof(uint2) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_curand_philox<<<(n + 127) / 128, 128>>>(dc, dk, dout, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  return (int)e;
}
