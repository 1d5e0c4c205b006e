// Test infrastructure: cuRAND's Philox4_32_10 generator (its documented
// device API) evaluated at given (counter, key) pairs, a third-party
// reference for the library's device Philox.  curand_init(seed,
// subsequence, offset) starts the generator at counter (offset/4 as a
// 64-bit value in words 0-1, subsequence in words 2-3) under key = seed;
// curand4 then returns the four words of that counter.
#include <cstdint>
#include <curand_kernel.h>

__global__ void k_curand_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long seed = ((unsigned long long)key[2 * i + 1] << 32) | key[2 * i];
  const unsigned long long low = ((unsigned long long)ctr[4 * i + 1] << 32) | ctr[4 * i];
  const unsigned long long high = ((unsigned long long)ctr[4 * i + 3] << 32) | ctr[4 * i + 2];
  curandStatePhilox4_32_10_t st;
  curand_init(seed, high, 0ull, &st);
  skipahead(low, &st);   // advances by `low` numbers: counter words 0-1 += low / 4
  skipahead(low, &st);
  skipahead(low, &st);
  skipahead(low, &st);   // four times: counter words 0-1 += low
  const uint4 v = curand4(&st);
  out[4 * i + 0] = v.x;
  out[4 * i + 1] = v.y;
  out[4 * i + 2] = v.z;
  out[4 * i + 3] = v.w;
}

extern "C" int curand_philox_words(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n) {
  uint32_t *dc, *dk, *dout;
  if (cudaMalloc(&dc, 16ull * n) != cudaSuccess || cudaMalloc(&dk, 8ull * n) != cudaSuccess ||
      cudaMalloc(&dout, 16ull * n) != cudaSuccess)
    return 1;
  cudaMemcpy(dc, ctr, 16ull * n, cudaMemcpyHostToDevice);
  cudaMemcpy(dk, key, 8ull * n, cudaMemcpyHostToDevice);
  k_curand_philox<<<(n + 127) / 128, 128>>>(dc, dk, dout, n);
  const cudaError_t e = cudaMemcpy(out, dout, 16ull * n, cudaMemcpyDeviceToHost);
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  return e == cudaSuccess ? 0 : 2;
}
