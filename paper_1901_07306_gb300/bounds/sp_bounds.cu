// sp_bounds.cu -- hardware probes behind the scan's roofline figures
// (include/sp_bounds.h): streaming HBM reads, random L2 atomic ORs and random
// shared-memory atomic ORs.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sp_bounds.h"

namespace {

__global__ void __launch_bounds__(256) k_probe_read(const uint4* __restrict__ p, uint64_t n16, uint32_t* sink) {
  uint32_t acc = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 v = __ldcs(p + i);
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  acc = __reduce_xor_sync(0xFFFFFFFFu, acc);
  __shared__ uint32_t s[8];
  if ((threadIdx.x & 31u) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t x = 0;
    for (int w = 0; w < 8; ++w) x ^= s[w];
    sink[blockIdx.x] = x;
  }
}

// x_{j+1} = 1664525 x_j + 1013904223 (mod 2^32); the word index is the top bits
__device__ __forceinline__ uint32_t lcg(uint32_t x) { return x * 1664525u + 1013904223u; }

__global__ void __launch_bounds__(256)
k_probe_red(uint32_t* __restrict__ words, uint32_t shift, uint32_t ops, uint32_t seed) {
  uint32_t x = seed ^ ((blockIdx.x * blockDim.x + threadIdx.x) * 0x9E3779B9u);
  for (uint32_t j = 0; j < ops; ++j) {
    x = lcg(x);
    atomicOr(words + (x >> shift), 1u << (x & 31u));
  }
}

__global__ void __launch_bounds__(512)
k_probe_smem(uint32_t* __restrict__ sink, uint32_t words_log2, uint32_t ops, uint32_t seed) {
  __shared__ uint32_t s[1u << 13];
  const uint32_t n = 1u << words_log2, shift = 32u - words_log2;
  for (uint32_t w = threadIdx.x; w < n; w += blockDim.x) s[w] = 0u;
  __syncthreads();
  uint32_t x = seed ^ ((blockIdx.x * blockDim.x + threadIdx.x) * 0x9E3779B9u);
  for (uint32_t j = 0; j < ops; ++j) {
    x = lcg(x);
    atomicOr(s + (x >> shift), 1u << (x & 31u));
  }
  __syncthreads();
  for (uint32_t w = threadIdx.x; w < n; w += blockDim.x)
    if (s[w]) atomicOr(sink + w, s[w]);
}

int sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

}  // namespace

extern "C" {

int sp_probe_stream_read(const void* dev_buf, uint64_t bytes, uint32_t* dev_sink, uint32_t grid, void* cuda_stream) {
  if (!dev_buf || !dev_sink || (bytes & 15u) || ((uintptr_t)dev_buf & 15u)) return -1;
  if (grid == 0) grid = (uint32_t)sms() * 8u;
  k_probe_read<<<grid, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(static_cast<const uint4*>(dev_buf),
                                                                        bytes / 16, dev_sink);
  return cudaGetLastError() == cudaSuccess ? 0 : -5;
}

int sp_probe_l2_red(uint32_t* dev_words, uint32_t words_log2, uint32_t ops_per_thread, uint32_t grid, uint32_t seed,
                    void* cuda_stream) {
  if (!dev_words || words_log2 < 1 || words_log2 > 31) return -1;
  if (grid == 0) grid = (uint32_t)sms() * 8u;
  k_probe_red<<<grid, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(dev_words, 32u - words_log2,
                                                                       ops_per_thread, seed);
  return cudaGetLastError() == cudaSuccess ? 0 : -5;
}

int sp_probe_smem_atomic(uint32_t* dev_sink, uint32_t words_log2, uint32_t ops_per_thread, uint32_t grid,
                         uint32_t seed, void* cuda_stream) {
  if (!dev_sink || words_log2 < 1 || words_log2 > 13) return -1;
  if (grid == 0) grid = (uint32_t)sms() * 4u;
  k_probe_smem<<<grid, 512, 0, static_cast<cudaStream_t>(cuda_stream)>>>(dev_sink, words_log2, ops_per_thread, seed);
  return cudaGetLastError() == cudaSuccess ? 0 : -5;
}

}  // extern "C"
