// sp_merge.cu -- window start and global sketch construction.
//
// k_zero: every bit of SEAV and LDCA is 0 at the beginning of a time period
//   (Sec. 3.1, Sec. 3.3).
// k_merge: the global server's SEAV/LDCA (Sec. 4.2) as the bitwise OR of the
//   watch points' equal-size sketches; one pass reads every source once and
//   writes the destination once (uint4, grid-stride, HBM bound).
#include "sp_internal.h"

namespace sp {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxSrc = 32;

struct SrcList {
  const uint4* p[kMaxSrc];
};

__global__ void __launch_bounds__(kThreads)
k_zero(uint4* __restrict__ p, uint64_t n16, uint32_t* __restrict__ flags, uint32_t n_flags) {
  const uint4 z = make_uint4(0u, 0u, 0u, 0u);
  const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (uint64_t i = gid; i < n16; i += (uint64_t)gridDim.x * blockDim.x) p[i] = z;
  for (uint64_t i = gid; i < n_flags; i += (uint64_t)gridDim.x * blockDim.x) flags[i] = 0u;
}

__global__ void __launch_bounds__(kThreads)
k_merge(uint4* __restrict__ dst, SrcList src, uint32_t n_src, uint64_t n16) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (uint64_t)gridDim.x * blockDim.x) {
    uint4 acc = dst[i];
    for (uint32_t s = 0; s < n_src; ++s) {
      const uint4 v = __ldcs(src.p[s] + i);
      acc.x |= v.x; acc.y |= v.y; acc.z |= v.z; acc.w |= v.w;
    }
    dst[i] = acc;
  }
}

int stream_grid() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * 8;
}

}  // namespace

// bytes must be a multiple of 16 and the pointer 16-byte aligned (sketch
// regions are padded to 256 bytes by the context).
cudaError_t launch_zero_flags(void* dev, uint64_t bytes, uint32_t* flags, uint32_t n_flags, cudaStream_t s) {
  const uint64_t n16 = bytes / 16;
  const uint64_t work = n16 > n_flags ? n16 : n_flags;
  if (work == 0) return cudaSuccess;
  uint64_t grid = (work + kThreads - 1) / kThreads;
  if (grid > (uint64_t)stream_grid()) grid = stream_grid();
  k_zero<<<(unsigned)grid, kThreads, 0, s>>>(reinterpret_cast<uint4*>(dev), n16, flags, n_flags);
  return cudaGetLastError();
}

cudaError_t launch_zero(void* dev, uint64_t bytes, cudaStream_t s) {
  return launch_zero_flags(dev, bytes, nullptr, 0u, s);
}

cudaError_t launch_merge(uint8_t* dst, const uint8_t* const* srcs, uint32_t n_src,
                         uint64_t bytes, cudaStream_t s) {
  const uint64_t n16 = bytes / 16;
  if (n16 == 0 || n_src == 0) return cudaSuccess;
  uint64_t grid = (n16 + kThreads - 1) / kThreads;
  if (grid > (uint64_t)stream_grid()) grid = stream_grid();
  for (uint32_t base = 0; base < n_src; base += kMaxSrc) {
    SrcList l{};
    const uint32_t m = (n_src - base) < (uint32_t)kMaxSrc ? (n_src - base) : (uint32_t)kMaxSrc;
    for (uint32_t j = 0; j < m; ++j) l.p[j] = reinterpret_cast<const uint4*>(srcs[base + j]);
    k_merge<<<(unsigned)grid, kThreads, 0, s>>>(reinterpret_cast<uint4*>(dst), l, m, n16);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sp
