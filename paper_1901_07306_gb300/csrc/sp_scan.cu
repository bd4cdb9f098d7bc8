// sp_scan.cu -- the per-pair scan of one watch point (Sec. 3.1-3.3, Sec. 4.1).
//
// Every pair <hip, oip> (Sec. 3.2) does two things:
//   SEAV (Sec. 3.1-3.2): if lsb(H1(oip)) >= tau, set bit H2(oip) of the SE at
//     column Idx(i, LP(hip)) (Eq. 2) in each row i of SEA RP(hip);
//   LDCA (Sec. 3.3): set bit H3(oip) of LDC LH_i(hip) in each row i.
// Setting a bit is idempotent, so concurrent threads need no ordering
// (Sec. 3.4): each update is one fire-and-forget atomic OR (a RED in L2).
//
// Layout: pairs are interleaved uint32 (hip, oip), read as uint4 (two pairs
// per 16-byte load, coalesced, streaming).  SEAV is bytes [2^r][sum SC(i)];
// LDCA is words [lr][LC][k / 32].  The grid is persistent: a multiple of the
// SM count times the resident blocks per SM, striding over the stream.
#include "sp_internal.h"

namespace sp {

namespace {

constexpr int kScanThreads = 256;

__device__ __forceinline__ void seav_update(const DevParams& d, uint8_t* seav, uint32_t hip, uint32_t h1) {
  const uint32_t bit = h1 >> 29;                                 // H2: 3 top bits (g = 8)
  const uint32_t rp = d.r ? (hip & ((1u << d.r) - 1u)) : 0u;
  const uint32_t lp = (uint32_t)((uint64_t)hip >> d.r);
  const uint64_t base = (uint64_t)rp * d.sea_bytes;
  for (uint32_t i = 0; i < d.sr; ++i) {
    const uint64_t off = base + d.row_off[i] + gather_idx(lp, d.isb[i], d.ibn[i], d.L);
    atomicOr(reinterpret_cast<uint32_t*>(seav + (off & ~3ull)), (1u << bit) << (8u * (uint32_t)(off & 3u)));
  }
}

template <int LR>
__device__ __forceinline__ void scan_pair(const DevParams& d, uint8_t* seav, uint32_t* ldca,
                                          uint32_t hip, uint32_t oip, uint32_t tau_mask) {
  const uint32_t h1 = mas(d.ha[0], d.hb[0], oip);
  if ((h1 & tau_mask) == 0u) seav_update(d, seav, hip, h1);     // lsb(h1) >= tau
  const uint32_t h3 = mas(d.ha[1], d.hb[1], oip) >> (32u - d.k_log2);
  const uint32_t word = h3 >> 5, mask = 1u << (h3 & 31u);
  const uint32_t wshift = d.k_log2 - 5u;
  const uint32_t cshift = 32u - d.lc_log2;                      // 32 when LC = 1
#pragma unroll
  for (int i = 0; i < LR; ++i) {
    const uint32_t col = (uint32_t)((uint64_t)mas(d.ha[2 + i], d.hb[2 + i], hip) >> cshift);
    const uint32_t line = ((uint32_t)i << d.lc_log2) | col;
    atomicOr(ldca + (((uint64_t)line << wshift) | word), mask);
  }
}

template <int LR>
__global__ void __launch_bounds__(kScanThreads)
k_scan(DevParams d, uint8_t* __restrict__ seav, uint32_t* __restrict__ ldca,
       const uint32_t* __restrict__ pairs, uint64_t n_pairs) {
  const uint32_t tau_mask = (d.tau >= 32u) ? 0xFFFFFFFFu : ((1u << d.tau) - 1u);
  // peel one pair when the stream is 8- but not 16-byte aligned
  const uint64_t head = (((uintptr_t)pairs & 15u) != 0u && n_pairs > 0) ? 1u : 0u;
  const uint64_t body = (n_pairs - head) >> 1;                     // uint4 = 2 pairs
  const uint4* p4 = reinterpret_cast<const uint4*>(pairs + 2 * head);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < body; j += stride) {
    const uint4 v = __ldcs(p4 + j);
    scan_pair<LR>(d, seav, ldca, v.x, v.y, tau_mask);
    scan_pair<LR>(d, seav, ldca, v.z, v.w, tau_mask);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (head) scan_pair<LR>(d, seav, ldca, pairs[0], pairs[1], tau_mask);
    if ((n_pairs - head) & 1u) {
      const uint64_t last = n_pairs - 1;
      scan_pair<LR>(d, seav, ldca, pairs[2 * last], pairs[2 * last + 1], tau_mask);
    }
  }
}

template <int LR>
int grid_for() {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan<LR>, kScanThreads, 0);
  if (per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

// ---- batched form: many (router, pairs) batches in one persistent launch ----
//
// The work unit is a chunk of kChunk pairs of one batch.  Every block scans
// the batch table once into a shared prefix of chunk counts (a batch with a
// router out of range or a misaligned stream counts 0 chunks and raises bit 1
// of *err), then takes chunks g = block, block + grid, ... and finds each
// chunk's batch by binary search.  Routers index the context's sketches.
constexpr uint32_t kChunk = 2048;

template <int LR, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_scan_multi(DevParams d, uint8_t* __restrict__ sketches, uint64_t stride, uint64_t seav_pad,
             uint32_t n_routers, const sp_batch* __restrict__ desc, uint32_t n_batches,
             uint32_t* __restrict__ err) {
  extern __shared__ uint64_t s_pref[];                     // [n_batches + 1]
  __shared__ uint64_t s_carry;
  const uint32_t tid = threadIdx.x;
  const uint32_t tau_mask = (1u << d.tau) - 1u;
  if (tid == 0) { s_carry = 0; s_pref[0] = 0; }
  __syncthreads();
  for (uint32_t base = 0; base < n_batches; base += THREADS) {
    const uint32_t b = base + tid;
    uint64_t c = 0;
    if (b < n_batches) {
      const sp_batch x = desc[b];
      const bool ok = x.router < n_routers && (x.n_pairs == 0 || (x.pairs && ((uintptr_t)x.pairs & 7u) == 0));
      if (!ok && blockIdx.x == 0) atomicOr(err, 2u);
      c = ok ? (x.n_pairs + kChunk - 1) / kChunk : 0;
    }
    // inclusive block scan of c (THREADS <= 1024) through shared memory
    __shared__ uint64_t s_tmp[1024];
    s_tmp[tid] = c;
    __syncthreads();
    for (uint32_t o = 1; o < THREADS; o <<= 1) {
      const uint64_t y = tid >= o ? s_tmp[tid - o] : 0;
      __syncthreads();
      s_tmp[tid] += y;
      __syncthreads();
    }
    if (b < n_batches) s_pref[b + 1] = s_carry + s_tmp[tid];
    __syncthreads();
    if (tid == THREADS - 1) s_carry += s_tmp[tid];
    __syncthreads();
  }
  const uint64_t total = s_pref[n_batches];
  for (uint64_t g = blockIdx.x; g < total; g += gridDim.x) {
    uint32_t lo = 0, hi = n_batches;                       // last b with s_pref[b] <= g
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_pref[mid] <= g) lo = mid; else hi = mid;
    }
    const sp_batch x = desc[lo];
    const uint64_t start = (g - s_pref[lo]) * kChunk;
    const uint32_t cnt = (uint32_t)((x.n_pairs - start) < kChunk ? (x.n_pairs - start) : kChunk);
    uint8_t* seav = sketches + (uint64_t)x.router * stride;
    uint32_t* ldca = reinterpret_cast<uint32_t*>(seav + seav_pad);
    const uint2* p2 = reinterpret_cast<const uint2*>(x.pairs) + start;
    for (uint32_t i = tid; i < cnt; i += THREADS) {
      const uint2 v = __ldcs(p2 + i);
      scan_pair<LR>(d, seav, ldca, v.x, v.y, tau_mask);
    }
  }
}

template <int LR>
cudaError_t multi_lr(const DevParams& d, uint8_t* sketches, uint64_t stride, uint64_t seav_pad, uint32_t n_routers,
                     const sp_batch* desc, uint32_t n_batches, uint32_t* err, int threads, int grid, cudaStream_t s) {
  const size_t smem = ((size_t)n_batches + 1) * sizeof(uint64_t);
  switch (threads) {
    case 128:
      cudaFuncSetAttribute(k_scan_multi<LR, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_scan_multi<LR, 128><<<grid, 128, smem, s>>>(d, sketches, stride, seav_pad, n_routers, desc, n_batches, err);
      break;
    case 512:
      cudaFuncSetAttribute(k_scan_multi<LR, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_scan_multi<LR, 512><<<grid, 512, smem, s>>>(d, sketches, stride, seav_pad, n_routers, desc, n_batches, err);
      break;
    default:
      cudaFuncSetAttribute(k_scan_multi<LR, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_scan_multi<LR, 256><<<grid, 256, smem, s>>>(d, sketches, stride, seav_pad, n_routers, desc, n_batches, err);
      break;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_scan_multi(const DevParams& d, uint8_t* sketches, uint64_t stride, uint64_t seav_pad,
                              uint32_t n_routers, const sp_batch* desc, uint32_t n_batches, uint32_t* err,
                              int threads, int grid, cudaStream_t s) {
  if (n_batches == 0) return cudaSuccess;
  switch (d.lr) {
    case 1: return multi_lr<1>(d, sketches, stride, seav_pad, n_routers, desc, n_batches, err, threads, grid, s);
    case 2: return multi_lr<2>(d, sketches, stride, seav_pad, n_routers, desc, n_batches, err, threads, grid, s);
    case 3: return multi_lr<3>(d, sketches, stride, seav_pad, n_routers, desc, n_batches, err, threads, grid, s);
    case 4: return multi_lr<4>(d, sketches, stride, seav_pad, n_routers, desc, n_batches, err, threads, grid, s);
    case 5: return multi_lr<5>(d, sketches, stride, seav_pad, n_routers, desc, n_batches, err, threads, grid, s);
    case 6: return multi_lr<6>(d, sketches, stride, seav_pad, n_routers, desc, n_batches, err, threads, grid, s);
    case 7: return multi_lr<7>(d, sketches, stride, seav_pad, n_routers, desc, n_batches, err, threads, grid, s);
    default: return multi_lr<8>(d, sketches, stride, seav_pad, n_routers, desc, n_batches, err, threads, grid, s);
  }
}

int multi_max_grid(int threads) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  per_sm = 2048 / threads;
  return sms * per_sm;
}

int scan_grid(const DevParams& d) {
  switch (d.lr) {
    case 1: return grid_for<1>();
    case 2: return grid_for<2>();
    case 3: return grid_for<3>();
    case 4: return grid_for<4>();
    case 5: return grid_for<5>();
    case 6: return grid_for<6>();
    case 7: return grid_for<7>();
    default: return grid_for<8>();
  }
}

cudaError_t launch_scan(const DevParams& d, uint8_t* seav, uint32_t* ldca,
                        const uint32_t* pairs, uint64_t n_pairs, int grid, cudaStream_t s) {
  if (n_pairs == 0) return cudaSuccess;
  const uint64_t need = (n_pairs / 2 + kScanThreads - 1) / kScanThreads;
  if ((uint64_t)grid > need) grid = (int)(need > 0 ? need : 1);
  switch (d.lr) {
    case 1: k_scan<1><<<grid, kScanThreads, 0, s>>>(d, seav, ldca, pairs, n_pairs); break;
    case 2: k_scan<2><<<grid, kScanThreads, 0, s>>>(d, seav, ldca, pairs, n_pairs); break;
    case 3: k_scan<3><<<grid, kScanThreads, 0, s>>>(d, seav, ldca, pairs, n_pairs); break;
    case 4: k_scan<4><<<grid, kScanThreads, 0, s>>>(d, seav, ldca, pairs, n_pairs); break;
    case 5: k_scan<5><<<grid, kScanThreads, 0, s>>>(d, seav, ldca, pairs, n_pairs); break;
    case 6: k_scan<6><<<grid, kScanThreads, 0, s>>>(d, seav, ldca, pairs, n_pairs); break;
    case 7: k_scan<7><<<grid, kScanThreads, 0, s>>>(d, seav, ldca, pairs, n_pairs); break;
    default: k_scan<8><<<grid, kScanThreads, 0, s>>>(d, seav, ldca, pairs, n_pairs); break;
  }
  return cudaGetLastError();
}

}  // namespace sp
