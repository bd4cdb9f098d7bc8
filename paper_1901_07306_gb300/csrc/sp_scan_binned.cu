// sp_scan_binned.cu -- the per-pair scan with the LDCA updates moved from L2
// atomics to shared-memory atomics (Sec. 3.3 update, Sec. 4.1 scan).
//
// Every pair sets the same bit b = H3(oip) in its LR LDCs LH_i(hip).  Call
// "plane b" the set of bit b of every LDC: LR x LC bits (32 KiB at k = 1024,
// LR = 4, LC = 2^16).  A pair touches exactly one plane, so:
//
//  k_bin    (persistent, one 1024-thread block per SM) reads the pairs with
//           coalesced 8-byte loads, does the SEAV update of Sec. 3.1-3.2 for
//           sampled pairs (L2 RED, 1 pair in 2^tau), and counting-sorts each
//           16K-pair tile by b in shared memory; each bin's run of hips is
//           appended to the block's private list for that bin (no global
//           atomics; lists[b][block][0 .. cap)).  A run that would overflow a
//           list is applied directly with L2 REDs instead (any input is
//           correct; only a skewed one is slower).
//  k_apply  (one block per plane) starts the plane in shared memory from
//           zero (or from the router's pending plane when earlier updates of
//           the window have not been folded yet), sets bit (i, LH_i(hip)) for
//           every listed hip and row i with shared atomic OR, and stores the
//           plane back (the block owns it).
//  k_fold   (before the next detect, merge or export of the router) ORs the
//           plane-major accumulator into the LDCA's logical layout
//           [LR][LC][k / 32]: a warp loads word J of 32 consecutive planes and
//           a 5-stage butterfly of warp shuffles transposes the 32 x 32 bit
//           block, giving lane t the 32-bit word of LDC 32 J + t.
//
// Applicable when the bins are the LDC's k bit positions (k <= 4096) and one
// plane fits in shared memory as whole words (LC >= 32, LR x LC <= 2^20 bits).
#include <math.h>

#include "sp_internal.h"

namespace sp {

namespace {

constexpr int kBinThreads = 1024;
constexpr int kTile = 16384;                       // pairs per block iteration
constexpr int kPerThread = kTile / kBinThreads;    // 16
constexpr int kApplyThreads = 512;
constexpr uint32_t kFull = 0xFFFFFFFFu;

__device__ __forceinline__ void seav_set(const DevParams& d, uint8_t* seav, uint32_t hip, uint32_t h1) {
  const uint32_t bit = h1 >> 29;
  const uint32_t rp = d.r ? (hip & ((1u << d.r) - 1u)) : 0u;
  const uint32_t lp = (uint32_t)((uint64_t)hip >> d.r);
  const uint64_t base = (uint64_t)rp * d.sea_bytes;
  for (uint32_t i = 0; i < d.sr; ++i) {
    const uint64_t off = base + d.row_off[i] + gather_idx(lp, d.isb[i], d.ibn[i], d.L);
    atomicOr(reinterpret_cast<uint32_t*>(seav + (off & ~3ull)), (1u << bit) << (8u * (uint32_t)(off & 3u)));
  }
}

template <int LR>
__device__ __forceinline__ void ldca_red(const DevParams& d, uint32_t* ldca, uint32_t hip, uint32_t h3) {
  const uint32_t cshift = 32u - d.lc_log2;
  const uint32_t wshift = d.k_log2 - 5u;
#pragma unroll
  for (int i = 0; i < LR; ++i) {
    const uint32_t col = (uint32_t)((uint64_t)mas(d.ha[2 + i], d.hb[2 + i], hip) >> cshift);
    atomicOr(ldca + (((uint64_t)(((uint32_t)i << d.lc_log2) | col) << wshift) | (h3 >> 5)), 1u << (h3 & 31u));
  }
}

// Block-wide exclusive scan of n <= 4 * blockDim.x counters in shared memory.
__device__ void block_exclusive_scan(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* s_warp) {
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t per = (n + blockDim.x - 1) / blockDim.x;     // 1..4
  uint32_t v[4] = {0, 0, 0, 0}, sum = 0;
  for (uint32_t j = 0; j < per; ++j) {
    const uint32_t idx = tid * per + j;
    v[j] = idx < n ? in[idx] : 0u;
    sum += v[j];
  }
  uint32_t incl = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, o);
    if ((int)lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? s_warp[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, w, o);
      if ((int)lane >= o) w += y;
    }
    if (lane < nw) s_warp[lane] = w;            // inclusive warp totals
  }
  __syncthreads();
  uint32_t run = (warp ? s_warp[warp - 1] : 0u) + incl - sum;
  for (uint32_t j = 0; j < per; ++j) {
    const uint32_t idx = tid * per + j;
    if (idx < n) out[idx] = run;
    run += v[j];
  }
  __syncthreads();
}

template <int LR>
__global__ void __launch_bounds__(kBinThreads, 1)
k_bin(DevParams d, uint8_t* __restrict__ seav, uint32_t* __restrict__ ldca,
      const uint32_t* __restrict__ pairs, uint64_t n_pairs,
      uint32_t* __restrict__ lists, uint32_t* __restrict__ counts, uint32_t cap) {
  extern __shared__ uint32_t smem[];
  const uint32_t bins = 1u << d.k_log2;
  uint32_t* s_count = smem;                 // per-tile count, then kept count
  uint32_t* s_off = s_count + bins;         // per-tile exclusive offsets
  uint32_t* s_cursor = s_off + bins;        // this block's fill of each list
  uint32_t* s_sorted = s_cursor + bins;     // kTile hips sorted by bin
  __shared__ uint32_t s_warp[32];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t G = gridDim.x, cta = blockIdx.x;
  const uint32_t tau_mask = (1u << d.tau) - 1u;
  const uint32_t h3_shift = 32u - d.k_log2;
  for (uint32_t b = tid; b < bins; b += kBinThreads) { s_count[b] = 0; s_cursor[b] = 0; }
  __syncthreads();
  const uint64_t n_tiles = (n_pairs + kTile - 1) / kTile;
  const uint2* p2 = reinterpret_cast<const uint2*>(pairs);
  for (uint64_t tile = cta; tile < n_tiles; tile += G) {
    const uint64_t base = tile * kTile;
    uint32_t hip[kPerThread], key[kPerThread];      // key = bin << 14 | rank, ~0 = none
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
      const uint64_t p = base + (uint64_t)q * kBinThreads + tid;
      key[q] = kFull;
      hip[q] = 0;
      if (p < n_pairs) {
        const uint2 v = __ldcs(p2 + p);
        const uint32_t h1 = mas(d.ha[0], d.hb[0], v.y);
        if ((h1 & tau_mask) == 0u) seav_set(d, seav, v.x, h1);
        const uint32_t h3 = mas(d.ha[1], d.hb[1], v.y) >> h3_shift;
        hip[q] = v.x;
        key[q] = (h3 << 14) | atomicAdd(&s_count[h3], 1u);
      }
    }
    __syncthreads();
    block_exclusive_scan(s_count, s_off, bins, s_warp);
    // reserve room in this block's lists; clip at the list capacity
    for (uint32_t b = tid; b < bins; b += kBinThreads) {
      const uint32_t c = s_count[b], have = s_cursor[b];
      const uint32_t keep = have + c <= cap ? c : (cap - have);
      s_count[b] = keep;
      s_cursor[b] = have + keep;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
      if (key[q] != kFull) {
        const uint32_t b = key[q] >> 14, rank = key[q] & 0x3FFFu;
        if (rank < s_count[b]) s_sorted[s_off[b] + rank] = hip[q];
        else ldca_red<LR>(d, ldca, hip[q], b);          // list full: apply in L2
      }
    }
    __syncthreads();
    // append each bin's run to list (b, cta), one warp per bin
    for (uint32_t b = warp; b < bins; b += kBinThreads / 32) {
      const uint32_t keep = s_count[b];
      if (keep == 0) continue;
      uint32_t* dst = lists + ((uint64_t)b * G + cta) * cap + (s_cursor[b] - keep);
      const uint32_t* src = s_sorted + s_off[b];
      for (uint32_t i = lane; i < keep; i += 32) dst[i] = src[i];
    }
    __syncthreads();
    for (uint32_t b = tid; b < bins; b += kBinThreads) s_count[b] = 0;
    __syncthreads();
  }
  for (uint32_t b = tid; b < bins; b += kBinThreads) counts[(uint64_t)b * G + cta] = s_cursor[b];
}

template <int LR>
__global__ void __launch_bounds__(kApplyThreads)
k_apply(DevParams d, const uint32_t* __restrict__ lists, const uint32_t* __restrict__ counts,
        uint32_t G, uint32_t cap, uint32_t* __restrict__ planes, bool accumulate) {
  extern __shared__ uint32_t s_plane[];
  const uint32_t b = blockIdx.x;
  const uint32_t words = ((uint32_t)LR << d.lc_log2) >> 5;       // plane words
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t nwarps = kApplyThreads / 32;
  const uint32_t cshift = 32u - d.lc_log2;
  uint32_t* dst = planes + (uint64_t)b * words;
  for (uint32_t w = tid; w < words; w += kApplyThreads) s_plane[w] = accumulate ? dst[w] : 0u;
  __syncthreads();
  for (uint32_t c = warp; c < G; c += nwarps) {
    const uint32_t n = counts[(uint64_t)b * G + c];
    const uint32_t* src = lists + ((uint64_t)b * G + c) * cap;
    for (uint32_t i = lane; i < n; i += 32) {
      const uint32_t hip = __ldcs(src + i);
#pragma unroll
      for (int r = 0; r < LR; ++r) {
        const uint32_t col = (uint32_t)((uint64_t)mas(d.ha[2 + r], d.hb[2 + r], hip) >> cshift);
        const uint32_t bit = ((uint32_t)r << d.lc_log2) | col;
        atomicOr(&s_plane[bit >> 5], 1u << (bit & 31u));
      }
    }
  }
  __syncthreads();
  for (uint32_t w = tid; w < words; w += kApplyThreads) dst[w] = s_plane[w];
}

// 32 x 32 bit transpose across a warp: lane l holds row l (bit j = column j);
// afterwards lane l holds column l (bit p = row p's bit l).
__device__ __forceinline__ uint32_t transpose32(uint32_t x, uint32_t lane) {
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const uint32_t s = 16u >> st, m = masks[st];
    const uint32_t y = __shfl_xor_sync(kFull, x, s);
    x = (lane & s) ? (((y >> s) & m) | (x & ~m)) : ((x & m) | ((y & m) << s));
  }
  return x;
}

// planes: [k][W] words (W = LR * LC / 32); ldca: [LR * LC][k / 32] words.
__global__ void __launch_bounds__(256)
k_fold(const uint32_t* __restrict__ planes, uint32_t* __restrict__ ldca, uint32_t W, uint32_t k_log2) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t wpl = 1u << (k_log2 - 5u);                       // words per LDC
  const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarp = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t J = gwarp; J < W; J += nwarp) {
    uint32_t* line = ldca + ((uint64_t)J * 32u + lane) * wpl;     // LDC 32 J + lane
    for (uint32_t q0 = 0; q0 < wpl; q0 += 4) {
      uint32_t acc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t q = q0 + u;
        const uint32_t x = q < wpl ? planes[((uint64_t)(q * 32u + lane)) * W + J] : 0u;
        acc[u] = transpose32(x, lane);
      }
      if (wpl >= 4) {
        uint4 o = *reinterpret_cast<uint4*>(line + q0);
        o.x |= acc[0]; o.y |= acc[1]; o.z |= acc[2]; o.w |= acc[3];
        *reinterpret_cast<uint4*>(line + q0) = o;
      } else {
        for (uint32_t u = 0; u < wpl; ++u) line[q0 + u] |= acc[u];
      }
    }
  }
}

template <int LR>
cudaError_t run_binned(const DevParams& d, uint8_t* seav, uint32_t* ldca, const uint32_t* pairs,
                       uint64_t n_pairs, const BinnedScratch& s, cudaStream_t st) {
  const uint32_t bins = 1u << d.k_log2;
  const size_t bin_smem = (size_t)(3u * bins + kTile) * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(k_bin<LR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bin_smem);
  if (e != cudaSuccess) return e;
  const uint32_t words = ((uint32_t)LR << d.lc_log2) >> 5;
  const size_t apply_smem = (size_t)words * sizeof(uint32_t);
  e = cudaFuncSetAttribute(k_apply<LR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)apply_smem);
  if (e != cudaSuccess) return e;
  uint64_t done = 0;
  bool accumulate = s.accumulate;
  while (done < n_pairs) {
    const uint64_t n = (n_pairs - done) < s.max_pairs ? (n_pairs - done) : s.max_pairs;
    const uint32_t cap = binned_list_cap(n, bins, s.ctas);
    k_bin<LR><<<s.ctas, kBinThreads, bin_smem, st>>>(d, seav, ldca, pairs + 2 * done, n, s.lists, s.counts, cap);
    k_apply<LR><<<bins, kApplyThreads, apply_smem, st>>>(d, s.lists, s.counts, s.ctas, cap, s.planes, accumulate);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    accumulate = true;
    done += n;
  }
  return cudaSuccess;
}

}  // namespace

bool binned_applicable(const DevParams& d) {
  const uint64_t plane_bits = (uint64_t)d.lr << d.lc_log2;
  return d.k_log2 >= 5 && d.k_log2 <= 12 && d.lc_log2 >= 5 && plane_bits <= (1ull << 20);
}

uint32_t binned_list_cap(uint64_t n_pairs, uint32_t bins, uint32_t ctas) {
  const double m = (double)n_pairs / ((double)bins * ctas);
  uint64_t cap = (uint64_t)(m + 8.0 * sqrt(m + 1.0) + 32.0);
  cap = (cap + 7) & ~7ull;                                   // 32-byte list starts
  return (uint32_t)cap;
}

int binned_ctas() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

int binned_fold_grid() {
  return binned_ctas() * 8;
}

cudaError_t launch_fold(const DevParams& d, const uint32_t* planes, uint32_t* ldca, int grid, cudaStream_t st) {
  const uint32_t words = (uint32_t)(((uint64_t)d.lr << d.lc_log2) >> 5);
  k_fold<<<grid, 256, 0, st>>>(planes, ldca, words, d.k_log2);
  return cudaGetLastError();
}

cudaError_t launch_scan_binned(const DevParams& d, uint8_t* seav, uint32_t* ldca, const uint32_t* pairs,
                               uint64_t n_pairs, const BinnedScratch& s, cudaStream_t st) {
  if (n_pairs == 0) return cudaSuccess;
  switch (d.lr) {
    case 1: return run_binned<1>(d, seav, ldca, pairs, n_pairs, s, st);
    case 2: return run_binned<2>(d, seav, ldca, pairs, n_pairs, s, st);
    case 3: return run_binned<3>(d, seav, ldca, pairs, n_pairs, s, st);
    case 4: return run_binned<4>(d, seav, ldca, pairs, n_pairs, s, st);
    case 5: return run_binned<5>(d, seav, ldca, pairs, n_pairs, s, st);
    case 6: return run_binned<6>(d, seav, ldca, pairs, n_pairs, s, st);
    case 7: return run_binned<7>(d, seav, ldca, pairs, n_pairs, s, st);
    default: return run_binned<8>(d, seav, ldca, pairs, n_pairs, s, st);
  }
}

}  // namespace sp
