// sp_scan_binned.cu -- the per-pair scan with the LDCA updates moved from L2
// atomics to shared-memory atomics (Sec. 3.3 update, Sec. 4.1 scan).
//
// Every pair sets the same bit b = H3(oip) in its LR LDCs LH_i(hip).  Call
// "plane b" the set of bit b of every LDC: LR x LC bits (32 KiB at k = 1024,
// LR = 4, LC = 2^16).  A pair touches exactly one plane, so:
//
//  k_bin    (persistent, one 1024-thread block per SM) streams 8K-pair tiles
//           into shared memory with TMA bulk copies, double buffered (the next
//           tile lands while this one is sorted; waits on the mbarrier are
//           bounded and end in an error flag), does the SEAV update of
//           Sec. 3.1-3.2 for sampled pairs (L2 RED, 1 pair in 2^tau), and
//           counting-sorts each tile by b in shared memory; each bin's run of
//           hips is appended to the block's private list for that bin, one
//           thread per sorted position (no global atomics;
//           lists[b][block][0 .. cap)).  A run that would overflow a list is
//           applied directly with L2 REDs instead (any input is correct; only
//           a skewed one is slower).
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
// Applicable when the bins are the LDC's k bit positions (k <= 1024) and one
// plane fits in shared memory as whole words (LC >= 32, LR x LC <= 2^20 bits).
#include <math.h>

#include "sp_internal.h"

namespace sp {

namespace {

constexpr int kBinThreads = 1024;
constexpr int kTile = 8192;                        // pairs per block iteration
constexpr int kPerThread = kTile / kBinThreads;    // 8
constexpr int kQueue = 1024;                       // sampled pairs queued per tile
constexpr int kApplyThreads = 512;
constexpr int kApplyUnroll = 8;                    // hip loads in flight per lane
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

// ---- TMA 1D bulk copies into shared memory, completed on an mbarrier ------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One thread: arm the barrier for `bytes` and start the copy (16-byte aligned
// source and destination, bytes a multiple of 16).
__device__ __forceinline__ void tma_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               :: "r"(smem_addr(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

// Bounded wait for the barrier phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_addr(bar);
  for (uint32_t it = 0; it < (1u << 20); ++it) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(addr), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// k_bin: tiles of kTile pairs, tile (cta + i G) in iteration i.  Thread 0
// prefetches tile i + 1 into the other raw buffer with one TMA bulk copy while
// the block sorts tile i.  Tiles that are partial, or a stream that is not
// 16-byte aligned, are read with plain loads instead.  Per tile:
//   1. every thread hashes its 8 pairs, counts each pair's bin with a shared
//      atomic (the count before it is the pair's rank in the bin) and queues
//      the sampled pairs (Sec. 3.1) for a converged SEAV pass;
//   2. one thread per bin: exclusive prefix of the counts (warp shuffles plus
//      one warp over the 32 warp totals), room in the bin's list, the bin's
//      64-bit record (tile offset | kept << 14, first list slot), count reset;
//   3. every pair goes to its sorted position with its list slot, and the
//      queued pairs set their SEAV bits;
//   4. one thread per sorted position writes the hip: consecutive positions of
//      a bin land in consecutive list slots.
template <int LR>
__global__ void __launch_bounds__(kBinThreads, 1)
k_bin(DevParams d, uint8_t* __restrict__ seav, uint32_t* __restrict__ ldca,
      BinSrc src, uint32_t* __restrict__ lists, uint32_t* __restrict__ counts, uint32_t cap,
      uint32_t* __restrict__ error, bool append, uint32_t rot) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  const uint32_t bins = 1u << d.k_log2;                                // <= kBinThreads
  uint2* raw = reinterpret_cast<uint2*>(smem_raw);                     // [2][kTile]
  uint2* s_entry = raw + 2 * kTile;                                     // [kTile] (hip, list slot or ~0)
  uint2* s_meta = s_entry + kTile;                                      // [bins] (offset | kept << 14, slot)
  uint2* s_queue = s_meta + bins;                                       // [kQueue] sampled (hip, h1)
  uint32_t* s_count = reinterpret_cast<uint32_t*>(s_queue + kQueue);    // [bins]
  uint32_t* s_cursor = s_count + bins;                                  // [bins] list fill
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_qn;
  __shared__ __align__(8) uint64_t s_bar[2];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t G = gridDim.x, cta = blockIdx.x;
  const uint32_t slot = (cta + rot) % G;          // which tiles this block takes
  const uint32_t tau_mask = (1u << d.tau) - 1u;
  const uint32_t h3_shift = 32u - d.k_log2;
  // tiles of the streams, back to back: stream b owns tiles [s_tpref[b], s_tpref[b + 1])
  __shared__ uint64_t s_tpref[kBinMaxSrc + 1];
  if (tid == 0) {
    uint64_t acc = 0;
    s_tpref[0] = 0;
    for (uint32_t b = 0; b < src.count; ++b) {
      acc += (src.n[b] + kTile - 1) / kTile;
      s_tpref[b + 1] = acc;
    }
    s_qn = 0;
  }
  // appending continues this block's lists from an earlier chunk of the round
  if (tid < bins) {
    s_count[tid] = 0;
    s_cursor[tid] = append ? counts[(uint64_t)tid * G + cta] : 0u;
  }
  if (tid == 0) { mbar_init(&s_bar[0]); mbar_init(&s_bar[1]); }
  __syncthreads();
  const uint64_t n_tiles = s_tpref[src.count];
  auto stream_of = [&](uint64_t tile) {       // the b with s_tpref[b] <= tile < s_tpref[b + 1]
    uint32_t b = 0;
    while (s_tpref[b + 1] <= tile) ++b;
    return b;
  };
  // tile of iteration i, and whether it comes through TMA
  auto tile_of = [&](uint64_t i) { return (uint64_t)slot + i * G; };
  auto by_tma = [&](uint64_t tile) {           // a whole tile of a 16-byte aligned stream
    const uint32_t b = stream_of(tile);
    const uint64_t local = tile - s_tpref[b];
    return ((uintptr_t)src.ptr[b] & 15u) == 0 && (local + 1) * kTile <= src.n[b];
  };
  auto tile_ptr = [&](uint64_t tile) {
    const uint32_t b = stream_of(tile);
    return reinterpret_cast<const uint2*>(src.ptr[b]) + (tile - s_tpref[b]) * kTile;
  };
  uint32_t phases = 0u;                          // bit b: parity of barrier b's next phase
  if (tid == 0 && tile_of(0) < n_tiles && by_tma(tile_of(0)))
    tma_load(raw, tile_ptr(tile_of(0)), kTile * 8u, &s_bar[0]);
  for (uint64_t i = 0; tile_of(i) < n_tiles; ++i) {
    const uint64_t tile = tile_of(i);
    const uint32_t buf = (uint32_t)(i & 1u);
    // prefetch the next tile into the other buffer (freed at the end of i - 1)
    const uint64_t next = tile_of(i + 1);
    if (tid == 0 && next < n_tiles && by_tma(next))
      tma_load(raw + (buf ^ 1u) * kTile, tile_ptr(next), kTile * 8u, &s_bar[buf ^ 1u]);
    const uint32_t sb = stream_of(tile);
    const uint64_t base = (tile - s_tpref[sb]) * kTile;                 // within stream sb
    const bool full = ((uintptr_t)src.ptr[sb] & 15u) == 0 && base + kTile <= src.n[sb];
    if (full) {
      const bool ok = __syncthreads_and(mbar_wait(&s_bar[buf], (phases >> buf) & 1u));
      phases ^= 1u << buf;
      if (!ok) {
        // give up: flag the error, let this block's copies in flight land
        // (bounded again), publish empty lists and leave
        if (tid == 0) {
          atomicOr(error, 1u);
          mbar_wait(&s_bar[buf], ((phases >> buf) & 1u) ^ 1u);
          if (next < n_tiles && by_tma(next)) mbar_wait(&s_bar[buf ^ 1u], (phases >> (buf ^ 1u)) & 1u);
        }
        if (tid < bins) counts[(uint64_t)tid * G + cta] = s_cursor[tid];
        return;
      }
    }
    const uint32_t tile_n = (uint32_t)((src.n[sb] - base) < (uint64_t)kTile ? (src.n[sb] - base) : kTile);
    const uint2* p2 = reinterpret_cast<const uint2*>(src.ptr[sb]);
    // 1. hash, count, queue the sampled pairs
    uint32_t hip[kPerThread], key[kPerThread];      // key = bin << 14 | rank, ~0 = none
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
      const uint32_t j = (uint32_t)q * kBinThreads + tid;
      const bool valid = j < tile_n;
      uint2 v = make_uint2(0u, 0u);
      if (valid) v = full ? raw[buf * kTile + j] : __ldcs(p2 + base + j);
      const uint32_t h1 = mas(d.ha[0], d.hb[0], v.y);
      const bool sampled = valid && (h1 & tau_mask) == 0u;
      // warp-aggregated push: one shared atomic per warp and round
      const uint32_t ballot = __ballot_sync(kFull, sampled);
      if (ballot) {
        uint32_t first = 0;
        if (lane == 0) first = atomicAdd(&s_qn, (uint32_t)__popc(ballot));
        first = __shfl_sync(kFull, first, 0);
        if (sampled) {
          const uint32_t at = first + (uint32_t)__popc(ballot & ((1u << lane) - 1u));
          if (at < (uint32_t)kQueue) s_queue[at] = make_uint2(v.x, h1);
          else seav_set(d, seav, v.x, h1);          // a queue overflow (small tau) sets the bits here
        }
      }
      const uint32_t h3 = mas(d.ha[1], d.hb[1], v.y) >> h3_shift;
      hip[q] = v.x;
      key[q] = valid ? ((h3 << 14) | atomicAdd(&s_count[h3], 1u)) : kFull;
    }
    __syncthreads();
    // 2. per bin: prefix of the counts, room in the list, record, reset
    const uint32_t qn = s_qn < (uint32_t)kQueue ? s_qn : (uint32_t)kQueue;
    const uint32_t c = tid < bins ? s_count[tid] : 0u;
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if ((int)lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = s_warp[lane];                   // 32 warps of 32 threads
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, w, o);
        if ((int)lane >= o) w += y;
      }
      s_warp[lane] = w;                            // inclusive warp totals
      if (lane == 0) s_qn = 0;                     // every thread has read it
    }
    __syncthreads();
    if (tid < bins) {
      const uint32_t off = (warp ? s_warp[warp - 1] : 0u) + incl - c;
      const uint32_t have = s_cursor[tid];
      const uint32_t keep = have + c <= cap ? c : (cap - have);
      // offset and kept count (both <= kTile < 2^14) and the first free list
      // slot (list entries < 2^32, a host check): one 64-bit lookup below
      s_meta[tid] = make_uint2(off | (keep << 14), (tid * G + cta) * cap + have);
      s_cursor[tid] = have + keep;
      s_count[tid] = 0;
    }
    __syncthreads();
    // 3. sorted positions with their list slots; the queued SEAV updates
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
      if (key[q] != kFull) {
        const uint32_t b = key[q] >> 14, rank = key[q] & 0x3FFFu;
        // every position of the tile gets (hip, list slot), the slot ~0 when
        // the list is full (then the pair is applied in L2 right here)
        const uint2 m = s_meta[b];
        const bool kept = rank < (m.x >> 14);
        s_entry[(m.x & 0x3FFFu) + rank] = make_uint2(hip[q], kept ? m.y + rank : kFull);
        if (!kept) ldca_red<LR>(d, ldca, hip[q], b);
      }
    }
    for (uint32_t e = tid; e < qn; e += kBinThreads) {
      const uint2 x = s_queue[e];
      seav_set(d, seav, x.x, x.y);
    }
    __syncthreads();
    // 4. one thread per sorted position: consecutive positions of a bin go to
    // consecutive list slots
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
      const uint32_t j = (uint32_t)q * kBinThreads + tid;
      if (j < tile_n) {
        const uint2 e = s_entry[j];
        if (e.y != kFull) lists[e.y] = e.x;
      }
    }
    // no barrier here: the next tile writes s_entry (step 3) only after the
    // barriers of its steps 1 and 2, which every thread reaches after this step
  }
  if (tid < bins) counts[(uint64_t)tid * G + cta] = s_cursor[tid];
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
    for (uint32_t i0 = 0; i0 < n; i0 += 32 * kApplyUnroll) {
      uint32_t hip[kApplyUnroll];
#pragma unroll
      for (int u = 0; u < kApplyUnroll; ++u) {          // all loads first: kApplyUnroll in flight
        const uint32_t i = i0 + (uint32_t)u * 32 + lane;
        hip[u] = i < n ? __ldcs(src + i) : 0u;
      }
#pragma unroll
      for (int u = 0; u < kApplyUnroll; ++u) {
        if (i0 + (uint32_t)u * 32 + lane < n) {
#pragma unroll
          for (int r = 0; r < LR; ++r) {
            const uint32_t col = (uint32_t)((uint64_t)mas(d.ha[2 + r], d.hb[2 + r], hip[u]) >> cshift);
            const uint32_t bit = ((uint32_t)r << d.lc_log2) | col;
            atomicOr(&s_plane[bit >> 5], 1u << (bit & 31u));
          }
        }
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
// A warp task is 8 consecutive plane words J0 .. J0 + 7 (one 32-byte sector
// of each plane it reads) times 4 consecutive LDC words: it transposes
// 32 planes x 32 LDCs per word and ORs the result into the lanes' LDC lines.
__global__ void __launch_bounds__(256)
k_fold(const uint32_t* __restrict__ planes, uint32_t* __restrict__ ldca, uint32_t W, uint32_t k_log2) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t wpl = 1u << (k_log2 - 5u);                       // words per LDC
  const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarp = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const bool vec = (W & 7u) == 0 && wpl >= 4;
  const uint64_t n_groups = (W + 7) / 8;
  const uint32_t n_q = (wpl + 3) / 4;                              // groups of 4 LDC words
  for (uint64_t t = gwarp; t < n_groups * n_q; t += nwarp) {
    const uint64_t g = t / n_q;
    const uint32_t J0 = (uint32_t)(g * 8);
    const uint32_t nj = (W - J0) < 8u ? (W - J0) : 8u;
    {
      const uint32_t q0 = (uint32_t)(t % n_q) * 4u;
      uint32_t x[4][8];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t q = q0 + u;
        const uint32_t* row = planes + (uint64_t)(q * 32u + lane) * W + J0;
        if (vec) {
          const uint4 a = *reinterpret_cast<const uint4*>(row);
          const uint4 c = *reinterpret_cast<const uint4*>(row + 4);
          x[u][0] = a.x; x[u][1] = a.y; x[u][2] = a.z; x[u][3] = a.w;
          x[u][4] = c.x; x[u][5] = c.y; x[u][6] = c.z; x[u][7] = c.w;
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) x[u][j] = (q < wpl && (uint32_t)j < nj) ? row[j] : 0u;
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if ((uint32_t)j >= nj) break;
        uint32_t acc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = transpose32(x[u][j], lane);
        uint32_t* line = ldca + ((uint64_t)(J0 + j) * 32u + lane) * wpl;
        if (wpl >= 4) {
          uint4 o = *reinterpret_cast<uint4*>(line + q0);
          o.x |= acc[0]; o.y |= acc[1]; o.z |= acc[2]; o.w |= acc[3];
          *reinterpret_cast<uint4*>(line + q0) = o;
        } else {
          for (uint32_t u = 0; u < wpl; ++u) line[u] |= acc[u];
        }
      }
    }
  }
}

template <int LR>
cudaError_t bin_chunk(const DevParams& d, uint8_t* seav, uint32_t* ldca, const BinSrc& src,
                      const BinnedScratch& s, uint32_t cap, bool append, uint32_t rot, cudaStream_t st) {
  const uint32_t bins = 1u << d.k_log2;
  // raw[2][kTile] pairs, (hip, slot) entries, a 64-bit record and 2 counters
  // per bin, the sampled-pair queue
  const size_t bin_smem = (size_t)2 * kTile * 8 + (size_t)kTile * 8 + (size_t)bins * 16 + (size_t)kQueue * 8;
  cudaError_t e = cudaFuncSetAttribute(k_bin<LR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bin_smem);
  if (e != cudaSuccess) return e;
  k_bin<LR><<<s.ctas, kBinThreads, bin_smem, st>>>(d, seav, ldca, src, s.lists, s.counts, cap, s.error,
                                                   append, rot);
  return cudaGetLastError();
}

template <int LR>
cudaError_t apply_round(const DevParams& d, const BinnedScratch& s, uint32_t cap, bool accumulate, cudaStream_t st) {
  const uint32_t bins = 1u << d.k_log2;
  const uint32_t words = ((uint32_t)LR << d.lc_log2) >> 5;
  const size_t apply_smem = (size_t)words * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(k_apply<LR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)apply_smem);
  if (e != cudaSuccess) return e;
  k_apply<LR><<<bins, kApplyThreads, apply_smem, st>>>(d, s.lists, s.counts, s.ctas, cap, s.planes, accumulate);
  return cudaGetLastError();
}

}  // namespace

bool binned_applicable(const DevParams& d) {
  const uint64_t plane_bits = (uint64_t)d.lr << d.lc_log2;
  return d.k_log2 >= 5 && d.k_log2 <= 10 && d.lc_log2 >= 5 && plane_bits <= (1ull << 20);
}

// List capacity for a round of n_pairs split into `chunks` binning launches:
// a block takes at most ceil(tiles / ctas) + 1 tiles per launch (the tile to
// block mapping rotates between launches), spread over the bins; 8 standard
// deviations plus 32 of headroom, so that only skewed inputs overflow.
uint32_t binned_list_cap(uint64_t n_pairs, uint32_t bins, uint32_t ctas, uint32_t chunks) {
  const uint64_t tiles = (n_pairs + kTile - 1) / kTile;
  const uint64_t per_cta = (tiles + ctas - 1) / ctas + (chunks > 1 ? chunks : 1);
  const double m = (double)(per_cta * kTile < n_pairs ? per_cta * kTile : n_pairs) / bins;
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

BinSrc bin_src_one(const uint32_t* pairs, uint64_t n_pairs) {
  BinSrc src{};
  src.ptr[0] = pairs;
  src.n[0] = n_pairs;
  src.count = 1;
  return src;
}

cudaError_t binned_bin_chunk(const DevParams& d, uint8_t* seav, uint32_t* ldca, const BinSrc& src,
                             const BinnedScratch& s, uint32_t cap, bool append, uint32_t rot, cudaStream_t st) {
  if (src.count == 0) return cudaSuccess;
  switch (d.lr) {
    case 1: return bin_chunk<1>(d, seav, ldca, src, s, cap, append, rot, st);
    case 2: return bin_chunk<2>(d, seav, ldca, src, s, cap, append, rot, st);
    case 3: return bin_chunk<3>(d, seav, ldca, src, s, cap, append, rot, st);
    case 4: return bin_chunk<4>(d, seav, ldca, src, s, cap, append, rot, st);
    case 5: return bin_chunk<5>(d, seav, ldca, src, s, cap, append, rot, st);
    case 6: return bin_chunk<6>(d, seav, ldca, src, s, cap, append, rot, st);
    case 7: return bin_chunk<7>(d, seav, ldca, src, s, cap, append, rot, st);
    default: return bin_chunk<8>(d, seav, ldca, src, s, cap, append, rot, st);
  }
}

cudaError_t binned_apply_round(const DevParams& d, const BinnedScratch& s, uint32_t cap, bool accumulate,
                               cudaStream_t st) {
  switch (d.lr) {
    case 1: return apply_round<1>(d, s, cap, accumulate, st);
    case 2: return apply_round<2>(d, s, cap, accumulate, st);
    case 3: return apply_round<3>(d, s, cap, accumulate, st);
    case 4: return apply_round<4>(d, s, cap, accumulate, st);
    case 5: return apply_round<5>(d, s, cap, accumulate, st);
    case 6: return apply_round<6>(d, s, cap, accumulate, st);
    case 7: return apply_round<7>(d, s, cap, accumulate, st);
    default: return apply_round<8>(d, s, cap, accumulate, st);
  }
}

uint32_t binned_tile_pairs() { return (uint32_t)kTile; }

cudaError_t launch_scan_binned(const DevParams& d, uint8_t* seav, uint32_t* ldca, const uint32_t* pairs,
                               uint64_t n_pairs, const BinnedScratch& s, cudaStream_t st) {
  uint64_t done = 0;
  bool accumulate = s.accumulate;
  while (done < n_pairs) {
    const uint64_t n = (n_pairs - done) < s.max_pairs ? (n_pairs - done) : s.max_pairs;
    const uint32_t cap = binned_list_cap(n, 1u << d.k_log2, s.ctas, 1);
    cudaError_t e = binned_bin_chunk(d, seav, ldca, bin_src_one(pairs + 2 * done, n), s, cap, false, 0, st);
    if (e == cudaSuccess) e = binned_apply_round(d, s, cap, accumulate, st);
    if (e != cudaSuccess) return e;
    accumulate = true;
    done += n;
  }
  return cudaSuccess;
}

}  // namespace sp
