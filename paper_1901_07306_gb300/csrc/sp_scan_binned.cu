// sp_scan_binned.cu -- the per-pair scan with the LDCA updates moved from L2
// atomics to shared-memory atomics (Sec. 3.3 update, Sec. 4.1 scan).
//
// Every pair sets the same bit b = H3(oip) in its LR LDCs LH_i(hip).  Call
// "plane b" the set of bit b of every LDC: LR x LC bits (32 KiB at k = 1024,
// LR = 4, LC = 2^16).  A pair touches exactly one plane, so:
//
//  k_bin    (persistent, one or two blocks per SM, shapes below) streams tiles
//           with 16-byte loads held in registers (the next tile's loads are
//           issued before the current tile's work), does the SEAV update of
//           Sec. 3.1-3.2 for sampled pairs (L2 RED, 1 pair in 2^tau), and
//           stages each hip in a shared-memory row of its bin b; a row's whole
//           8-hip chunks go to the block's private list for that bin with one
//           32-byte store each (no global atomics; lists[b][block][0 .. cap)).
//           A row or a list that is full sends its hips to L2 REDs instead
//           (any input is correct; only a skewed one is slower).
//  k_apply  (one block per plane) starts the plane in shared memory from
//           zero (or from the router's pending plane when earlier updates of
//           the window have not been folded yet), sets bit (i, LH_i(hip)) for
//           every listed hip and row i with shared atomic OR, and stores the
//           plane back (the block owns it).
//  k_fold   (before the next detect, merge or export of the router) ORs the
//           plane accumulator into the LDCA's logical layout
//           [LR][LC][k / 32]: a warp loads word J of 32 consecutive planes and
//           a 5-stage butterfly of warp shuffles transposes the 32 x 32 bit
//           block, giving lane t the 32-bit word of LDC 32 J + t.
//
// Applicable when the bins are the LDC's k bit positions (k <= 1024) and one
// plane fits in shared memory as whole words (LC >= 32, LR x LC <= 2^20 bits).
//
// Staging shapes (the autotuner picks one per context; every shape gives the
// same bits):  k_bin block size, staging row length, tiles per flush round
// and blocks per SM -- a 1024-thread block with 44-hip rows flushing every two
// tiles, or two 512-thread blocks per SM with 20-hip rows flushing every tile,
// so one block's flush overlaps the other's hashing -- and the k_apply block
// size.
#include <math.h>

#include "sp_internal.h"

namespace sp {

namespace {

constexpr int kVec = 4;                            // 16-byte loads (2 pairs) per thread and tile
constexpr int kGroup = 4;                          // pairs hashed and staged together
constexpr int kChunk = 8;                          // hips per list store (32 bytes)
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

// One L2 RED per LDCA row: the rare overflow path of k_bin (a full staging
// row or list), so the row count is read at run time.
__device__ __forceinline__ void ldca_red(const DevParams& d, uint32_t* ldca, uint32_t hip, uint32_t h3) {
  const uint32_t cshift = 32u - d.lc_log2;
  const uint32_t wshift = d.k_log2 - 5u;
#pragma unroll
  for (uint32_t i = 0; i < 8; ++i) {               // constant indices into the parameter block
    if (i < d.lr) {
      const uint32_t col = (uint32_t)((uint64_t)mas(d.ha[2 + i], d.hb[2 + i], hip) >> cshift);
      atomicOr(ldca + (((uint64_t)((i << d.lc_log2) | col) << wshift) | (h3 >> 5)), 1u << (h3 & 31u));
    }
  }
}

// 256-bit store of 8 hips (a 32-byte aligned list chunk, one full sector).
__device__ __forceinline__ void st_chunk(uint32_t* dst, uint4 a, uint4 b) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
               :: "l"(dst), "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
               : "memory");
}

// k_bin: tiles of TILE = THREADS * 2 kVec pairs, tile (slot + i G) in iteration i.  Each
// thread holds kVec 16-byte loads (2 pairs each) of a tile in registers and
// issues the loads of tile i + 1 before it works on tile i, so the copy from
// HBM overlaps the work.  Tiles that are partial, or a stream that is not
// 16-byte aligned, are read pair by pair instead.  Every bin owns a staging
// row of STAGE hips in shared memory that persists across tiles (a
// write-combining buffer for the bin's list).  Per tile:
//   1. every thread hashes its pairs, queues the sampled pairs (Sec. 3.1) for
//      a converged SEAV pass, takes a place in its pair's bin row with one
//      shared atomic and stores the hip there (a row that is full sends the
//      pair to L2 REDs instead);
//   2. (after every TPR tiles) each thread takes bins tid, tid + THREADS, ...:
//      it moves the row's whole 8-hip chunks to the bin's list with 32-byte
//      stores and keeps the remainder (< 8 hips) at the front of the row; the
//      queued pairs set their SEAV bits, taken by consecutive threads.
// At the end the remainders go to the lists with plain stores; an appending
// launch first takes the tail of a list that is not a whole chunk back into
// the row, so lists stay dense and chunk stores stay 32-byte aligned.
template <int THREADS, int STAGE, int TPR, int PER_SM>
__global__ void __launch_bounds__(THREADS, PER_SM)
k_bin(DevParams d, uint8_t* __restrict__ seav, uint32_t* __restrict__ ldca,
      BinSrc src, uint32_t* __restrict__ lists, uint32_t* __restrict__ counts, uint32_t cap,
      bool append, uint32_t rot, uint32_t* __restrict__ ovf) {
  constexpr int TILE = THREADS * kVec * 2;
  constexpr int QUEUE = TPR * TILE / 32;              // sampled pairs per round: 4x the expected 2^-7
  extern __shared__ __align__(128) uint8_t smem_raw[];
  const uint32_t bins = 1u << d.k_log2;                                // <= 1024
  uint32_t* stage = reinterpret_cast<uint32_t*>(smem_raw);             // [bins][STAGE], then a 32-word sink
  uint32_t* sink = stage + bins * STAGE;                                // stores of pairs a full row refused
  uint2* s_queue = reinterpret_cast<uint2*>(sink + 32);               // [QUEUE] sampled (hip, h1)
  uint32_t* s_fill = reinterpret_cast<uint32_t*>(s_queue + QUEUE);     // [bins] hips in the row
  uint32_t* s_cursor = s_fill + bins;                                   // [bins] list fill (whole chunks)
  __shared__ uint32_t s_qn[2];                                          // queue fill, by tile parity
  __shared__ uint64_t s_tpref[kBinMaxSrc + 1];
  const uint32_t tid = threadIdx.x;
  const uint32_t G = gridDim.x, cta = blockIdx.x;
  const uint32_t slot = (cta + rot) % G;          // which tiles this block takes
  const uint32_t tau_mask = (1u << d.tau) - 1u;
  const uint32_t h3_shift = 32u - d.k_log2;
  const uint32_t lane = tid & 31u;
  uint32_t lt_mask;                                // lanes below this one
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt_mask));
  // a hip whose row or list was full: its LDCA bits go straight to L2, and
  // the router's flag tells the fold that the LDCA is no longer all zero
  auto spill = [&](uint32_t hip, uint32_t b) {
    ldca_red(d, ldca, hip, b);
    if (ovf) *ovf = 1u;
  };
  // tiles of the streams, back to back: stream b owns tiles [s_tpref[b], s_tpref[b + 1])
  if (tid == 0) {
    uint64_t acc = 0;
    s_tpref[0] = 0;
    for (uint32_t b = 0; b < src.count; ++b) {
      acc += (src.n[b] + TILE - 1) / TILE;
      s_tpref[b + 1] = acc;
    }
    s_qn[0] = s_qn[1] = 0;
  }
  auto list_of = [&](uint32_t b) { return lists + ((uint64_t)b * G + cta) * cap; };
  for (uint32_t b = tid; b < bins; b += THREADS) {
    // an appending launch continues the list: its partial chunk returns to the row
    const uint32_t have = append ? counts[(uint64_t)b * G + cta] : 0u;
    const uint32_t tail = have & (kChunk - 1u);
    for (uint32_t e = 0; e < tail; ++e) stage[b * STAGE + e] = list_of(b)[have - tail + e];
    s_fill[b] = tail;
    s_cursor[b] = have - tail;
  }
  __syncthreads();
  const uint64_t n_tiles = s_tpref[src.count];
  auto tile_of = [&](uint64_t i) { return (uint64_t)slot + i * G; };
  // a tile: its first pair, its pair count, whether it is read with 16-byte loads
  struct TileRef { const uint2* p; uint32_t n; bool vec; };
  uint32_t stream_hint = 0;                      // this block's tiles come in stream order
  auto tile_ref = [&](uint64_t tile) {
    uint32_t b = stream_hint;
    while (s_tpref[b + 1] <= tile) ++b;
    stream_hint = b;
    const uint64_t base = (tile - s_tpref[b]) * TILE;
    const uint64_t left = src.n[b] - base;
    TileRef t;
    t.p = reinterpret_cast<const uint2*>(src.ptr[b]) + base;
    t.n = left < (uint64_t)TILE ? (uint32_t)left : (uint32_t)TILE;
    t.vec = ((uintptr_t)src.ptr[b] & 15u) == 0 && t.n == (uint32_t)TILE;
    return t;
  };
  // 16-byte streaming loads of this thread's share of a whole tile; volatile,
  // so they are issued where they stand (before the work on the previous tile)
  auto load_tile = [&](uint4 (&r)[kVec], const uint2* p) {
    const uint4* p4 = reinterpret_cast<const uint4*>(p) + tid;
#pragma unroll
    for (int u = 0; u < kVec; ++u)
      asm volatile("ld.global.cs.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(r[u].x), "=r"(r[u].y), "=r"(r[u].z), "=r"(r[u].w) : "l"(p4 + u * THREADS));
  };
  // step 1 for a group of kGroup pairs (valid: bit q = pair q exists):
  // hashes, the sampled-pair queue (one warp-aggregated push per pair
  // position), the row places (independent shared atomics), the staging
  // stores; a pair whose row is full is marked in the returned mask
  auto stage_group = [&](const uint32_t (&hip)[kGroup], const uint32_t (&oip)[kGroup], uint32_t valid,
                         uint32_t par, uint32_t (&bin)[kGroup]) {
    uint32_t at[kGroup], over = 0;
#pragma unroll
    for (int q = 0; q < kGroup; ++q) {
      const uint32_t h1 = mas(d.ha[0], d.hb[0], oip[q]);
      const uint32_t ballot = __ballot_sync(kFull, ((valid >> q) & 1u) && (h1 & tau_mask) == 0u);
      if (ballot) {
        uint32_t first = 0;
        if (lane == 0) first = atomicAdd(&s_qn[par], (uint32_t)__popc(ballot));
        first = __shfl_sync(kFull, first, 0) + (uint32_t)__popc(ballot & lt_mask);
        if (((ballot >> lane) & 1u) && first < (uint32_t)QUEUE) s_queue[first] = make_uint2(hip[q], h1);
        else if ((ballot >> lane) & 1u) over |= 1u << (kGroup + q);   // queue full: SEAV bits directly
      }
      bin[q] = mas(d.ha[1], d.hb[1], oip[q]) >> h3_shift;
    }
#pragma unroll
    for (int q = 0; q < kGroup; ++q)
      at[q] = ((valid >> q) & 1u) ? atomicAdd(&s_fill[bin[q]], 1u) : 0xFFFFu;
#pragma unroll
    for (int q = 0; q < kGroup; ++q) {
      // no branch: a pair that finds its row full (or no pair) stores to
      // this lane's sink word instead
      uint32_t* dst = at[q] < (uint32_t)STAGE ? stage + bin[q] * STAGE + at[q] : sink + lane;
      *dst = hip[q];
      over |= (at[q] >= (uint32_t)STAGE && at[q] != 0xFFFFu ? 1u : 0u) << q;
    }
    return over;
  };
  // the rare leftovers of a group: pairs whose row was full (LDCA bits with
  // L2 REDs) and sampled pairs the full queue did not take (SEAV bits)
  auto group_leftovers = [&](const uint32_t (&hip)[kGroup], const uint32_t (&oip)[kGroup],
                             const uint32_t (&bin)[kGroup], uint32_t over) {
    if (__any_sync(kFull, over != 0u)) {
#pragma unroll
      for (int q = 0; q < kGroup; ++q) {
        if ((over >> q) & 1u) spill(hip[q], bin[q]);
        if ((over >> (kGroup + q)) & 1u) seav_set(d, seav, hip[q], mas(d.ha[0], d.hb[0], oip[q]));
      }
    }
  };
  // whole chunks of bin b's row (fill f <= STAGE) to its list, remainder to the front
  auto flush_row = [&](uint32_t b, uint32_t f) {
    uint32_t* row = stage + b * STAGE;
    uint32_t* list = list_of(b);
    uint32_t cur = s_cursor[b];
    const uint32_t nch = f / kChunk;
    for (uint32_t c = 0; c < nch; ++c) {
      const uint4 x = *reinterpret_cast<const uint4*>(row + c * kChunk);
      const uint4 y = *reinterpret_cast<const uint4*>(row + c * kChunk + 4);
      if (cur + kChunk <= cap) {
        st_chunk(list + cur, x, y);
        cur += kChunk;
      } else {                                      // list full: straight to L2
        const uint32_t h[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
        for (int e = 0; e < 8; ++e) spill(h[e], b);
      }
    }
    const uint32_t rem = f - nch * kChunk;
    for (uint32_t e = 0; e < rem; e += 4)           // within the row: nch * 8 + rem <= STAGE
      *reinterpret_cast<uint4*>(row + e) = *reinterpret_cast<const uint4*>(row + nch * kChunk + e);
    s_fill[b] = rem;
    s_cursor[b] = cur;
  };
  // 1. hash, queue the sampled pairs, stage the hips of one tile in their bins' rows
  auto stage_tile = [&](const uint4 (&r)[kVec], const TileRef& t, uint32_t par) {
    if (t.vec) {
#pragma unroll
      for (int g = 0; g < kVec / (kGroup / 2); ++g) {
        uint32_t hip[kGroup], oip[kGroup], bin[kGroup];
#pragma unroll
        for (int u = 0; u < kGroup / 2; ++u) {
          const uint4 v = r[g * (kGroup / 2) + u];
          hip[2 * u] = v.x; oip[2 * u] = v.y;
          hip[2 * u + 1] = v.z; oip[2 * u + 1] = v.w;
        }
        const uint32_t over = stage_group(hip, oip, (1u << kGroup) - 1u, par, bin);
        group_leftovers(hip, oip, bin, over);
      }
    } else {
      for (uint32_t j0 = 0; j0 < (uint32_t)TILE; j0 += kGroup * THREADS) {
        uint32_t hip[kGroup], oip[kGroup], bin[kGroup], valid = 0;
#pragma unroll
        for (int q = 0; q < kGroup; ++q) {
          const uint32_t j = j0 + (uint32_t)q * THREADS + tid;
          uint2 v = make_uint2(0u, 0u);
          if (j < t.n) { v = __ldcs(t.p + j); valid |= 1u << q; }
          hip[q] = v.x; oip[q] = v.y;
        }
        const uint32_t over = stage_group(hip, oip, valid, par, bin);
        group_leftovers(hip, oip, bin, over);
      }
    }
  };
  // the flush round: whole chunks to the lists; the queued SEAV updates,
  // spread over the warps
  auto flush_round = [&](uint32_t par) {
    __syncthreads();
    const uint32_t qn = s_qn[par] < (uint32_t)QUEUE ? s_qn[par] : (uint32_t)QUEUE;
    if (tid == 0) s_qn[par ^ 1u] = 0;            // read by every thread before the last barrier
    for (uint32_t b = tid; b < bins; b += THREADS) {
      const uint32_t f = s_fill[b];
      if (f >= (uint32_t)kChunk) flush_row(b, f < (uint32_t)STAGE ? f : (uint32_t)STAGE);
    }
    for (uint32_t e = tid; e < qn; e += THREADS) {   // consecutive threads: the fewest warps
      const uint2 x = s_queue[e];
      seav_set(d, seav, x.x, x.y);
    }
    __syncthreads();
  };
  // Tiles in pairs (i, i + 1) in the two register buffers.  A buffer's loads
  // for tile t + 2 go out as soon as tile t is staged, so the flush round
  // runs with both next tiles in flight (the flush's stores and the stream's
  // loads overlap); a flush round after every TPR tiles.
  uint4 ra[kVec], rb[kVec];
  TileRef ta{nullptr, 0u, false}, tb{nullptr, 0u, false};
  if (tile_of(0) < n_tiles) {
    ta = tile_ref(tile_of(0));
    if (ta.vec) load_tile(ra, ta.p);
  }
  if (tile_of(1) < n_tiles) {
    tb = tile_ref(tile_of(1));
    if (tb.vec) load_tile(rb, tb.p);
  }
  uint32_t par = 0;
  for (uint64_t i = 0; tile_of(i) < n_tiles; i += 2) {
    const bool has_b = tile_of(i + 1) < n_tiles;
    stage_tile(ra, ta, par);
    if (tile_of(i + 2) < n_tiles) {
      ta = tile_ref(tile_of(i + 2));
      if (ta.vec) load_tile(ra, ta.p);
    }
    if (TPR == 1) {
      flush_round(par);
      par ^= 1u;
    }
    if (has_b) {
      stage_tile(rb, tb, par);
      if (tile_of(i + 3) < n_tiles) {
        tb = tile_ref(tile_of(i + 3));
        if (tb.vec) load_tile(rb, tb.p);
      }
    }
    flush_round(par);
    par ^= 1u;
  }
  // remainders (< 8 hips per row) with plain stores
  for (uint32_t b = tid; b < bins; b += THREADS) {
    const uint32_t f = s_fill[b];
    uint32_t* list = list_of(b);
    uint32_t c = s_cursor[b];
    for (uint32_t e = 0; e < f; ++e) {
      const uint32_t h = stage[b * STAGE + e];
      if (c < cap) list[c++] = h;
      else spill(h, b);
    }
    counts[(uint64_t)b * G + cta] = c;
  }
}

// A list read once streams past L2 (evict first); a list that SPLIT > 1
// blocks read, close together in time, stays there for the second read.
template <int SPLIT>
__device__ __forceinline__ uint32_t load_hip(const uint32_t* p) {
  return SPLIT == 1 ? __ldcs(p) : __ldg(p);
}

// k_apply, LCL = log2 LC when it is fixed at compile time (profiles D, D3
// and S: constant shifts and row offsets), 0 for any LC.  SPLIT blocks share
// a plane, each holding LR / SPLIT of its LDCA rows in shared memory and
// reading the whole hip list: wide planes (LC = 2^18: 128 KiB for four rows)
// would otherwise leave one block per SM.
template <int LR, int THREADS, int LCL, int SPLIT>
__global__ void __launch_bounds__(THREADS)
k_apply(DevParams d, const uint32_t* __restrict__ lists, const uint32_t* __restrict__ counts,
        uint32_t G, uint32_t cap, uint32_t* __restrict__ planes, bool accumulate) {
  extern __shared__ uint32_t s_plane[];
  constexpr int LRP = LR / SPLIT;                                  // rows of this block
  const uint32_t b = blockIdx.x / SPLIT;
  const uint32_t row0 = (blockIdx.x % SPLIT) * (uint32_t)LRP;
  const uint32_t lc_log2 = LCL ? (uint32_t)LCL : d.lc_log2;
  const uint32_t words = ((uint32_t)LRP << lc_log2) >> 5;         // words of the block's rows
  const uint32_t word0 = row0 << (lc_log2 - 5u);                  // their first plane word
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t nwarps = THREADS / 32;
  // LH_i(hip) = h >> cshift (5 <= lc_log2 <= 20): LDC h >> cshift of row i is
  // bit (h >> cshift) mod 32 of plane word (i << (lc_log2 - 5)) + (h >> (cshift + 5))
  const uint32_t cshift = 32u - lc_log2;
  const uint32_t row_words_log2 = lc_log2 - 5u;
  // accumulator layout [ceil(words / 8)][k][8]: word w of plane b at
  // (w / 8) k 8 + 8 b + w mod 8, so that a 32-byte chunk holds 8 words of one plane
  const uint64_t chunk_stride = (uint64_t)(1u << d.k_log2) * 8u;
  uint32_t* dst = planes + (uint64_t)b * 8u;
  auto at_word = [&](uint32_t w) {
    w += word0;
    return dst + (uint64_t)(w >> 3) * chunk_stride + (w & 7u);
  };
  // the rows' hash words, held in registers
  uint32_t a_lo[LRP], a_hi[LRP];
  uint64_t bw[LRP];
#pragma unroll
  for (int r = 0; r < LRP; ++r) {
    a_lo[r] = (uint32_t)d.ha[2 + row0 + r];
    a_hi[r] = (uint32_t)(d.ha[2 + row0 + r] >> 32);
    bw[r] = d.hb[2 + row0 + r];
  }
  for (uint32_t w = tid; w < words; w += THREADS) s_plane[w] = accumulate ? *at_word(w) : 0u;
  __syncthreads();
  auto set_bits = [&](uint32_t hip) {
#pragma unroll
    for (int r = 0; r < LRP; ++r) {
      const uint64_t lo = (uint64_t)a_lo[r] * hip + bw[r];
      const uint32_t h = (uint32_t)(lo >> 32) + a_hi[r] * hip;      // MAS (Sec. 3.3 LH_r)
      if (LCL) {
        atomicOr(&s_plane[((uint32_t)r << row_words_log2) + (h >> (cshift + 5u))], 1u << ((h >> cshift) & 31u));
      } else {
        // the clamping funnel shift gives 0 for the shift of 32 at lc_log2 = 5;
        // the wrapping one takes the bit position mod 32
        atomicOr(&s_plane[((uint32_t)r << row_words_log2) + __funnelshift_rc(h, 0u, cshift + 5u)],
                 __funnelshift_l(0u, 1u, h >> cshift));
      }
    }
  };
  for (uint32_t c = warp; c < G; c += nwarps) {
    const uint32_t n = counts[(uint64_t)b * G + c];
    const uint32_t* src = lists + ((uint64_t)b * G + c) * cap + lane;
    uint32_t i0 = 0;
    for (; i0 + 32 * kApplyUnroll <= n; i0 += 32 * kApplyUnroll) {     // whole rounds: no bounds checks
      uint32_t hip[kApplyUnroll];
#pragma unroll
      for (int u = 0; u < kApplyUnroll; ++u) hip[u] = load_hip<SPLIT>(src + i0 + u * 32);   // all in flight
#pragma unroll
      for (int u = 0; u < kApplyUnroll; ++u) set_bits(hip[u]);
    }
    if (i0 < n) {                                   // the last, partial round: masked, loads still in flight together
      uint32_t hip[kApplyUnroll];
#pragma unroll
      for (int u = 0; u < kApplyUnroll; ++u)
        hip[u] = (i0 + u * 32 + lane < n) ? load_hip<SPLIT>(src + i0 + u * 32) : 0u;
#pragma unroll
      for (int u = 0; u < kApplyUnroll; ++u)
        if (i0 + u * 32 + lane < n) set_bits(hip[u]);
    }
  }
  __syncthreads();
  for (uint32_t w = tid; w < words; w += THREADS) *at_word(w) = s_plane[w];
}

// 32 x 32 bit transpose across a warp: lane l holds row l (bit j = column j);
// afterwards lane l holds column l (bit p = row p's bit l).  Stage s = 16, 8,
// 4, 2, 1 swaps s x s blocks between lanes l and l ^ s.  With m the columns
// whose bit s is clear, the lane whose bit s is clear keeps its m columns and
// takes the partner's m columns moved up by s; the other lane keeps its ~m
// columns and takes the partner's ~m columns moved down by s.  Either move is
// a rotation of the partner's word (left by s, or by 32 - s) whose other bits
// land in the columns the lane keeps, so a stage is one shuffle, one
// funnel-shift rotation and one bitwise select.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, uint32_t lane) {
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const uint32_t s = 16u >> st;
    const bool high = (lane & s) != 0u;
    const uint32_t keep = high ? ~masks[st] : masks[st];
    const uint32_t y = __shfl_xor_sync(kFull, x, s);
    const uint32_t t = __funnelshift_l(y, y, high ? 32u - s : s);
    x = (x & keep) | (t & ~keep);
  }
  return x;
}

// planes: [ceil(W / 8)][k][8] words (W = LR * LC / 32 words per plane, 8-word
// chunks of the k planes side by side); ldca: [LR * LC][k / 32] words.
// A warp task is 8 consecutive plane words J0 .. J0 + 7 (one 32-byte chunk of
// each plane it reads; 32 planes' chunks are 1 KiB of contiguous memory)
// times 4 consecutive LDC words: it transposes 32 planes x 32 LDCs per word
// and ORs the result into the lanes' LDC lines.
__global__ void __launch_bounds__(256)
k_fold(const uint32_t* __restrict__ planes, uint32_t* __restrict__ ldca, uint32_t W, uint32_t k_log2,
       const uint32_t* __restrict__ fresh) {
  const bool write_only = fresh != nullptr && *fresh == 0u;       // the LDCA is all zero: no read
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t wpl = 1u << (k_log2 - 5u);                       // words per LDC
  const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarp = ((uint64_t)gridDim.x * blockDim.x) >> 5;
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
        const uint32_t keep = q < wpl ? kFull : 0u;     // planes past k (k < 128 only) read as zero
        const uint4* chunk = reinterpret_cast<const uint4*>(planes + g * ((uint64_t)wpl * 256u) +
                                                            (uint64_t)((q < wpl ? q : 0u) * 32u + lane) * 8u);
        const uint4 a = chunk[0], c = chunk[1];
        x[u][0] = a.x & keep; x[u][1] = a.y & keep; x[u][2] = a.z & keep; x[u][3] = a.w & keep;
        x[u][4] = c.x & keep; x[u][5] = c.y & keep; x[u][6] = c.z & keep; x[u][7] = c.w & keep;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if ((uint32_t)j >= nj) break;
        uint32_t acc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = transpose32(x[u][j], lane);
        uint32_t* line = ldca + ((uint64_t)(J0 + j) * 32u + lane) * wpl;
        if (wpl >= 4) {
          uint4 o = write_only ? make_uint4(0u, 0u, 0u, 0u) : *reinterpret_cast<uint4*>(line + q0);
          o.x |= acc[0]; o.y |= acc[1]; o.z |= acc[2]; o.w |= acc[3];
          *reinterpret_cast<uint4*>(line + q0) = o;
        } else {
          for (uint32_t u = 0; u < wpl; ++u) line[u] = (write_only ? 0u : line[u]) | acc[u];
        }
      }
    }
  }
}

// k_fold8 (k >= 256): a warp task is 8 plane words J0 .. J0 + 7 times 8
// consecutive LDC words q0 .. q0 + 7, so each lane ORs one whole 32-byte
// sector into each of its 8 LDC lines; the 8 chunks of 8 planes' words are
// loaded up front (16 loads in flight per lane).
__global__ void __launch_bounds__(256)
k_fold8(const uint32_t* __restrict__ planes, uint32_t* __restrict__ ldca, uint32_t W, uint32_t k_log2,
        const uint32_t* __restrict__ fresh) {
  const bool write_only = fresh != nullptr && *fresh == 0u;       // the LDCA is all zero: no read
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t wpl = 1u << (k_log2 - 5u);                       // words per LDC, >= 8
  const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarp = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t n_groups = (W + 7) / 8;
  const uint32_t n_q = wpl / 8;                                    // groups of 8 LDC words
  for (uint64_t t = gwarp; t < n_groups * n_q; t += nwarp) {
    const uint64_t g = t / n_q;
    const uint32_t J0 = (uint32_t)(g * 8);
    const uint32_t nj = (W - J0) < 8u ? (W - J0) : 8u;
    const uint32_t q0 = (uint32_t)(t % n_q) * 8u;
    uint32_t x[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const uint4* chunk = reinterpret_cast<const uint4*>(planes + g * ((uint64_t)wpl * 256u) +
                                                          (uint64_t)((q0 + u) * 32u + lane) * 8u);
      const uint4 a = chunk[0], c = chunk[1];
      x[u][0] = a.x; x[u][1] = a.y; x[u][2] = a.z; x[u][3] = a.w;
      x[u][4] = c.x; x[u][5] = c.y; x[u][6] = c.z; x[u][7] = c.w;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if ((uint32_t)j >= nj) break;
      uint4* line = reinterpret_cast<uint4*>(ldca + ((uint64_t)(J0 + j) * 32u + lane) * wpl + q0);
      uint4 o0 = make_uint4(0u, 0u, 0u, 0u), o1 = o0;
      if (!write_only) {
        o0 = line[0];
        o1 = line[1];
      }
      o0.x |= transpose32(x[0][j], lane); o0.y |= transpose32(x[1][j], lane);
      o0.z |= transpose32(x[2][j], lane); o0.w |= transpose32(x[3][j], lane);
      o1.x |= transpose32(x[4][j], lane); o1.y |= transpose32(x[5][j], lane);
      o1.z |= transpose32(x[6][j], lane); o1.w |= transpose32(x[7][j], lane);
      line[0] = o0;
      line[1] = o1;
    }
  }
}

template <int THREADS, int STAGE, int TPR, int PER_SM>
cudaError_t bin_chunk(const DevParams& d, uint8_t* seav, uint32_t* ldca, const BinSrc& src,
                      const BinnedScratch& s, uint32_t cap, bool append, uint32_t rot, cudaStream_t st) {
  const uint32_t bins = 1u << d.k_log2;
  // the bins' staging rows, the sampled-pair queue, 2 counters per bin
  const size_t bin_smem = (size_t)bins * STAGE * 4 + 32 * 4 + (size_t)(TPR * THREADS * kVec * 2 / 32) * 8 +
                          (size_t)bins * 8;
  auto kern = k_bin<THREADS, STAGE, TPR, PER_SM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bin_smem);
  if (e != cudaSuccess) return e;
  kern<<<s.ctas, THREADS, bin_smem, st>>>(d, seav, ldca, src, s.lists, s.counts, cap, append, rot, s.ovf);
  return cudaGetLastError();
}

template <int LR, int THREADS, int LCL, int SPLIT = 1>
cudaError_t apply_round_t(const DevParams& d, const BinnedScratch& s, uint32_t cap, bool accumulate, cudaStream_t st) {
  const uint32_t bins = 1u << d.k_log2;
  const uint32_t words = ((uint32_t)(LR / SPLIT) << d.lc_log2) >> 5;
  const size_t apply_smem = (size_t)words * sizeof(uint32_t);
  auto kern = k_apply<LR, THREADS, LCL, SPLIT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)apply_smem);
  if (e != cudaSuccess) return e;
  kern<<<bins * SPLIT, THREADS, apply_smem, st>>>(d, s.lists, s.counts, s.ctas, cap, s.planes, accumulate);
  return cudaGetLastError();
}

template <int LR, int THREADS>
cudaError_t apply_round_lc(const DevParams& d, const BinnedScratch& s, uint32_t cap, bool accumulate,
                           cudaStream_t st) {
  if constexpr (LR == 4) {            // the profiles' LDCA widths get constant shifts
    if (d.lc_log2 == 16) return apply_round_t<LR, THREADS, 16>(d, s, cap, accumulate, st);
    if (d.lc_log2 == 18) return apply_round_t<LR, THREADS, 18, 2>(d, s, cap, accumulate, st);
    if (d.lc_log2 == 14) return apply_round_t<LR, THREADS, 14>(d, s, cap, accumulate, st);
  }
  return apply_round_t<LR, THREADS, 0>(d, s, cap, accumulate, st);
}

template <int LR>
cudaError_t apply_round(const DevParams& d, const BinnedScratch& s, uint32_t cap, bool accumulate, cudaStream_t st) {
  return s.shape.apply_threads == 256 ? apply_round_lc<LR, 256>(d, s, cap, accumulate, st)
                                      : apply_round_lc<LR, 512>(d, s, cap, accumulate, st);
}

}  // namespace

bool binned_applicable(const DevParams& d) {
  const uint64_t plane_bits = (uint64_t)d.lr << d.lc_log2;
  return d.k_log2 >= 5 && d.k_log2 <= 10 && d.lc_log2 >= 5 && plane_bits <= (1ull << 20);
}

// The compiled staging shapes: {k_bin threads, row hips, tiles per flush
// round, blocks per SM, k_apply threads}.  Rows hold 4 x odd hips, so the
// flush's 16-byte row reads of 8 consecutive bins hit all 32 banks; a row
// holds the < 8 hips a flush leaves plus a round's arrivals with headroom
// (one block per SM: 2 tiles of 8K pairs, 16 per bin on average, 44-hip rows;
// two per SM: 2 tiles of 4K pairs, 20-hip rows).
constexpr BinShape kShapes[] = {
  {1024, 44, 2, 1, 512}, {1024, 44, 2, 1, 256},
  {512, 20, 2, 2, 512},  {512, 20, 2, 2, 256},
};

int binned_shape_count() { return (int)(sizeof(kShapes) / sizeof(kShapes[0])); }
BinShape binned_shape(int i) { return kShapes[(i >= 0 && i < binned_shape_count()) ? i : 0]; }

// List capacity for a round of n_pairs split into `chunks` binning launches:
// a block takes at most ceil(tiles / ctas) + 1 tiles per launch (the tile to
// block mapping rotates between launches), spread over the bins; 8 standard
// deviations plus 32 of headroom, so that only skewed inputs overflow.
uint32_t binned_list_cap(uint64_t n_pairs, uint32_t bins, const BinShape& shape, uint32_t ctas, uint32_t chunks) {
  const uint64_t tile = binned_tile_pairs(shape);
  const uint64_t tiles = (n_pairs + tile - 1) / tile;
  const uint64_t per_cta = (tiles + ctas - 1) / ctas + (chunks > 1 ? chunks : 1);
  const double m = (double)(per_cta * tile < n_pairs ? per_cta * tile : n_pairs) / bins;
  uint64_t cap = (uint64_t)(m + 8.0 * sqrt(m + 1.0) + 32.0);
  cap = (cap + 7) & ~7ull;                                   // 32-byte list starts
  return (uint32_t)cap;
}

static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

int binned_ctas(const BinShape& shape) { return sm_count() * (int)shape.per_sm; }

int binned_fold_grid() { return sm_count() * 8; }

cudaError_t launch_fold(const DevParams& d, const uint32_t* planes, uint32_t* ldca, int grid, cudaStream_t st,
                        const uint32_t* fresh) {
  const uint32_t words = (uint32_t)(((uint64_t)d.lr << d.lc_log2) >> 5);
  if (d.k_log2 >= 8) k_fold8<<<grid, 256, 0, st>>>(planes, ldca, words, d.k_log2, fresh);
  else k_fold<<<grid, 256, 0, st>>>(planes, ldca, words, d.k_log2, fresh);
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
  // the list stride never exceeds what was allocated (hips past a full list go
  // to L2 REDs, so a smaller cap only costs speed)
  if (cap > s.cap_alloc) cap = s.cap_alloc;
  const BinShape& h = s.shape;
  if (h.threads == 512) return bin_chunk<512, 20, 2, 2>(d, seav, ldca, src, s, cap, append, rot, st);
  return bin_chunk<1024, 44, 2, 1>(d, seav, ldca, src, s, cap, append, rot, st);
}

cudaError_t binned_apply_round(const DevParams& d, const BinnedScratch& s, uint32_t cap, bool accumulate,
                               cudaStream_t st) {
  if (cap > s.cap_alloc) cap = s.cap_alloc;          // the same clamp as the round's binning launches
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

uint32_t binned_tile_pairs(const BinShape& shape) { return shape.threads * (uint32_t)kVec * 2u; }

uint64_t binned_planes_bytes(const DevParams& d) {
  const uint64_t words = ((uint64_t)d.lr << d.lc_log2) >> 5;          // per plane
  return ((words + 7) / 8) * 8 * ((uint64_t)1 << d.k_log2) * sizeof(uint32_t);
}

cudaError_t launch_scan_binned(const DevParams& d, uint8_t* seav, uint32_t* ldca, const uint32_t* pairs,
                               uint64_t n_pairs, const BinnedScratch& s, cudaStream_t st) {
  uint64_t done = 0;
  bool accumulate = s.accumulate;
  while (done < n_pairs) {
    const uint64_t n = (n_pairs - done) < s.max_pairs ? (n_pairs - done) : s.max_pairs;
    const uint32_t cap = binned_list_cap(n, 1u << d.k_log2, s.shape, s.ctas, 1);
    cudaError_t e = binned_bin_chunk(d, seav, ldca, bin_src_one(pairs + 2 * done, n), s, cap, false, 0, st);
    if (e == cudaSuccess) e = binned_apply_round(d, s, cap, accumulate, st);
    if (e != cudaSuccess) return e;
    accumulate = true;
    done += n;
  }
  return cudaSuccess;
}

}  // namespace sp
