// sp_detect.cu -- end-of-window restore and filter (Sec. 3.2-3.3, Sec. 4.2).
//
// k_detect: one warp per SEA (grid-stride over the 2^r SEAs).
//   1. HSE(i): lanes test the SEs of a row for weight >= 3 (4 per lane per
//      32-bit load on rows of 128+ SEs) and a ballot/popc prefix compacts the
//      hot columns into a per-warp list in shared memory (Sec. 3.2, "hot SE").
//   2. CIS: lanes split the product HSE(0) x HSE(1); each lane then walks
//      rows 2 .. SR-1 depth first.  A partial tuple is dropped as soon as two
//      rows disagree on a shared LP bit (it then matches no LP) or the AND of
//      its SEs falls below weight 3 -- AND only clears bits, so the pruning
//      loses nothing against testing complete tuples (Sec. 3.2, SEU test).
//   3. A complete tuple fixes every LP bit (Eq. 3, coverage constraint);
//      ip = LP << r | RP goes to a per-warp queue.  When the SEA is done the
//      warp tests the queued hosts together: the LDC union (AND over the LR
//      rows, Sec. 3.3) of one host is read as LR lines of k bits spread over
//      the lanes (one coalesced load per row and lane), z0 = k - popc by a
//      warp reduction.  The host survives when z0 <= Z_theta, the integer
//      form of Est >= threshold (Eq. 4).  A full queue falls back to the
//      same test in one lane.  For a sliding router (Sec. 5.2) a line word
//      is the union of the slice bits not yet committed and the 32 stamps of
//      the word that are active at the router's slice clock.
//   Survivors are appended as (ip << 32 | z0) keys with one atomic per hit.
// k_sort_emit: sorts the keys by ip (ascending; ips are unique) and writes
//   sp_candidate records with est taken from a table of -k ln(z0 / k).  Up to
//   8,192 keys one block sorts them in shared memory (bitonic).  Above that,
//   the cooperative grid sorts runs of 8,192 keys in shared memory, one block
//   per run, then merges pairs of runs in log2(runs) rounds between grid-wide
//   barriers: each key's place in the merged run is its index in its own run
//   plus the number of keys of the sibling run below it (binary search).
//   The rounds alternate between the key buffer and the record buffer (which
//   holds at least as many bytes), ending in the key buffer.
#include <cooperative_groups.h>

#include "sp_internal.h"

namespace cg = cooperative_groups;

namespace sp {

namespace {

constexpr int kDetectWarps = 8;
constexpr int kDetectThreads = kDetectWarps * 32;
constexpr int kHostQueue = 256;                  // complete tuples queued per warp
constexpr uint32_t kFull = 0xFFFFFFFFu;
// SEAs of 512 bytes (profiles D, D3 and S) are staged in shared memory: a
// ring of kSeaRing SEAs per warp, filled kSeaRing - 1 SEAs ahead of use
constexpr uint32_t kStagedSea = 512;
constexpr int kSeaRing = 4;

// 16-byte asynchronous copy from global to shared memory (one per lane)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

struct Found {
  uint64_t* keys;
  uint32_t cap;
  uint64_t max_join;
  DetectStatus* status;
};

// Where the LDCA test reads the bits of an LDC line.  Discrete window: the
// LDCA itself.  Sliding window (Sec. 5.2): word w of the window LDCA is the
// union of the bits of the slice sketch not yet committed (bits[w]) and the
// stamps of word w (32 bytes at stamps + 32 w) active at the router's clock.
// Only the lines of tested hosts are read, so a detect touches a few MB of
// stamps instead of streaming the whole counter pool.
struct LdcaRead {
  const uint32_t* bits;
  const uint4* stamps;
  uint32_t cur4, k4;
};

template <bool kSliding>
__device__ __forceinline__ uint32_t ldc_word(const LdcaRead& a, uint64_t w) {
  if (!kSliding) return a.bits[w];
  return a.bits[w] | active32(a.stamps[2 * w], a.stamps[2 * w + 1], a.cur4, a.k4);
}

// word index of the first word of host ip's LDC line in LDCA row i
__device__ __forceinline__ uint64_t ldc_line(const DevParams& d, uint32_t ip, uint32_t i) {
  const uint32_t col = (uint32_t)((uint64_t)mas(d.ha[2 + i], d.hb[2 + i], ip) >> (32u - d.lc_log2));
  return (uint64_t)((i << d.lc_log2) | col) << (d.k_log2 - 5u);
}

template <bool kSliding>
__device__ __forceinline__ uint32_t ldc_zeros(const DevParams& d, const LdcaRead& a, uint32_t ip) {
  const uint32_t wpl = 1u << (d.k_log2 - 5u);
  uint64_t line[8];
  for (uint32_t i = 0; i < d.lr; ++i) line[i] = ldc_line(d, ip, i);
  uint32_t ones = 0;
  if (kSliding) {
    for (uint32_t w = 0; w < wpl; ++w) {
      uint32_t u = ldc_word<true>(a, line[0] + w);
      for (uint32_t i = 1; i < d.lr; ++i) u &= ldc_word<true>(a, line[i] + w);
      ones += __popc(u);
    }
    return (1u << d.k_log2) - ones;
  }
  const uint32_t* ldca = a.bits;
  if (wpl >= 4) {
    for (uint32_t w = 0; w < wpl; w += 4) {
      uint4 u = *reinterpret_cast<const uint4*>(ldca + line[0] + w);
      for (uint32_t i = 1; i < d.lr; ++i) {
        const uint4 v = *reinterpret_cast<const uint4*>(ldca + line[i] + w);
        u.x &= v.x; u.y &= v.y; u.z &= v.z; u.w &= v.w;
      }
      ones += __popc(u.x) + __popc(u.y) + __popc(u.z) + __popc(u.w);
    }
  } else {
    for (uint32_t w = 0; w < wpl; ++w) {
      uint32_t u = ldca[line[0] + w];
      for (uint32_t i = 1; i < d.lr; ++i) u &= ldca[line[i] + w];
      ones += __popc(u);
    }
  }
  return (1u << d.k_log2) - ones;
}

__device__ __forceinline__ void keep_host(uint32_t ip, uint32_t z0, uint32_t z_theta, const Found& f) {
  if (z0 <= z_theta) {
    const uint32_t slot = atomicAdd(&f.status->count, 1u);
    if (slot < f.cap) f.keys[slot] = ((uint64_t)ip << 32) | z0;
    else atomicOr(&f.status->overflow, 1u);
  }
}

// One complete, consistent tuple: count it against the join bound and queue
// its IP for the warp's LDCA test (tested here when the queue is full).
// Returns false when the detect must stop (a bound was hit).
template <bool kSliding>
__device__ __forceinline__ bool emit_lp(const DevParams& d, const LdcaRead& ldca,
                                        uint32_t rp, uint32_t lp, uint32_t z_theta,
                                        const Found& f, uint32_t& join_local,
                                        uint32_t* queue, uint32_t* queue_n) {
  if (++join_local == 64u) {
    const unsigned long long prev = atomicAdd(reinterpret_cast<unsigned long long*>(&f.status->join), 64ull);
    join_local = 0;
    if (prev + 64ull > f.max_join) { atomicOr(&f.status->overflow, 2u); return false; }
  }
  const uint32_t ip = (uint32_t)(((uint64_t)lp << d.r) | rp);
  const uint32_t at = atomicAdd(queue_n, 1u);
  if (at < (uint32_t)kHostQueue) queue[at] = ip;
  else keep_host(ip, ldc_zeros<kSliding>(d, ldca, ip), z_theta, f);
  return true;
}

// The warp's LDCA test of n queued hosts (all lanes call it).  A host's LR
// lines of wpl words are split over the lanes: with wpl >= 32 each lane
// takes every 32nd word of each line and two hosts go per pass; with
// wpl < 32 a pass takes 32 / wpl hosts, one word per lane.
template <bool kSliding>
__device__ void test_queue(const DevParams& d, const LdcaRead& ldca, const uint32_t* queue,
                           uint32_t n, uint32_t z_theta, const Found& f, uint32_t lane) {
  const uint32_t wpl = 1u << (d.k_log2 - 5u);
  const uint32_t k = 1u << d.k_log2;
  if (wpl >= 32) {
    for (uint32_t q = 0; q < n; q += 2) {
      const bool two = q + 1 < n;
      const uint32_t ip0 = queue[q], ip1 = two ? queue[q + 1] : ip0;
      uint32_t ones0 = 0, ones1 = 0;
      for (uint32_t w = lane; w < wpl; w += 32) {
        uint32_t u0 = kFull, u1 = kFull;
        for (uint32_t i = 0; i < d.lr; ++i) {
          u0 &= ldc_word<kSliding>(ldca, ldc_line(d, ip0, i) + w);
          u1 &= ldc_word<kSliding>(ldca, ldc_line(d, ip1, i) + w);
        }
        ones0 += __popc(u0);
        ones1 += __popc(u1);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ones0 += __shfl_xor_sync(kFull, ones0, o);
        ones1 += __shfl_xor_sync(kFull, ones1, o);
      }
      if (lane == 0) {
        keep_host(ip0, k - ones0, z_theta, f);
        if (two) keep_host(ip1, k - ones1, z_theta, f);
      }
    }
  } else {
    const uint32_t per = 32u / wpl;                 // hosts per pass
    const uint32_t sub = lane / wpl, w = lane % wpl;
    for (uint32_t q0 = 0; q0 < n; q0 += per) {
      const uint32_t q = q0 + sub;
      uint32_t ones = 0;
      if (q < n) {
        const uint32_t ip = queue[q];
        uint32_t u = kFull;
        for (uint32_t i = 0; i < d.lr; ++i) u &= ldc_word<kSliding>(ldca, ldc_line(d, ip, i) + w);
        ones = __popc(u);
      }
      for (uint32_t o = wpl >> 1; o > 0; o >>= 1) ones += __shfl_xor_sync(kFull, ones, o);
      if (w == 0 && q < n) keep_host(queue[q], k - ones, z_theta, f);
    }
  }
}

template <bool kSliding>
__global__ void __launch_bounds__(kDetectThreads, 4)
k_detect(DevParams d, const uint8_t* __restrict__ seav, LdcaRead ldca, const uint64_t* __restrict__ clock,
         uint32_t k_slices, uint32_t z_theta, Found f, bool staged) {
  extern __shared__ __align__(16) uint32_t s_dyn[];
  if (kSliding) {                                   // the window of the router's current slice
    ldca.cur4 = ((uint32_t)(*clock % 255u) + 1u) * 0x01010101u;
    ldca.k4 = k_slices * 0x01010101u;
  }
  __shared__ uint32_t s_queue_n[kDetectWarps];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  uint32_t* queue = s_dyn + warp * kHostQueue;           // [kDetectWarps][kHostQueue] IPs
  uint32_t* queue_n = &s_queue_n[warp];
  uint16_t* lists = reinterpret_cast<uint16_t*>(s_dyn + kDetectWarps * kHostQueue) + warp * d.sea_bytes;
  if (lane == 0) *queue_n = 0;
  __syncwarp();
  const uint32_t n_sea = 1u << d.r;
  const uint32_t stride = gridDim.x * kDetectWarps;
  // staged SEAs (512 bytes, 16-byte aligned SEAV): the warp's ring of
  // kSeaRing SEAs after the lists; 16 bytes per lane and SEA by cp.async,
  // one commit group per SEA (empty past the last SEA, so that the count of
  // groups in flight stays fixed)
  uint8_t* ring = reinterpret_cast<uint8_t*>(s_dyn + kDetectWarps * kHostQueue) +
                  (size_t)kDetectWarps * d.sea_bytes * sizeof(uint16_t) + (size_t)warp * kSeaRing * kStagedSea;
  auto stage_sea = [&](uint32_t rp, uint32_t slot) {
    if (rp < n_sea) cp_async16(ring + slot * kStagedSea + 16u * lane, seav + (uint64_t)rp * kStagedSea + 16u * lane);
    cp_async_commit();
  };
  uint32_t rp = blockIdx.x * kDetectWarps + warp;
  if (staged) {
#pragma unroll
    for (int j = 0; j < kSeaRing - 1; ++j) stage_sea(rp + (uint32_t)j * stride, (uint32_t)j);
  }
  uint32_t join_local = 0;
  bool stop = false;
  for (uint32_t it = 0; rp < n_sea && !stop; rp += stride, ++it) {
    // the join-bound flag (warp-uniform: lane 0 reads it, every lane sees its
    // value) is read here and tested after this SEA, so the read overlaps the
    // work; a warp stops at most one SEA later than the bound was hit
    const uint32_t ov = lane == 0 ? *reinterpret_cast<volatile uint32_t*>(&f.status->overflow) : 0u;
    const uint8_t* sea = seav + (uint64_t)rp * d.sea_bytes;
    if (staged) {
      // the SEA kSeaRing - 1 ahead goes to the slot this warp read last
      // (every lane passed the __syncwarp at the end of that iteration); then
      // wait for this SEA's copy and make every lane's bytes visible
      stage_sea(rp + (uint32_t)(kSeaRing - 1) * stride, (it + kSeaRing - 1) % kSeaRing);
      cp_async_wait<kSeaRing - 1>();
      __syncwarp();
      sea = ring + (it % kSeaRing) * kStagedSea;
    }
    // 1. hot SEs per row
    uint32_t cnt[8];
    bool empty = false;
    for (uint32_t i = 0; i < d.sr; ++i) {
      const uint32_t sc = 1u << d.ibn[i];
      const uint8_t* row = sea + d.row_off[i];
      uint32_t n = 0;
      if (sc >= 128 && ((uintptr_t)row & 3u) == 0) {
        // rows of 128+ SEs, word aligned: 4 SEs per lane per load; the list
        // is ordered by (byte of the word, lane), which only changes the order
        // in which candidates are tried
        for (uint32_t c0 = 0; c0 < sc; c0 += 128) {
          const uint32_t w = *reinterpret_cast<const uint32_t*>(row + c0 + 4 * lane);
#pragma unroll
          for (uint32_t j = 0; j < 4; ++j) {
            const bool hot = __popc((w >> (8 * j)) & 0xFFu) >= 3;
            const uint32_t bal = __ballot_sync(kFull, hot);
            if (hot) lists[d.row_off[i] + n + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)(c0 + 4 * lane + j);
            n += __popc(bal);
          }
        }
      } else {
        for (uint32_t c0 = 0; c0 < sc; c0 += 32) {
          const uint32_t c = c0 + lane;
          const bool hot = c < sc && __popc((uint32_t)row[c]) >= 3;
          const uint32_t bal = __ballot_sync(kFull, hot);
          if (hot) lists[d.row_off[i] + n + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)c;
          n += __popc(bal);
        }
      }
      cnt[i] = n;
      if (n == 0) {                                  // no tuple can cover this row: the SEA yields nothing
        empty = true;
        break;
      }
    }
    __syncwarp();
    if (!empty) {
      // 2. lanes split HSE(0) x HSE(1); depth-first over the remaining rows
      const uint32_t n1 = d.sr > 1 ? cnt[1] : 1u;
      const uint32_t total = cnt[0] * n1;
      for (uint32_t t = lane; t < total && !stop; t += 32) {
        const uint32_t c0 = lists[d.row_off[0] + t / n1];
        uint32_t km = d.cover[0];
        uint32_t kv = spread_idx(c0, d.isb[0], d.L);
        uint32_t seu = sea[d.row_off[0] + c0];
        uint32_t start = 1;
        if (d.sr > 1) {
          const uint32_t c1 = lists[d.row_off[1] + t % n1];
          const uint32_t v1 = spread_idx(c1, d.isb[1], d.L);
          if (((v1 ^ kv) & d.cover[1] & km) != 0u) continue;
          seu &= sea[d.row_off[1] + c1];
          if (__popc(seu) < 3) continue;
          km |= d.cover[1];
          kv |= v1;
          start = 2;
        }
        if (start == d.sr) {
          if (!emit_lp<kSliding>(d, ldca, rp, kv, z_theta, f, join_local, queue, queue_n)) stop = true;
          continue;
        }
        uint32_t pos[8], skm[8], skv[8], sseu[8];
        int dd = (int)start;
        pos[dd] = 0; skm[dd] = km; skv[dd] = kv; sseu[dd] = seu;
        while (dd >= (int)start && !stop) {
          if (pos[dd] >= cnt[dd]) {
            if (--dd >= (int)start) ++pos[dd];
            continue;
          }
          const uint32_t c = lists[d.row_off[dd] + pos[dd]];
          const uint32_t v = spread_idx(c, d.isb[dd], d.L);
          const uint32_t s2 = sseu[dd] & sea[d.row_off[dd] + c];
          if (((v ^ skv[dd]) & d.cover[dd] & skm[dd]) == 0u && __popc(s2) >= 3) {
            if (dd == (int)d.sr - 1) {
              if (!emit_lp<kSliding>(d, ldca, rp, skv[dd] | v, z_theta, f, join_local, queue, queue_n)) stop = true;
              ++pos[dd];
            } else {
              const int nx = dd + 1;
              pos[nx] = 0; skm[nx] = skm[dd] | d.cover[dd]; skv[nx] = skv[dd] | v; sseu[nx] = s2;
              dd = nx;
            }
          } else {
            ++pos[dd];
          }
        }
      }
    }
    __syncwarp();
    // 3. the warp's LDCA test of this SEA's complete tuples
    const uint32_t nq = min(*queue_n, (uint32_t)kHostQueue);
    if (nq) test_queue<kSliding>(d, ldca, queue, nq, z_theta, f, lane);
    __syncwarp();
    if (lane == 0) *queue_n = 0;
    __syncwarp();
    const bool bound = (__shfl_sync(kFull, ov, 0) & 2u) != 0u;
    stop = __any_sync(kFull, stop) || bound;
  }
  if (staged) cp_async_wait<0>();                  // no copy in flight at exit
  if (join_local) atomicAdd(reinterpret_cast<unsigned long long*>(&f.status->join), (unsigned long long)join_local);
}

// ---- sort + emit ----------------------------------------------------------
constexpr int kSortThreads = 1024;
constexpr uint32_t kSmemSortCap = 8192;   // 64 KiB of keys

__device__ __forceinline__ void emit_record(uint64_t key, const double* est_table, sp_candidate* out) {
  sp_candidate c;
  c.ip = (uint32_t)(key >> 32);
  c.z0 = (uint32_t)key;
  c.est = est_table[c.z0];
  c.flags = c.z0 == 0u ? SP_FLAG_SATURATED : 0u;
  c.pad = 0u;
  *out = c;
}

// bitonic sort of m (a power of two, <= kSmemSortCap) keys in shared memory, ascending
__device__ void smem_bitonic(uint64_t* a, uint32_t m) {
  for (uint32_t size = 2; size <= m; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < m / 2; i += blockDim.x) {
        const uint32_t lo = 2 * i - (i & (stride - 1));
        const uint32_t hi = lo + stride;
        const bool up = (lo & size) == 0;
        const uint64_t x = a[lo], y = a[hi];
        if ((x > y) == up) { a[lo] = y; a[hi] = x; }
      }
      __syncthreads();
    }
  }
}

// number of keys of run[0, len) below key (the keys of a run are sorted and unique)
__device__ __forceinline__ uint32_t count_below(const uint64_t* run, uint32_t len, uint64_t key) {
  uint32_t lo = 0, hi = len;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (run[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kSortThreads)
k_sort_emit(uint64_t* keys, uint32_t cap, const DetectStatus* status, const double* est_table,
            sp_candidate* out) {
  extern __shared__ uint64_t s_keys[];
  const uint32_t n = min(status->count, cap);        // the same for every block
  if (n == 0) return;
  if (n <= kSmemSortCap) {                          // one block, in shared memory
    if (blockIdx.x != 0) return;
    uint32_t m = 1;
    while (m < n) m <<= 1;
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) s_keys[i] = i < n ? keys[i] : ~0ull;
    __syncthreads();
    smem_bitonic(s_keys, m);
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) emit_record(s_keys[i], est_table, out + i);
    return;
  }
  cg::grid_group grid = cg::this_grid();
  // 1. runs of kSmemSortCap keys, sorted in shared memory, written back in place
  const uint32_t runs = (n + kSmemSortCap - 1) / kSmemSortCap;
  for (uint32_t r = blockIdx.x; r < runs; r += gridDim.x) {
    const uint32_t base = r * kSmemSortCap;
    const uint32_t len = min(kSmemSortCap, n - base);
    for (uint32_t i = threadIdx.x; i < kSmemSortCap; i += blockDim.x) s_keys[i] = i < len ? keys[base + i] : ~0ull;
    __syncthreads();
    smem_bitonic(s_keys, kSmemSortCap);
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) keys[base + i] = s_keys[i];
    __syncthreads();
  }
  // 2. merge rounds; an odd number of rounds starts with a copy so that the
  // last round writes the key buffer
  uint32_t rounds = 0;
  for (uint64_t w = kSmemSortCap; w < n; w <<= 1) ++rounds;
  uint64_t* tmp = reinterpret_cast<uint64_t*>(out);  // cap records of 24 bytes hold n keys
  uint64_t* src = keys;
  uint64_t* dst = tmp;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t gsize = (uint64_t)gridDim.x * blockDim.x;
  grid.sync();
  if (rounds & 1u) {
    for (uint64_t i = gtid; i < n; i += gsize) tmp[i] = keys[i];
    src = tmp;
    dst = keys;
    grid.sync();
  }
  for (uint64_t w = kSmemSortCap; w < n; w <<= 1) {
    for (uint64_t i = gtid; i < n; i += gsize) {
      const uint64_t base = i / (2 * w) * (2 * w);
      const uint64_t mid = base + w < n ? base + w : n;
      const uint64_t end = base + 2 * w < n ? base + 2 * w : n;
      const uint64_t key = src[i];
      uint64_t pos;
      if (i < mid) pos = i + count_below(src + mid, (uint32_t)(end - mid), key);          // run A
      else pos = (i - mid) + base + count_below(src + base, (uint32_t)(mid - base), key);  // run B
      dst[pos] = key;
    }
    grid.sync();
    uint64_t* t = src;
    src = dst;
    dst = t;
  }
  // 3. records (src is the key buffer now)
  for (uint64_t i = gtid; i < n; i += gsize) emit_record(src[i], est_table, out + i);
}

}  // namespace

namespace {

template <bool kSliding>
cudaError_t detect_launch(const DevParams& d, const uint8_t* seav, const LdcaRead& ldca, const uint64_t* clock,
                          uint32_t k_slices, uint32_t z_theta, uint64_t* keys, uint32_t cap, uint64_t max_join,
                          DetectStatus* status, cudaStream_t s) {
  // 512-byte SEAs of a 16-byte aligned SEAV are staged in shared memory
  const bool staged = d.sea_bytes == kStagedSea && ((uintptr_t)seav & 15u) == 0u;
  const size_t smem = (size_t)kDetectWarps * kHostQueue * sizeof(uint32_t) +
                      (size_t)kDetectWarps * d.sea_bytes * sizeof(uint16_t) +
                      (staged ? (size_t)kDetectWarps * kSeaRing * kStagedSea : 0u);
  cudaError_t e = cudaFuncSetAttribute(k_detect<kSliding>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_detect<kSliding>, kDetectThreads, smem);
  if (per_sm < 1) per_sm = 1;
  const uint64_t n_sea = 1ull << d.r;
  uint64_t grid = (n_sea + kDetectWarps - 1) / kDetectWarps;
  if (grid > (uint64_t)sms * per_sm) grid = (uint64_t)sms * per_sm;
  Found f{keys, cap, max_join, status};
  k_detect<kSliding><<<(unsigned)grid, kDetectThreads, smem, s>>>(d, seav, ldca, clock, k_slices, z_theta, f, staged);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_detect(const DevParams& d, const uint8_t* seav, const uint32_t* ldca,
                          uint32_t z_theta, uint64_t* keys, uint32_t cap, uint64_t max_join,
                          DetectStatus* status, cudaStream_t s) {
  return detect_launch<false>(d, seav, LdcaRead{ldca, nullptr, 0u, 0u}, nullptr, 0u, z_theta, keys, cap, max_join,
                              status, s);
}

cudaError_t launch_detect_sliding(const DevParams& d, const uint8_t* seav, const uint32_t* ldca,
                                  const uint8_t* st_ldca, const uint64_t* clock, uint32_t k, uint32_t z_theta,
                                  uint64_t* keys, uint32_t cap, uint64_t max_join, DetectStatus* status,
                                  cudaStream_t s) {
  const LdcaRead a{ldca, reinterpret_cast<const uint4*>(st_ldca), 0u, 0u};
  return detect_launch<true>(d, seav, a, clock, k, z_theta, keys, cap, max_join, status, s);
}

cudaError_t launch_sort_emit(uint64_t* keys, uint32_t cap, const DetectStatus* status,
                             const double* est_table, uint32_t /*k_log2*/,
                             sp_candidate* out, cudaStream_t s) {
  const size_t smem = kSmemSortCap * sizeof(uint64_t);
  cudaError_t e = cudaFuncSetAttribute(k_sort_emit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // a cooperative grid (every block resident) of at most one block per SM,
  // and no more blocks than runs of the largest count
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort_emit, kSortThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint32_t max_runs = (cap + kSmemSortCap - 1) / kSmemSortCap;
  const unsigned grid = (unsigned)(max_runs < (uint32_t)sms ? (max_runs ? max_runs : 1u) : (uint32_t)sms);
  void* args[] = {&keys, &cap, &status, &est_table, &out};
  e = cudaLaunchCooperativeKernel((const void*)k_sort_emit, dim3(grid), dim3(kSortThreads), args, smem, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace sp
