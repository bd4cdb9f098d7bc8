// sp_slide.cu -- the sliding time window extension (Sec. 5).
//
// Sec. 5.2 replaces every bit of SEAV and LDCA by a small timestamp counter
// (the paper's "asynchronous timestamp"; its internals are in a cited paper
// that is not available).  Reading used here: a bit is active in the window
// W(t, k) iff it was set in one of the slices t-k+1 .. t.
//
// Counter: one byte per bit holding the id of the last slice that set it,
// id(t) = t mod 255 + 1 (0 = never set).  Its age at slice t is
// (id(t) - stamp) mod 255, exact as long as the true age is below 255.
//   The scan of Sec. 3.1-3.3 runs unchanged (direct, binned or batched) into
//   a per-router bit sketch of the current slice: the counters are never the
//   target of random stores, which on a counter pool larger than L2 would
//   cost a DRAM read-modify-write per store.
//   k_commit      stamps id(t) on the counters of every bit set in the slice's
//                 bit sketch and clears the sketch (one pass over the sketch;
//                 counters of clear bits keep their stamp).  It runs when the
//                 slice closes and before a merge reads the counters.
//   k_commit_window  the same commit fused with one streaming pass over the
//                 counters that writes the window's bits (active counters) as
//                 an ordinary SEAV/LDCA.  Export reads that image.  A detect
//                 runs it over the SEAV alone: its LDCA test reads the stamps
//                 of the tested hosts' lines (k_detect), and the slice's LDCA
//                 bits are committed when the slice closes.
//   k_clean       at every slide, one of M = 255 - k segments of the counter
//                 pool is swept and counters of age >= k are reset to 0; each
//                 counter is swept at most M slices after it expired, so its
//                 age never reaches 255 and ids never alias (the per-slice
//                 maintenance of Sec. 5.2, spread over slices).
//   k_merge_stamp keeps, per counter, the youngest stamp over the routers
//                 (the OR of Sec. 4.2 for counters of a common slice clock).
//   k_tick        advances a router's slice clock by one.
// Every router's slice clock t lives in device memory and the kernels read
// it there, so the launches of a slice (slide, scan, detect) take the same
// arguments at every slice and can be recorded once in a CUDA graph and
// replayed slice after slice.
#include "sp_internal.h"

namespace sp {

namespace {

constexpr int kThreads = 256;

// id(t) = t mod 255 + 1 of the slice clock t
__device__ __forceinline__ uint32_t slice_id(const uint64_t* clock) { return (uint32_t)(*clock % 255u) + 1u; }

__device__ __forceinline__ uint32_t age_of(uint32_t stamp, uint32_t cur) {
  return cur >= stamp ? cur - stamp : cur + 255u - stamp;
}

// Segment (t mod M) of a router's stamps, M = 255 - k, of units16 16-byte
// units: reset those of age >= k (16 per uint4).
__global__ void __launch_bounds__(kThreads)
k_clean(uint4* __restrict__ st, uint64_t units16, const uint64_t* __restrict__ clock, uint32_t k) {
  const uint64_t t = *clock, M = 255u - k, seg = t % M;
  const uint64_t lo16 = units16 * seg / M, hi16 = units16 * (seg + 1) / M;
  const uint32_t cur = (uint32_t)(t % 255u) + 1u;
  const uint32_t cur4 = cur * 0x01010101u, k4 = k * 0x01010101u;
  for (uint64_t i = lo16 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi16;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 v = st[i];
    const uint4 o = make_uint4(v.x & active_mask4(v.x, cur4, k4), v.y & active_mask4(v.y, cur4, k4),
                               v.z & active_mask4(v.z, cur4, k4), v.w & active_mask4(v.w, cur4, k4));
    if (o.x != v.x || o.y != v.y || o.z != v.z || o.w != v.w) st[i] = o;
  }
}

// byte j of the result is 0xFF iff bit j of n is set (n < 16)
__device__ __forceinline__ uint32_t expand4(uint32_t n) {
  return ((n * 0x00204081u) & 0x01010101u) * 0xFFu;
}

// The 32 stamps of one sketch word (stamp j <-> bit j: eight 32-bit lanes of
// four stamps): id4 is written where the word's bits are set.
__device__ __forceinline__ void stamp_word(uint32_t bits, uint32_t (&v)[8], uint32_t id4) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const uint32_t m = expand4((bits >> (4 * q)) & 0xFu);
    v[q] = (v[q] & ~m) | (id4 & m);
  }
}

__device__ __forceinline__ void load8(const uint4* st, uint64_t i, uint32_t (&v)[8]) {
  const uint4 a = st[2 * i], b = st[2 * i + 1];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

__device__ __forceinline__ void store8(uint4* st, uint64_t i, const uint32_t (&v)[8]) {
  st[2 * i] = make_uint4(v[0], v[1], v[2], v[3]);
  st[2 * i + 1] = make_uint4(v[4], v[5], v[6], v[7]);
}

// Commit of one slice: every bit set in the slice's bit sketch stamps its
// counter with the slice id; counters of unset bits keep their stamp.  The
// slice sketch is consumed (nonzero words cleared), so the next updates of the
// router start a fresh slice sketch.  Zero words cost one 4-byte read.
__global__ void __launch_bounds__(kThreads)
k_commit(uint32_t* __restrict__ seav, uint4* __restrict__ st_seav, uint64_t seav_words,
         uint32_t* __restrict__ ldca, uint4* __restrict__ st_ldca, uint64_t ldca_words,
         const uint64_t* __restrict__ clock) {
  const uint32_t id4 = slice_id(clock) * 0x01010101u;
  const uint64_t n = seav_words + ldca_words;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
    const bool in_seav = j < seav_words;
    uint32_t* sk = in_seav ? seav : ldca;
    uint4* st = in_seav ? st_seav : st_ldca;
    const uint64_t i = in_seav ? j : j - seav_words;
    const uint32_t bits = sk[i];
    if (bits == 0u) continue;
    sk[i] = 0u;
    uint32_t v[8];
    load8(st, i, v);
    stamp_word(bits, v, id4);
    store8(st, i, v);
  }
}

// The same commit fused with the read of the window W(t, k): after stamping,
// bit j of the window word is set iff stamp j is active.  One streaming pass
// over the stamps (32 bytes per word) feeds the detect and export of a
// sliding router with an ordinary bit sketch.
__global__ void __launch_bounds__(kThreads)
k_commit_window(uint32_t* __restrict__ seav, uint4* __restrict__ st_seav, uint64_t seav_words,
                uint32_t* __restrict__ ldca, uint4* __restrict__ st_ldca, uint64_t ldca_words,
                uint32_t* __restrict__ wseav, uint32_t* __restrict__ wldca, const uint64_t* __restrict__ clock,
                uint32_t k) {
  const uint32_t id4 = slice_id(clock) * 0x01010101u, k4 = k * 0x01010101u;   // k <= 128 < 256
  const uint64_t n = seav_words + ldca_words;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
    const bool in_seav = j < seav_words;
    uint32_t* sk = in_seav ? seav : ldca;
    uint4* st = in_seav ? st_seav : st_ldca;
    uint32_t* w = in_seav ? wseav : wldca;
    const uint64_t i = in_seav ? j : j - seav_words;
    // the stamps are loaded with the slice word, not after it: one DRAM
    // round trip per word
    const uint32_t bits = sk[i];
    const uint4 a = __ldcs(st + 2 * i), b = __ldcs(st + 2 * i + 1);
    uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    if (bits != 0u) {
      sk[i] = 0u;
      stamp_word(bits, v, id4);
      store8(st, i, v);
    }
    uint32_t out = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) out |= active4(v[q], id4, k4) << (4 * q);
    w[i] = out;
  }
}

struct StampSrc {
  const uint4* p[32];
};

// dst = youngest stamp over dst and the sources (all at dst's slice clock)
__global__ void __launch_bounds__(kThreads)
k_merge_stamp(uint4* __restrict__ dst, StampSrc src, uint32_t n_src, uint64_t n16,
              const uint64_t* __restrict__ clock) {
  const uint32_t cur = slice_id(clock);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (uint64_t)gridDim.x * blockDim.x) {
    uint4 a = dst[i];
    uint32_t w[4] = {a.x, a.y, a.z, a.w};
    for (uint32_t s = 0; s < n_src; ++s) {
      const uint4 b = src.p[s][i];
      const uint32_t u[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t out = 0;
#pragma unroll
        for (int byte = 0; byte < 4; ++byte) {
          const uint32_t x = (w[q] >> (8 * byte)) & 0xFFu, y = (u[q] >> (8 * byte)) & 0xFFu;
          uint32_t pick;
          if (x == 0u) pick = y;
          else if (y == 0u) pick = x;
          else pick = age_of(y, cur) < age_of(x, cur) ? y : x;
          out |= pick << (8 * byte);
        }
        w[q] = out;
      }
    }
    dst[i] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

__global__ void k_tick(uint64_t* clock) { *clock += 1u; }

int grid_cap() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * 8;
}

unsigned grid_for(uint64_t work) {
  uint64_t g = (work + kThreads - 1) / kThreads;
  const uint64_t cap = (uint64_t)grid_cap();
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

cudaError_t launch_commit(uint32_t* seav, uint8_t* st_seav, uint64_t seav_words, uint32_t* ldca,
                          uint8_t* st_ldca, uint64_t ldca_words, const uint64_t* clock, cudaStream_t s) {
  k_commit<<<grid_for(seav_words + ldca_words), kThreads, 0, s>>>(
      seav, reinterpret_cast<uint4*>(st_seav), seav_words, ldca, reinterpret_cast<uint4*>(st_ldca), ldca_words,
      clock);
  return cudaGetLastError();
}

cudaError_t launch_commit_window(uint32_t* seav, uint8_t* st_seav, uint64_t seav_words, uint32_t* ldca,
                                 uint8_t* st_ldca, uint64_t ldca_words, uint32_t* wseav, uint32_t* wldca,
                                 const uint64_t* clock, uint32_t k, cudaStream_t s) {
  k_commit_window<<<grid_for(seav_words + ldca_words), kThreads, 0, s>>>(
      seav, reinterpret_cast<uint4*>(st_seav), seav_words, ldca, reinterpret_cast<uint4*>(st_ldca), ldca_words,
      wseav, wldca, clock, k);
  return cudaGetLastError();
}

cudaError_t launch_tick_clean(uint8_t* stamps, uint64_t bytes, uint64_t* clock, uint32_t k, cudaStream_t s) {
  k_tick<<<1, 1, 0, s>>>(clock);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const uint64_t units16 = bytes / 16, M = 255u - k;
  k_clean<<<grid_for(units16 / M + 1), kThreads, 0, s>>>(reinterpret_cast<uint4*>(stamps), units16, clock, k);
  return cudaGetLastError();
}

cudaError_t launch_merge_stamp(uint8_t* dst, const uint8_t* const* srcs, uint32_t n_src, uint64_t bytes,
                               const uint64_t* clock, cudaStream_t s) {
  const uint64_t n16 = bytes / 16;
  for (uint32_t base = 0; base < n_src; base += 32) {
    StampSrc l{};
    const uint32_t m = (n_src - base) < 32u ? (n_src - base) : 32u;
    for (uint32_t j = 0; j < m; ++j) l.p[j] = reinterpret_cast<const uint4*>(srcs[base + j]);
    k_merge_stamp<<<grid_for(n16), kThreads, 0, s>>>(reinterpret_cast<uint4*>(dst), l, m, n16, clock);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sp
