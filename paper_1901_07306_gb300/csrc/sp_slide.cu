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
//   k_scan_stamp  the scan of Sec. 3.1-3.3 with "set bit" replaced by
//                 "store id(t)": every writer of a location in one slice stores
//                 the same byte, so the update needs no atomics (Sec. 5.2:
//                 the counters run in parallel).
//   k_clean       at every slide, one of M = 255 - k segments of the counter
//                 pool is swept and counters of age >= k are reset to 0; each
//                 counter is swept at most M slices after it expired, so its
//                 age never reaches 255 and ids never alias (the per-slice
//                 maintenance of Sec. 5.2, spread over slices).
//   k_materialize writes the window's bits (active counters) into the
//                 ordinary SEAV/LDCA, which the detect of Sec. 3.2-3.3 reads.
//   k_merge_stamp keeps, per counter, the youngest stamp over the routers
//                 (the OR of Sec. 4.2 for counters of a common slice clock).
#include "sp_internal.h"

namespace sp {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint32_t age_of(uint32_t stamp, uint32_t cur) {
  return cur >= stamp ? cur - stamp : cur + 255u - stamp;
}

template <int LR>
__device__ __forceinline__ void stamp_pair(const DevParams& d, uint8_t* __restrict__ st_seav,
                                           uint8_t* __restrict__ st_ldca, uint32_t hip, uint32_t oip,
                                           uint32_t tau_mask, uint8_t id) {
  const uint32_t h1 = mas(d.ha[0], d.hb[0], oip);
  if ((h1 & tau_mask) == 0u) {                                 // lsb(H1) >= tau (Sec. 3.1)
    const uint32_t bit = h1 >> 29;
    const uint32_t rp = d.r ? (hip & ((1u << d.r) - 1u)) : 0u;
    const uint32_t lp = (uint32_t)((uint64_t)hip >> d.r);
    const uint64_t base = (uint64_t)rp * d.sea_bytes;
    for (uint32_t i = 0; i < d.sr; ++i) {
      const uint64_t se = base + d.row_off[i] + gather_idx(lp, d.isb[i], d.ibn[i], d.L);
      st_seav[se * 8u + bit] = id;
    }
  }
  const uint32_t h3 = mas(d.ha[1], d.hb[1], oip) >> (32u - d.k_log2);
  const uint32_t cshift = 32u - d.lc_log2;
#pragma unroll
  for (int i = 0; i < LR; ++i) {
    const uint32_t col = (uint32_t)((uint64_t)mas(d.ha[2 + i], d.hb[2 + i], hip) >> cshift);
    const uint64_t ldc = ((uint64_t)i << d.lc_log2) | col;
    st_ldca[(ldc << d.k_log2) | h3] = id;
  }
}

template <int LR>
__global__ void __launch_bounds__(kThreads)
k_scan_stamp(DevParams d, uint8_t* __restrict__ st_seav, uint8_t* __restrict__ st_ldca,
             const uint32_t* __restrict__ pairs, uint64_t n_pairs, uint32_t id) {
  const uint32_t tau_mask = (1u << d.tau) - 1u;
  const uint2* p2 = reinterpret_cast<const uint2*>(pairs);
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_pairs;
       j += (uint64_t)gridDim.x * blockDim.x) {
    const uint2 v = __ldcs(p2 + j);
    stamp_pair<LR>(d, st_seav, st_ldca, v.x, v.y, tau_mask, (uint8_t)id);
  }
}

// stamps[lo, hi): reset those of age >= k (16 per uint4)
__global__ void __launch_bounds__(kThreads)
k_clean(uint4* __restrict__ st, uint64_t lo16, uint64_t hi16, uint32_t cur, uint32_t k);

// Four stamps at once: byte j of the result is 0xFF iff byte j of s is an
// active stamp (non-zero, age (cur - stamp) mod 255 below k).  Byte-wise
// SIMD: d = cur - s mod 256, and age = d - 1 where cur < s (the mod-255 wrap).
__device__ __forceinline__ uint32_t active_mask4(uint32_t s, uint32_t cur4, uint32_t k4) {
  const uint32_t d = __vsub4(cur4, s);
  const uint32_t age = __vadd4(d, __vcmpltu4(cur4, s));       // + 0xFF = - 1 where cur < s
  return __vcmpltu4(age, k4) & ~__vcmpeq4(s, 0u);
}

// The same test as 4 bits (bit j for byte j): the four partial products of
// the multiply land on distinct bits 21..24, so nothing carries.
__device__ __forceinline__ uint32_t active4(uint32_t s, uint32_t cur4, uint32_t k4) {
  return (((active_mask4(s, cur4, k4) & 0x01010101u) * 0x00204081u) >> 21) & 0xFu;
}

__global__ void __launch_bounds__(kThreads)
k_clean(uint4* __restrict__ st, uint64_t lo16, uint64_t hi16, uint32_t cur, uint32_t k) {
  const uint32_t cur4 = cur * 0x01010101u, k4 = k * 0x01010101u;
  for (uint64_t i = lo16 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi16;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 v = st[i];
    const uint4 o = make_uint4(v.x & active_mask4(v.x, cur4, k4), v.y & active_mask4(v.y, cur4, k4),
                               v.z & active_mask4(v.z, cur4, k4), v.w & active_mask4(v.w, cur4, k4));
    if (o.x != v.x || o.y != v.y || o.z != v.z || o.w != v.w) st[i] = o;
  }
}

// SEAV bytes from 8 stamps each; LDCA words from 32 stamps each.
__global__ void __launch_bounds__(kThreads)
k_materialize(const uint2* __restrict__ st_seav, uint8_t* __restrict__ seav, uint64_t seav_bytes,
              const uint4* __restrict__ st_ldca, uint32_t* __restrict__ ldca, uint64_t ldca_words,
              uint32_t cur, uint32_t k) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t cur4 = cur * 0x01010101u, k4 = k * 0x01010101u;   // k <= 128 < 256
  for (uint64_t i = t0; i < seav_bytes; i += stride) {
    const uint2 v = __ldcs(st_seav + i);
    seav[i] = (uint8_t)(active4(v.x, cur4, k4) | (active4(v.y, cur4, k4) << 4));
  }
  for (uint64_t i = t0; i < ldca_words; i += stride) {
    const uint4 a = __ldcs(st_ldca + 2 * i), b = __ldcs(st_ldca + 2 * i + 1);
    ldca[i] = active4(a.x, cur4, k4) | (active4(a.y, cur4, k4) << 4) | (active4(a.z, cur4, k4) << 8) |
              (active4(a.w, cur4, k4) << 12) | (active4(b.x, cur4, k4) << 16) | (active4(b.y, cur4, k4) << 20) |
              (active4(b.z, cur4, k4) << 24) | (active4(b.w, cur4, k4) << 28);
  }
}

struct StampSrc {
  const uint4* p[32];
};

// dst = youngest stamp over dst and the sources (all at slice id `cur`)
__global__ void __launch_bounds__(kThreads)
k_merge_stamp(uint4* __restrict__ dst, StampSrc src, uint32_t n_src, uint64_t n16, uint32_t cur) {
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

cudaError_t launch_scan_stamp(const DevParams& d, uint8_t* st_seav, uint8_t* st_ldca, const uint32_t* pairs,
                              uint64_t n_pairs, uint32_t id, cudaStream_t s) {
  if (n_pairs == 0) return cudaSuccess;
  const unsigned g = grid_for(n_pairs);
  switch (d.lr) {
    case 1: k_scan_stamp<1><<<g, kThreads, 0, s>>>(d, st_seav, st_ldca, pairs, n_pairs, id); break;
    case 2: k_scan_stamp<2><<<g, kThreads, 0, s>>>(d, st_seav, st_ldca, pairs, n_pairs, id); break;
    case 3: k_scan_stamp<3><<<g, kThreads, 0, s>>>(d, st_seav, st_ldca, pairs, n_pairs, id); break;
    case 4: k_scan_stamp<4><<<g, kThreads, 0, s>>>(d, st_seav, st_ldca, pairs, n_pairs, id); break;
    case 5: k_scan_stamp<5><<<g, kThreads, 0, s>>>(d, st_seav, st_ldca, pairs, n_pairs, id); break;
    case 6: k_scan_stamp<6><<<g, kThreads, 0, s>>>(d, st_seav, st_ldca, pairs, n_pairs, id); break;
    case 7: k_scan_stamp<7><<<g, kThreads, 0, s>>>(d, st_seav, st_ldca, pairs, n_pairs, id); break;
    default: k_scan_stamp<8><<<g, kThreads, 0, s>>>(d, st_seav, st_ldca, pairs, n_pairs, id); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_clean(uint8_t* stamps, uint64_t lo, uint64_t hi, uint32_t cur, uint32_t k, cudaStream_t s) {
  const uint64_t lo16 = lo / 16, hi16 = hi / 16;
  if (hi16 <= lo16) return cudaSuccess;
  k_clean<<<grid_for(hi16 - lo16), kThreads, 0, s>>>(reinterpret_cast<uint4*>(stamps), lo16, hi16, cur, k);
  return cudaGetLastError();
}

cudaError_t launch_materialize(const uint8_t* st_seav, uint8_t* seav, uint64_t seav_bytes, const uint8_t* st_ldca,
                               uint32_t* ldca, uint64_t ldca_words, uint32_t cur, uint32_t k, cudaStream_t s) {
  const uint64_t work = seav_bytes > ldca_words ? seav_bytes : ldca_words;
  k_materialize<<<grid_for(work), kThreads, 0, s>>>(reinterpret_cast<const uint2*>(st_seav), seav, seav_bytes,
                                                   reinterpret_cast<const uint4*>(st_ldca), ldca, ldca_words, cur, k);
  return cudaGetLastError();
}

cudaError_t launch_merge_stamp(uint8_t* dst, const uint8_t* const* srcs, uint32_t n_src, uint64_t bytes,
                               uint32_t cur, cudaStream_t s) {
  const uint64_t n16 = bytes / 16;
  for (uint32_t base = 0; base < n_src; base += 32) {
    StampSrc l{};
    const uint32_t m = (n_src - base) < 32u ? (n_src - base) : 32u;
    for (uint32_t j = 0; j < m; ++j) l.p[j] = reinterpret_cast<const uint4*>(srcs[base + j]);
    k_merge_stamp<<<grid_for(n16), kThreads, 0, s>>>(reinterpret_cast<uint4*>(dst), l, m, n16, cur);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sp
