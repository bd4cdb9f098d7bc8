// sp_internal.h -- device-side parameter block and kernel launchers of the
// super point library (arXiv 1901.07306, Sec. 3-5).  Private to csrc/.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/superpoint.h"

namespace sp {

// Everything a kernel needs, derived once from sp_params at sp_create.
struct DevParams {
  uint64_t ha[10];          // multiply-add-shift words: 0 = H1, 1 = H3, 2 + i = LH_i
  uint64_t hb[10];
  uint32_t r;               // RP bits (Sec. 3.2)
  uint32_t L;               // LP bits = 32 - r
  uint32_t sr;              // SEA rows
  uint32_t tau;             // Eq. 1
  uint32_t k_log2;          // LDC bits (Sec. 3.3)
  uint32_t lr;              // LDCA rows
  uint32_t lc_log2;         // LDCA columns
  uint32_t sea_bytes;       // bytes of one SEA = sum SC(i)
  uint32_t isb[8];          // Def. 3
  uint32_t ibn[8];          // Def. 4
  uint32_t row_off[8];      // byte offset of row i inside an SEA
  uint32_t cover[8];        // LP bits covered by row i (Eq. 2), as a mask
  uint64_t seav_bytes;      // 2^r * sea_bytes
  uint64_t ldca_words;      // lr * LC * k / 32
};

// Detect status word, one per context, device resident.
struct DetectStatus {
  uint32_t count;           // super points found (may exceed the buffer)
  uint32_t overflow;        // bit 0: result buffer full, bit 1: join bound hit
  uint64_t join;            // LPs that reached the LDCA test
};

// Multiply-add-shift hash (Dietzfelbinger 1996): top 32 bits of
// (a * x + b) mod 2^64, written as one wide and one narrow multiply-add.
__host__ __device__ __forceinline__ uint32_t mas(uint64_t a, uint64_t b, uint32_t x) {
  const uint64_t lo = (uint64_t)(uint32_t)a * x + b;
  return (uint32_t)(lo >> 32) + (uint32_t)(a >> 32) * x;
}

// Places index bits of row i at their LP positions (inverse of Eq. 2,
// i.e. Eq. 3): index bit j goes to LP bit (isb + j) mod L.
__host__ __device__ __forceinline__ uint32_t spread_idx(uint32_t c, uint32_t isb, uint32_t L) {
  const uint64_t t = (uint64_t)c << isb;
  const uint64_t maskL = (L == 32) ? 0xFFFFFFFFull : ((1ull << L) - 1);
  return (uint32_t)((t | (t >> L)) & maskL);
}

// Eq. 2: Idx(i, LP) = bits isb .. isb + ibn - 1 of LP, cyclically mod L.
__host__ __device__ __forceinline__ uint32_t gather_idx(uint32_t lp, uint32_t isb, uint32_t ibn, uint32_t L) {
  const uint64_t twice = (uint64_t)lp | ((uint64_t)lp << L);
  return (uint32_t)(twice >> isb) & ((1u << ibn) - 1u);
}

// Up to kBinMaxSrc streams of one router, binned by one k_bin launch.
constexpr int kBinMaxSrc = 32;
struct BinSrc {
  const uint32_t* ptr[kBinMaxSrc];
  uint64_t n[kBinMaxSrc];
  uint32_t count;
};

// Staging shape of the binned scan (sp_scan_binned.cu); every compiled shape
// gives the same bits, the autotuner picks the fastest.
struct BinShape {
  uint32_t threads;             // k_bin block size
  uint32_t stage;               // staged hips per bin row
  uint32_t tpr;                 // tiles per flush round
  uint32_t per_sm;              // k_bin blocks per SM
  uint32_t apply_threads;       // k_apply block size
};
int binned_shape_count();
BinShape binned_shape(int i);   // i in [0, binned_shape_count()); 0 is the default

// Scratch of the binned scan (sp_scan_binned.cu), shared by a context's routers.
struct BinnedScratch {
  uint32_t* lists = nullptr;    // [bins][ctas][cap] hips
  uint32_t* counts = nullptr;   // [bins][ctas]
  uint32_t* planes = nullptr;   // plane accumulator of one router, [ceil(W / 8)][k][8] words, W = LR * LC / 32
  bool accumulate = false;      // planes hold earlier bits (load instead of zero)
  BinShape shape{};             // staging shape of the launches
  uint32_t ctas = 0;            // persistent binning blocks of this shape (SMs x per_sm)
  uint32_t cap_alloc = 0;       // hips per list the allocation holds at this shape: every cap is clamped to it
  uint64_t list_words = 0;      // hips the lists allocation holds
  uint64_t max_pairs = 0;       // pairs per binning round the lists are sized for
  int fold_grid = 0;
  uint32_t* ovf = nullptr;      // the router's flag: set when a pair's LDCA bit bypassed the lists
};

// ---- launchers (return cudaGetLastError() of the launch) -------------------
cudaError_t launch_zero(void* dev, uint64_t bytes, cudaStream_t s);
// launch_zero, and flags[0, n_flags) = 0 in the same launch
cudaError_t launch_zero_flags(void* dev, uint64_t bytes, uint32_t* flags, uint32_t n_flags, cudaStream_t s);
cudaError_t launch_scan(const DevParams& d, uint8_t* seav, uint32_t* ldca,
                        const uint32_t* pairs, uint64_t n_pairs, int grid, cudaStream_t s);
int scan_grid(const DevParams& d);
// batched direct scan over a device table of batches (sp_batch, include/superpoint.h)
cudaError_t launch_scan_multi(const DevParams& d, uint8_t* sketches, uint64_t stride, uint64_t seav_pad,
                              uint32_t n_routers, const sp_batch* desc, uint32_t n_batches, uint32_t* err,
                              int threads, int grid, cudaStream_t s);
int multi_max_grid(int threads);
bool binned_applicable(const DevParams& d);
// list capacity for a round of n_pairs binned by `chunks` launches of a shape
uint32_t binned_list_cap(uint64_t n_pairs, uint32_t bins, const BinShape& shape, uint32_t ctas, uint32_t chunks);
uint32_t binned_tile_pairs(const BinShape& shape);
// bytes of one router's plane accumulator ([ceil(W / 8)][k][8] words)
uint64_t binned_planes_bytes(const DevParams& d);
// one binning launch over pairs[0, n) into the lists (append: continue them)
cudaError_t binned_bin_chunk(const DevParams& d, uint8_t* seav, uint32_t* ldca, const BinSrc& src,
                             const BinnedScratch& s, uint32_t cap, bool append, uint32_t rot, cudaStream_t st);
BinSrc bin_src_one(const uint32_t* pairs, uint64_t n_pairs);
// the planes of the lists' hips (accumulate: on top of the pending planes)
cudaError_t binned_apply_round(const DevParams& d, const BinnedScratch& s, uint32_t cap, bool accumulate,
                               cudaStream_t st);
int binned_ctas(const BinShape& shape);
int binned_fold_grid();
// scan with the LDCA bits accumulated in s.planes (no fold)
cudaError_t launch_scan_binned(const DevParams& d, uint8_t* seav, uint32_t* ldca, const uint32_t* pairs,
                               uint64_t n_pairs, const BinnedScratch& s, cudaStream_t st);
// ldca |= transpose(planes)
// fresh: the router's flag (BinnedScratch::ovf) when its LDCA was zeroed
// and nothing but binned rounds wrote it since; the fold then writes the
// transposed planes without reading the LDCA, unless the flag is set.
// nullptr: ldca |= transpose(planes).
cudaError_t launch_fold(const DevParams& d, const uint32_t* planes, uint32_t* ldca, int grid, cudaStream_t st,
                        const uint32_t* fresh = nullptr);
// Sliding window stamps (Sec. 5.2): one byte per bit holding the id of the
// last slice that set it, id(t) = t mod 255 + 1 (0 = never set).  Byte j of
// active_mask4 is 0xFF iff byte j of s is an active stamp: non-zero, of age
// (cur - stamp) mod 255 below k (byte-wise SIMD: d = cur - s mod 256, and
// age = d - 1 where cur < s, the mod-255 wrap).  cur4 and k4 hold cur and k
// in every byte (k <= 128).
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

// The 32 active bits of one sketch word from its 32 stamps (two uint4).
__device__ __forceinline__ uint32_t active32(const uint4& a, const uint4& b, uint32_t cur4, uint32_t k4) {
  return active4(a.x, cur4, k4) | active4(a.y, cur4, k4) << 4 | active4(a.z, cur4, k4) << 8 |
         active4(a.w, cur4, k4) << 12 | active4(b.x, cur4, k4) << 16 | active4(b.y, cur4, k4) << 20 |
         active4(b.z, cur4, k4) << 24 | active4(b.w, cur4, k4) << 28;
}

// sliding window (sp_slide.cu); a sketch region is nw 32-bit words, word i
// owning the 32 stamps [32 i, 32 i + 32) of its stamp region; `clock` is the
// router's slice counter t in device memory (slice id t mod 255 + 1)
// stamps id(t) on the counters of the slice sketch's set bits, then clears the sketch
cudaError_t launch_commit(uint32_t* seav, uint8_t* st_seav, uint64_t seav_words, uint32_t* ldca,
                          uint8_t* st_ldca, uint64_t ldca_words, const uint64_t* clock, cudaStream_t s);
// launch_commit, and the window's bits (active stamps) into wseav / wldca
cudaError_t launch_commit_window(uint32_t* seav, uint8_t* st_seav, uint64_t seav_words, uint32_t* ldca,
                                 uint8_t* st_ldca, uint64_t ldca_words, uint32_t* wseav, uint32_t* wldca,
                                 const uint64_t* clock, uint32_t k, cudaStream_t s);
// t += 1, then the sweep of segment (t mod (255 - k)) of the router's stamps[0, bytes)
cudaError_t launch_tick_clean(uint8_t* stamps, uint64_t bytes, uint64_t* clock, uint32_t k, cudaStream_t s);
cudaError_t launch_merge_stamp(uint8_t* dst, const uint8_t* const* srcs, uint32_t n_src, uint64_t bytes,
                               const uint64_t* clock, cudaStream_t s);
cudaError_t launch_merge(uint8_t* dst, const uint8_t* const* srcs, uint32_t n_src,
                         uint64_t bytes, cudaStream_t s);
cudaError_t launch_detect(const DevParams& d, const uint8_t* seav, const uint32_t* ldca,
                          uint32_t z_theta, uint64_t* keys, uint32_t cap, uint64_t max_join,
                          DetectStatus* status, cudaStream_t s);
// The detect of a sliding router: seav is its window SEAV; an LDCA bit is in
// the window iff its stamp (st_ldca, one byte per bit) is active at the
// router's clock or it is set in the slice sketch ldca (not yet committed).
cudaError_t launch_detect_sliding(const DevParams& d, const uint8_t* seav, const uint32_t* ldca,
                                  const uint8_t* st_ldca, const uint64_t* clock, uint32_t k, uint32_t z_theta,
                                  uint64_t* keys, uint32_t cap, uint64_t max_join, DetectStatus* status,
                                  cudaStream_t s);
cudaError_t launch_sort_emit(uint64_t* keys, uint32_t cap, const DetectStatus* status,
                             const double* est_table, uint32_t k_log2,
                             sp_candidate* out, cudaStream_t s);

}  // namespace sp
