// sp_api.cu -- host side of the C ABI declared in include/superpoint.h.
//
// Owns the per-context device memory (n_routers sketches, detect scratch,
// staging buffers for the host path), validates parameters against Sec. 3.2's
// constraints, derives the hash words from the seed, and enqueues the kernels
// of sp_scan.cu, sp_merge.cu and sp_detect.cu on the context's stream.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <new>
#include <thread>
#include <vector>

#include "sp_internal.h"

using sp::DetectStatus;
using sp::DevParams;

namespace {

constexpr uint64_t kDefaultMaxCandidates = 1ull << 20;
constexpr uint64_t kDefaultMaxJoin = 1ull << 26;
constexpr uint64_t kStagingPairs = 1ull << 22;      // 32 MiB per staging buffer
constexpr uint64_t kBinnedMinPairs = 1ull << 22;    // auto mode: smaller updates go direct
constexpr uint64_t kBinnedRoundPairs = 1ull << 26;  // pairs per binning round
// Host-path binning rounds: each round's plane pass overlaps the next round's
// copies, so after the last copy only one round of 2^24 pairs is left to apply.
constexpr uint64_t kHostRoundPairs = 1ull << 24;
constexpr uint32_t kResultPrefix = 4096;            // records fetched with the status
constexpr uint32_t kDefaultTimeoutMs = 60000;       // bound of every wait on the stream
constexpr uint64_t kAlign = 256;

uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// SplitMix64 (Steele, Lea, Flood 2014).
uint64_t splitmix64_next(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

bool row_covers(uint32_t isb, uint32_t ibn, uint32_t L, uint32_t bit) {
  // is LP bit `bit` one of isb, isb + 1, ..., isb + ibn - 1 (mod L)?
  const uint32_t d = (bit + L - isb) % L;
  return d < ibn;
}

uint64_t sea_bytes_of(const sp_params* p) {
  uint64_t s = 0;
  for (uint32_t i = 0; i < p->sr; ++i) s += 1ull << p->ibn[i];
  return s;
}

uint32_t log2_ceil_u64(uint64_t x) {
  uint32_t b = 0;
  while ((1ull << b) < x) ++b;
  return b;
}

// 64-bit FNV-1a over bytes.
uint64_t fnv1a64(const void* data, uint64_t n, uint64_t h = 0xCBF29CE484222325ull) {
  const uint8_t* p = static_cast<const uint8_t*>(data);
  for (uint64_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 0x100000001B3ull;
  }
  return h;
}

struct ImageHeader {
  char magic[8];             // "SPSKETCH"
  uint32_t version;          // 1
  uint32_t header_bytes;     // sizeof(ImageHeader)
  uint32_t r, sr, isb[8], ibn[8], k_log2, lr, lc_log2, theta;
  uint64_t seed;
  uint64_t seav_bytes, ldca_bytes;
};

}  // namespace

struct sp_ctx {
  sp_params p;
  DevParams d;
  cudaStream_t stream = nullptr;
  int device = 0;
  int scan_grid = 0;
  uint64_t seav_bytes = 0, ldca_bytes = 0, seav_pad = 0, stride = 0;
  uint8_t* sketches = nullptr;              // n_routers * stride bytes
  uint64_t* keys = nullptr;                 // detect scratch: next_pow2(cap) keys
  sp_candidate* records = nullptr;          // sorted results, cap records
  DetectStatus* status = nullptr;
  uint32_t* kerr = nullptr;                 // kernel error word (bad device batch table entries)
  double* est_table = nullptr;              // -k ln(z / k), z = 0 .. k
  uint32_t cap = 0;
  uint32_t timeout_ms = kDefaultTimeoutMs;  // 0: waits are unbounded
  cudaEvent_t ev_wait = nullptr;            // marks the stream's work for a bounded wait
  cudaEvent_t ev_arena = nullptr;           // sp_update_batched_host: the copies into the arena are done
  bool detect_issued = false;
  uint32_t last_threshold = 0;
  // results: status, error word and the first kResultPrefix records land in
  // one pinned buffer with a single wait
  uint8_t* result_host = nullptr;
  // host path (Sec. 4.1): two staging buffers and a copy stream
  uint32_t* staging[2] = {nullptr, nullptr};
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  cudaEvent_t ev_free[2] = {nullptr, nullptr};
  // binned scan: shared lists, one plane-major accumulator per router
  sp::BinnedScratch bs;
  uint32_t** planes = nullptr;              // [n_routers], lazily allocated
  bool* planes_dirty = nullptr;             // bits not yet folded into the LDCA
  // ldca_zero[r]: since r's last zeroing only binned rounds wrote its LDCA
  // (discrete contexts), so the next fold may write the planes without
  // reading the LDCA -- unless a binning launch spilled a bit past a full
  // list, which sets the device flag ovf[r] (cleared with the zeroing)
  bool* ldca_zero = nullptr;
  uint32_t* ovf = nullptr;
  // sliding window (Sec. 5): one stamp byte per bit, per-router slice clock;
  // the bit sketch of a sliding router holds the current slice's bits until
  // they are committed to the stamps
  bool sliding = false;
  bool* slice_dirty = nullptr;              // slice bits not yet committed
  uint8_t* stamps = nullptr;                // n_routers * st_stride bytes
  uint8_t* window = nullptr;                // n_routers * stride: the window's bits, rebuilt per read
  uint64_t st_seav_pad = 0, st_stride = 0;
  uint64_t* slice = nullptr;                // host count of sp_slide calls per router (merge's same-slice check)

  // batched scan: a ring of batch tables (pinned host copy, device copy), so
  // the host waits only for the upload issued kTableRing calls earlier
  struct TableSlot {
    sp_batch* host = nullptr;
    sp_batch* dev = nullptr;
    uint32_t cap = 0;
    cudaEvent_t ev = nullptr;               // this slot's last upload has left `host`
    bool pending = false;
  };
  static constexpr int kTableRing = 4;
  TableSlot tables[kTableRing];
  uint32_t table_next = 0;
  int multi_threads = 256;
  int multi_grid = 0;
  uint32_t bs_shape_index = 0;              // staging shape of the binned scan (sp_autotune_binned)

  uint8_t* st_seav(uint32_t router) const { return stamps + (uint64_t)router * st_stride; }
  uint8_t* st_ldca(uint32_t router) const { return stamps + (uint64_t)router * st_stride + st_seav_pad; }
  uint64_t* clock = nullptr;                // device: slice counter t of each router (the kernels' clock)
  uint64_t* dev_clock(uint32_t router) const { return clock + router; }
  // SEAV as 32-bit words (the padding past seav_bytes is zero in every region)
  uint64_t seav_words() const { return (seav_bytes + 3) / 4; }

  uint8_t* seav(uint32_t router) const { return sketches + (uint64_t)router * stride; }
  uint8_t* wseav(uint32_t router) const { return window + (uint64_t)router * stride; }
  uint32_t* wldca(uint32_t router) const { return reinterpret_cast<uint32_t*>(window + (uint64_t)router * stride + seav_pad); }
  uint32_t* ldca(uint32_t router) const { return reinterpret_cast<uint32_t*>(sketches + (uint64_t)router * stride + seav_pad); }
};

// Polls an event that was recorded on the context's stream until it has
// completed, or until the context's bound has passed (SP_ERR_TIMEOUT; the
// work stays in flight and a later wait may collect it).  No failure
// detection of this kind is in the paper: it keeps a host thread from
// waiting forever on a stream that stopped making progress.
static int wait_event_bounded(const sp_ctx* ctx, cudaEvent_t ev) {
  // the first 20 ms poll with yields only (a sleep can last far longer than
  // asked for, which would add to every detect's latency); longer waits
  // sleep between polls
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t q = cudaEventQuery(ev);
    if (q == cudaSuccess) return SP_OK;
    if (q != cudaErrorNotReady) {
      cudaGetLastError();
      return SP_ERR_CUDA;
    }
    if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();   // not an error: keep launches' checks clean
    const auto waited = std::chrono::steady_clock::now() - t0;
    if (ctx->timeout_ms && waited >= std::chrono::milliseconds(ctx->timeout_ms)) return SP_ERR_TIMEOUT;
    if (waited < std::chrono::milliseconds(20)) std::this_thread::yield();
    else std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
}

// Bounded wait for all work issued on the context's stream so far.
static int wait_stream(sp_ctx* ctx) {
  if (cudaEventRecord(ctx->ev_wait, ctx->stream) != cudaSuccess) return SP_ERR_CUDA;
  return wait_event_bounded(ctx, ctx->ev_wait);
}

extern "C" {

int sp_version(void) { return 1 * 10000 + 0 * 100 + 0; }

const char* sp_strerror(int code) {
  switch (code) {
    case SP_OK: return "ok";
    case SP_WARN_THETA_BELOW_INIT: return "warning: detect threshold below the theta that fixed tau";
    case SP_ERR_PARAM: return "invalid argument or parameter set";
    case SP_ERR_ROUTER: return "router index out of range";
    case SP_ERR_TRUNCATED: return "more results than the output capacity";
    case SP_ERR_CANDIDATE_OVERFLOW: return "candidate buffer or join bound overflowed; results incomplete";
    case SP_ERR_CUDA: return "CUDA runtime error";
    case SP_ERR_TIMEOUT: return "bounded wait timed out";
    case SP_ERR_CHECKSUM: return "sketch image checksum or parameter mismatch";
    case SP_ERR_NOMEM: return "allocation failed";
    case SP_ERR_STATE: return "call not valid in the current state";
    default: return "unknown status";
  }
}

int sp_default_params(sp_params* out) {
  if (!out) return SP_ERR_PARAM;
  memset(out, 0, sizeof(*out));
  out->r = 14;
  out->sr = 4;
  const uint32_t L = 32 - out->r, step = (L + out->sr - 1) / out->sr, a = 2;
  for (uint32_t i = 0; i < out->sr; ++i) {
    out->isb[i] = i * step;
    out->ibn[i] = step + a;
  }
  out->k_log2 = 10;
  out->lr = 4;
  out->lc_log2 = 16;
  out->theta = 1024;
  out->n_routers = 1;
  out->window_slices = 1;
  out->max_candidates = 0;
  out->seed = 0x5EED;
  out->max_join = 0;
  return SP_OK;
}

int sp_check_params(const sp_params* p) {
  if (!p) return SP_ERR_PARAM;
  if (p->r > 24 || p->sr < 1 || p->sr > 8) return SP_ERR_PARAM;
  const uint32_t L = 32 - p->r;
  for (uint32_t i = 0; i < p->sr; ++i) {
    if (p->ibn[i] < 1 || p->ibn[i] > 12 || p->ibn[i] > L || p->isb[i] >= L) return SP_ERR_PARAM;
  }
  if (sea_bytes_of(p) > 4096) return SP_ERR_PARAM;
  // constraint 1 (Sec. 3.2): every LP bit lies in some row's index
  for (uint32_t bit = 0; bit < L; ++bit) {
    bool covered = false;
    for (uint32_t i = 0; i < p->sr && !covered; ++i) covered = row_covers(p->isb[i], p->ibn[i], L, bit);
    if (!covered) return SP_ERR_PARAM;
  }
  // constraint 2 (Sec. 3.2), read as: row i shares an LP bit with row i + 1 mod SR
  if (p->sr > 1) {
    for (uint32_t i = 0; i < p->sr; ++i) {
      const uint32_t n = (i + 1) % p->sr;
      bool shared = false;
      for (uint32_t bit = 0; bit < L && !shared; ++bit)
        shared = row_covers(p->isb[i], p->ibn[i], L, bit) && row_covers(p->isb[n], p->ibn[n], L, bit);
      if (!shared) return SP_ERR_PARAM;
    }
  }
  if (p->k_log2 < 5 || p->k_log2 > 16) return SP_ERR_PARAM;
  if (p->lr < 1 || p->lr > 8 || p->lc_log2 > 24) return SP_ERR_PARAM;
  if ((uint64_t)p->lr << (p->lc_log2 + p->k_log2) > (1ull << 32)) return SP_ERR_PARAM;
  if (p->theta == 0) return SP_ERR_PARAM;
  if (p->n_routers < 1 || p->n_routers > 4096) return SP_ERR_PARAM;
  if (p->window_slices < 1 || p->window_slices > 128) return SP_ERR_PARAM;
  if (p->scan_mode > SP_SCAN_BINNED) return SP_ERR_PARAM;
  return SP_OK;
}

int sp_sketch_bytes(const sp_params* p, uint64_t* seav_bytes, uint64_t* ldca_bytes) {
  if (sp_check_params(p) != SP_OK) return SP_ERR_PARAM;
  if (seav_bytes) *seav_bytes = sea_bytes_of(p) << p->r;
  if (ldca_bytes) *ldca_bytes = ((uint64_t)p->lr << (p->lc_log2 + p->k_log2)) / 8;
  return SP_OK;
}

uint32_t sp_tau(uint32_t theta) {
  // Eq. 1: tau = ceil(log2(theta / 8)), at least 0: smallest t with 8 * 2^t >= theta
  uint32_t t = 0;
  while (t < 29 && (8ull << t) < (uint64_t)theta) ++t;
  return t;
}

static double est_of(uint32_t k_log2, uint32_t z) {
  const double k = (double)(1ull << k_log2);
  return -k * log((double)z / k);   // Eq. 4
}

uint32_t sp_z_theta(uint32_t k_log2, uint32_t threshold) {
  const uint32_t k = 1u << k_log2;
  for (uint32_t z = k; z > 0; --z)
    if (est_of(k_log2, z) >= (double)threshold) return z;
  return 0;
}

double sp_psu(uint64_t n_pairs, uint32_t k_log2, uint32_t lr, uint32_t lc_log2) {
  const double k = (double)(1ull << k_log2);
  const double zero_in_one_ldc = pow(1.0 - 1.0 / k, (double)n_pairs / (double)(1ull << lc_log2));
  return pow(1.0 - zero_in_one_ldc, (double)lr);
}

int sp_size_ldca(uint64_t n_pairs, uint32_t k_log2, uint64_t ldc_budget, uint32_t* lr, uint32_t* lc_log2,
                 double* psu, double* lr_star) {
  if (n_pairs == 0 || k_log2 < 5 || k_log2 > 16 || ldc_budget == 0) return SP_ERR_PARAM;
  double best = 2.0;
  uint32_t best_lr = 1, best_c = 0;
  for (uint32_t rows = 1; rows <= 8; ++rows) {
    for (uint32_t c = 0; c <= 24; ++c) {
      if ((uint64_t)rows << c > ldc_budget) break;
      if (((uint64_t)rows << (c + k_log2)) > (1ull << 32)) break;
      const double v = sp_psu(n_pairs, k_log2, rows, c);
      if (v < best) { best = v; best_lr = rows; best_c = c; }
    }
  }
  if (lr) *lr = best_lr;
  if (lc_log2) *lc_log2 = best_c;
  if (psu) *psu = best;
  if (lr_star) {
    const double k = (double)(1ull << k_log2);
    *lr_star = -(double)ldc_budget * log(2.0) / ((double)n_pairs * log(1.0 - 1.0 / k));
  }
  return SP_OK;
}

void sp_destroy(sp_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->copy_stream) {
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamDestroy(ctx->copy_stream);
  }
  for (int i = 0; i < 2; ++i) {
    if (ctx->ev_copied[i]) cudaEventDestroy(ctx->ev_copied[i]);
    if (ctx->ev_free[i]) cudaEventDestroy(ctx->ev_free[i]);
    if (ctx->staging[i]) cudaFree(ctx->staging[i]);
  }
  if (ctx->planes) {
    for (uint32_t r = 0; r < ctx->p.n_routers; ++r) cudaFree(ctx->planes[r]);
    free(ctx->planes);
  }
  free(ctx->planes_dirty);
  free(ctx->slice);
  cudaFree(ctx->clock);
  free(ctx->slice_dirty);
  if (ctx->result_host) cudaFreeHost(ctx->result_host);
  for (auto& t : ctx->tables) {
    if (t.host) cudaFreeHost(t.host);
    cudaFree(t.dev);
    if (t.ev) cudaEventDestroy(t.ev);
  }
  cudaFree(ctx->stamps);
  cudaFree(ctx->window);
  cudaFree(ctx->bs.lists);
  cudaFree(ctx->bs.counts);
  cudaFree(ctx->ovf);
  free(ctx->ldca_zero);
  cudaFree(ctx->sketches);
  cudaFree(ctx->keys);
  cudaFree(ctx->records);
  cudaFree(ctx->status);
  cudaFree(ctx->kerr);
  cudaFree(ctx->est_table);
  if (ctx->ev_wait) cudaEventDestroy(ctx->ev_wait);
  if (ctx->ev_arena) cudaEventDestroy(ctx->ev_arena);
  delete ctx;
}

int sp_create(const sp_params* p, void* cuda_stream, sp_ctx** out) {
  if (!out) return SP_ERR_PARAM;
  *out = nullptr;
  if (sp_check_params(p) != SP_OK) return SP_ERR_PARAM;
  sp_ctx* c = new (std::nothrow) sp_ctx();
  if (!c) return SP_ERR_NOMEM;
  c->p = *p;
  if (c->p.max_candidates == 0) c->p.max_candidates = (uint32_t)kDefaultMaxCandidates;
  if (c->p.max_join == 0) c->p.max_join = kDefaultMaxJoin;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&c->device);

  DevParams& d = c->d;
  memset(&d, 0, sizeof(d));
  uint64_t s = p->seed;
  for (uint32_t i = 0; i < 2 + p->lr; ++i) {
    d.ha[i] = splitmix64_next(&s);
    d.hb[i] = splitmix64_next(&s);
  }
  d.r = p->r;
  d.L = 32 - p->r;
  d.sr = p->sr;
  d.tau = sp_tau(p->theta);
  d.k_log2 = p->k_log2;
  d.lr = p->lr;
  d.lc_log2 = p->lc_log2;
  uint32_t off = 0;
  for (uint32_t i = 0; i < p->sr; ++i) {
    d.isb[i] = p->isb[i];
    d.ibn[i] = p->ibn[i];
    d.row_off[i] = off;
    d.cover[i] = sp::spread_idx((1u << p->ibn[i]) - 1u, p->isb[i], d.L);
    off += 1u << p->ibn[i];
  }
  d.sea_bytes = off;
  sp_sketch_bytes(p, &c->seav_bytes, &c->ldca_bytes);
  d.seav_bytes = c->seav_bytes;
  d.ldca_words = c->ldca_bytes / 4;
  c->seav_pad = align_up(c->seav_bytes, kAlign);
  c->stride = c->seav_pad + align_up(c->ldca_bytes, kAlign);
  c->cap = c->p.max_candidates;
  const uint64_t key_slots = 1ull << log2_ceil_u64(c->cap);

  int rc = SP_OK;
  if (cudaMalloc(&c->sketches, c->stride * p->n_routers) != cudaSuccess ||
      cudaMalloc(&c->keys, key_slots * sizeof(uint64_t)) != cudaSuccess ||
      cudaMalloc(&c->records, (uint64_t)c->cap * sizeof(sp_candidate)) != cudaSuccess ||
      cudaMalloc(&c->status, sizeof(DetectStatus)) != cudaSuccess ||
      cudaMalloc(&c->kerr, sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&c->ovf, sizeof(uint32_t) * p->n_routers) != cudaSuccess ||
      cudaMalloc(&c->est_table, ((1ull << p->k_log2) + 1) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    rc = SP_ERR_NOMEM;
  }
  if (rc == SP_OK && cudaEventCreateWithFlags(&c->ev_wait, cudaEventDisableTiming) != cudaSuccess) rc = SP_ERR_CUDA;
  if (rc == SP_OK) {
    const uint32_t k = 1u << p->k_log2;
    double* table = static_cast<double*>(malloc((k + 1) * sizeof(double)));
    if (!table) rc = SP_ERR_NOMEM;
    else {
      table[0] = (double)k * log((double)k);   // saturated union: reported as k ln k
      for (uint32_t z = 1; z <= k; ++z) table[z] = est_of(p->k_log2, z);
      if (cudaMemcpy(c->est_table, table, (k + 1) * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = SP_ERR_CUDA;
      free(table);
    }
  }
  if (rc == SP_OK && sp::launch_zero_flags(c->sketches, c->stride * p->n_routers, c->ovf, p->n_routers, c->stream) !=
                         cudaSuccess)
    rc = SP_ERR_CUDA;
  if (rc == SP_OK && cudaMemsetAsync(c->status, 0, sizeof(DetectStatus), c->stream) != cudaSuccess) rc = SP_ERR_CUDA;
  if (rc == SP_OK && cudaMemsetAsync(c->kerr, 0, sizeof(uint32_t), c->stream) != cudaSuccess) rc = SP_ERR_CUDA;
  if (rc == SP_OK) {
    c->scan_grid = sp::scan_grid(d);
    c->multi_grid = sp::multi_max_grid(c->multi_threads);
    c->planes = static_cast<uint32_t**>(calloc(p->n_routers, sizeof(uint32_t*)));
    c->planes_dirty = static_cast<bool*>(calloc(p->n_routers, sizeof(bool)));
    c->ldca_zero = static_cast<bool*>(calloc(p->n_routers, sizeof(bool)));
    if (c->ldca_zero && p->window_slices <= 1)
      for (uint32_t r = 0; r < p->n_routers; ++r) c->ldca_zero[r] = true;
    c->slice = static_cast<uint64_t*>(calloc(p->n_routers, sizeof(uint64_t)));
    c->slice_dirty = static_cast<bool*>(calloc(p->n_routers, sizeof(bool)));
    if (!c->planes || !c->planes_dirty || !c->slice || !c->slice_dirty || !c->ldca_zero) rc = SP_ERR_NOMEM;
  }
  if (rc == SP_OK && p->window_slices > 1) {
    c->sliding = true;
    c->st_seav_pad = align_up(c->seav_bytes * 8, kAlign);
    c->st_stride = c->st_seav_pad + align_up(c->ldca_bytes * 8, kAlign);
    if (cudaMalloc(&c->stamps, c->st_stride * p->n_routers) != cudaSuccess ||
        cudaMalloc(&c->window, c->stride * p->n_routers) != cudaSuccess ||
        cudaMalloc(&c->clock, sizeof(uint64_t) * p->n_routers) != cudaSuccess) { cudaGetLastError(); rc = SP_ERR_NOMEM; }
    else if (sp::launch_zero(c->stamps, c->st_stride * p->n_routers, c->stream) != cudaSuccess ||
             cudaMemsetAsync(c->clock, 0, sizeof(uint64_t) * p->n_routers, c->stream) != cudaSuccess) rc = SP_ERR_CUDA;
  }
  if (rc == SP_OK) rc = wait_stream(c);
  if (rc != SP_OK) {
    sp_destroy(c);
    return rc;
  }
  *out = c;
  return SP_OK;
}

int sp_set_stream(sp_ctx* ctx, void* cuda_stream) {
  if (!ctx) return SP_ERR_PARAM;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return SP_OK;
}

int sp_set_timeout(sp_ctx* ctx, uint32_t timeout_ms) {
  if (!ctx) return SP_ERR_PARAM;
  ctx->timeout_ms = timeout_ms;
  return SP_OK;
}

int sp_get_params(const sp_ctx* ctx, sp_params* out) {
  if (!ctx || !out) return SP_ERR_PARAM;
  *out = ctx->p;
  return SP_OK;
}

// Folds a router's pending binned-scan planes into its LDCA.
static int fold_router(sp_ctx* ctx, uint32_t router) {
  if (!ctx->planes_dirty[router]) return SP_OK;
  const uint32_t* fresh = ctx->ldca_zero[router] ? ctx->ovf + router : nullptr;
  if (sp::launch_fold(ctx->d, ctx->planes[router], ctx->ldca(router), ctx->bs.fold_grid, ctx->stream, fresh) !=
      cudaSuccess)
    return SP_ERR_CUDA;
  ctx->planes_dirty[router] = false;
  ctx->ldca_zero[router] = false;
  return SP_OK;
}

// Selects a staging shape of the binned scan: its block count and the list
// capacity the allocation gives it.
static void set_binned_shape(sp_ctx* ctx, int index) {
  ctx->bs.shape = sp::binned_shape(index);
  ctx->bs_shape_index = (uint32_t)index;
  ctx->bs.ctas = (uint32_t)sp::binned_ctas(ctx->bs.shape);
  const uint64_t per_list = ctx->bs.list_words / ((uint64_t)(1u << ctx->p.k_log2) * ctx->bs.ctas);
  ctx->bs.cap_alloc = (uint32_t)((per_list > 0xFFFFFFF8ull ? 0xFFFFFFF8ull : per_list) & ~7ull);
}

static int ensure_binned(sp_ctx* ctx, uint32_t router) {
  if (!ctx->bs.lists) {
    ctx->bs.max_pairs = kBinnedRoundPairs;
    ctx->bs.fold_grid = sp::binned_fold_grid();
    const uint32_t bins = 1u << ctx->p.k_log2;
    // room for the largest round of every shape: max_pairs split into host staging chunks
    const uint32_t chunks = (uint32_t)((ctx->bs.max_pairs + kStagingPairs - 1) / kStagingPairs);
    uint64_t words = 0, max_ctas = 0;
    for (int i = 0; i < sp::binned_shape_count(); ++i) {
      const sp::BinShape h = sp::binned_shape(i);
      const uint64_t ctas = (uint64_t)sp::binned_ctas(h);
      const uint64_t w = (uint64_t)bins * ctas * sp::binned_list_cap(ctx->bs.max_pairs, bins, h, (uint32_t)ctas, chunks);
      if (w > words) words = w;
      if (ctas > max_ctas) max_ctas = ctas;
    }
    if (words >= (1ull << 32)) return SP_ERR_PARAM;   // 32-bit list slots
    ctx->bs.list_words = words;
    if (cudaMalloc(&ctx->bs.lists, words * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&ctx->bs.counts, (uint64_t)bins * max_ctas * sizeof(uint32_t)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(ctx->bs.lists);
      ctx->bs.lists = nullptr;
      return SP_ERR_NOMEM;
    }
    set_binned_shape(ctx, (int)ctx->bs_shape_index);
  }
  if (!ctx->planes[router]) {
    if (cudaMalloc(&ctx->planes[router], sp::binned_planes_bytes(ctx->d)) != cudaSuccess) {
      cudaGetLastError();
      return SP_ERR_NOMEM;
    }
    ctx->planes_dirty[router] = false;
  }
  return SP_OK;
}

// Whether an update of n pairs takes the binned scan.
static bool use_binned(const sp_ctx* ctx, uint64_t n_pairs) {
  if (!sp::binned_applicable(ctx->d)) return false;
  if (ctx->p.scan_mode == SP_SCAN_BINNED) return true;
  return ctx->p.scan_mode == SP_SCAN_AUTO && n_pairs >= kBinnedMinPairs;
}

static sp::BinnedScratch binned_scratch(const sp_ctx* ctx, uint32_t router) {
  sp::BinnedScratch s = ctx->bs;
  s.planes = ctx->planes[router];
  s.accumulate = ctx->planes_dirty[router];
  s.ovf = ctx->ovf + router;
  return s;
}

// One update of one router through the direct or the binned scan.
static int do_update(sp_ctx* ctx, uint32_t router, const uint32_t* dev_pairs, uint64_t n_pairs) {
  ctx->slice_dirty[router] = true;
  if (use_binned(ctx, n_pairs)) {
    int rc = ensure_binned(ctx, router);
    if (rc != SP_OK) return rc;
    sp::BinnedScratch s = binned_scratch(ctx, router);
    if (sp::launch_scan_binned(ctx->d, ctx->seav(router), ctx->ldca(router), dev_pairs, n_pairs, s,
                               ctx->stream) != cudaSuccess) return SP_ERR_CUDA;
    ctx->planes_dirty[router] = true;
    return SP_OK;
  }
  ctx->ldca_zero[router] = false;
  return sp::launch_scan(ctx->d, ctx->seav(router), ctx->ldca(router), dev_pairs, n_pairs,
                         ctx->scan_grid, ctx->stream) == cudaSuccess ? SP_OK : SP_ERR_CUDA;
}

// Sliding contexts: stamps the router's pending slice bits with the current
// slice id and clears its bit sketch (Sec. 5.2).  The close of a slice and a
// merge commit first.
static int commit(sp_ctx* ctx, uint32_t router) {
  if (!ctx->sliding) return SP_OK;
  int rc = fold_router(ctx, router);
  if (rc != SP_OK || !ctx->slice_dirty[router]) return rc;
  if (sp::launch_commit(reinterpret_cast<uint32_t*>(ctx->seav(router)), ctx->st_seav(router), ctx->seav_words(),
                        ctx->ldca(router), ctx->st_ldca(router), ctx->ldca_bytes / 4, ctx->dev_clock(router),
                        ctx->stream) != cudaSuccess)
    return SP_ERR_CUDA;
  ctx->slice_dirty[router] = false;
  return SP_OK;
}

// Sliding contexts: commit, and the window's bits into the router's window
// image (what detect and export read).
static int commit_window(sp_ctx* ctx, uint32_t router) {
  int rc = fold_router(ctx, router);
  if (rc != SP_OK) return rc;
  if (sp::launch_commit_window(reinterpret_cast<uint32_t*>(ctx->seav(router)), ctx->st_seav(router),
                               ctx->seav_words(), ctx->ldca(router), ctx->st_ldca(router), ctx->ldca_bytes / 4,
                               reinterpret_cast<uint32_t*>(ctx->wseav(router)), ctx->wldca(router),
                               ctx->dev_clock(router), ctx->p.window_slices, ctx->stream) != cudaSuccess)
    return SP_ERR_CUDA;
  ctx->slice_dirty[router] = false;
  return SP_OK;
}

// Sliding contexts, before a detect: commits the slice's SEAV bits and
// writes the window SEAV (one pass over the SEAV stamps).  The slice's LDCA
// bits stay in the bit sketch until the slice closes (or a merge or export
// reads the window): the detect reads them there, beside the active stamps
// of the lines it tests, instead of streaming the LDCA stamps.
static int commit_seav_window(sp_ctx* ctx, uint32_t router) {
  int rc = fold_router(ctx, router);
  if (rc != SP_OK) return rc;
  if (sp::launch_commit_window(reinterpret_cast<uint32_t*>(ctx->seav(router)), ctx->st_seav(router),
                               ctx->seav_words(), ctx->ldca(router), ctx->st_ldca(router), 0,
                               reinterpret_cast<uint32_t*>(ctx->wseav(router)), ctx->wldca(router),
                               ctx->dev_clock(router), ctx->p.window_slices, ctx->stream) != cudaSuccess)
    return SP_ERR_CUDA;
  return SP_OK;
}

int sp_reset(sp_ctx* ctx, uint32_t router) {
  if (!ctx) return SP_ERR_PARAM;
  if (router >= ctx->p.n_routers) return SP_ERR_ROUTER;
  ctx->planes_dirty[router] = false;     // pending planes belong to the old window
  ctx->slice_dirty[router] = false;
  if (ctx->sliding) {
    ctx->slice[router] = 0;
    if (cudaMemsetAsync(ctx->dev_clock(router), 0, sizeof(uint64_t), ctx->stream) != cudaSuccess) return SP_ERR_CUDA;
    if (sp::launch_zero(ctx->st_seav(router), ctx->st_stride, ctx->stream) != cudaSuccess) return SP_ERR_CUDA;
  }
  if (sp::launch_zero_flags(ctx->seav(router), ctx->stride, ctx->ovf + router, 1, ctx->stream) != cudaSuccess)
    return SP_ERR_CUDA;
  ctx->ldca_zero[router] = !ctx->sliding;
  return SP_OK;
}

int sp_reset_range(sp_ctx* ctx, uint32_t first, uint32_t count) {
  if (!ctx) return SP_ERR_PARAM;
  if (count == 0) return SP_OK;
  if (first >= ctx->p.n_routers || count > ctx->p.n_routers - first) return SP_ERR_ROUTER;
  if (ctx->sliding) {                            // stamps and clocks are per router
    for (uint32_t r = first; r < first + count; ++r) {
      const int rc = sp_reset(ctx, r);
      if (rc != SP_OK) return rc;
    }
    return SP_OK;
  }
  // the routers' regions are contiguous: one zeroing launch for all of them
  if (sp::launch_zero_flags(ctx->seav(first), ctx->stride * count, ctx->ovf + first, count, ctx->stream) !=
      cudaSuccess)
    return SP_ERR_CUDA;
  for (uint32_t r = first; r < first + count; ++r) {
    ctx->planes_dirty[r] = false;                // pending planes belong to the old window
    ctx->slice_dirty[r] = false;
    ctx->ldca_zero[r] = true;
  }
  return SP_OK;
}

int sp_update(sp_ctx* ctx, uint32_t router, const uint32_t* dev_pairs, uint64_t n_pairs) {
  if (!ctx) return SP_ERR_PARAM;
  if (router >= ctx->p.n_routers) return SP_ERR_ROUTER;
  if (n_pairs == 0) return SP_OK;
  if (!dev_pairs || ((uintptr_t)dev_pairs & 7u)) return SP_ERR_PARAM;
  return do_update(ctx, router, dev_pairs, n_pairs);
}

static int ensure_staging(sp_ctx* ctx) {
  if (ctx->staging[0]) return SP_OK;
  for (int i = 0; i < 2; ++i) {
    if (cudaMalloc(&ctx->staging[i], kStagingPairs * 8) != cudaSuccess) { cudaGetLastError(); return SP_ERR_NOMEM; }
    if (cudaEventCreateWithFlags(&ctx->ev_copied[i], cudaEventDisableTiming) != cudaSuccess) return SP_ERR_CUDA;
    if (cudaEventCreateWithFlags(&ctx->ev_free[i], cudaEventDisableTiming) != cudaSuccess) return SP_ERR_CUDA;
  }
  if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess) return SP_ERR_CUDA;
  return SP_OK;
}

int sp_update_host(sp_ctx* ctx, uint32_t router, const uint32_t* host_pairs, uint64_t n_pairs) {
  if (!ctx) return SP_ERR_PARAM;
  if (router >= ctx->p.n_routers) return SP_ERR_ROUTER;
  if (n_pairs == 0) return SP_OK;
  if (!host_pairs) return SP_ERR_PARAM;
  int rc = ensure_staging(ctx);
  if (rc != SP_OK) return rc;
  const bool binned = use_binned(ctx, n_pairs);
  if (binned && (rc = ensure_binned(ctx, router)) != SP_OK) return rc;
  ctx->slice_dirty[router] = true;
  const uint32_t bins = 1u << ctx->p.k_log2;
  // Chunks of the host stream go through two device staging buffers: the copy
  // of chunk j + 1 (copy stream) overlaps the scan of chunk j (main stream);
  // ev_free[b] marks the last scan that reads buffer b.  A binned update bins
  // every chunk of a round into the same lists and applies them once.
  uint64_t done = 0;
  uint32_t j = 0;
  while (done < n_pairs) {
    const uint64_t round_cap = ctx->bs.max_pairs < kHostRoundPairs ? ctx->bs.max_pairs : kHostRoundPairs;
    const uint64_t round_n = binned ? ((n_pairs - done) < round_cap ? (n_pairs - done) : round_cap)
                                    : (n_pairs - done);
    const uint32_t chunks = (uint32_t)((round_n + kStagingPairs - 1) / kStagingPairs);
    const uint32_t cap = binned ? sp::binned_list_cap(round_n, bins, ctx->bs.shape, ctx->bs.ctas, chunks) : 0u;
    const sp::BinnedScratch s = binned ? binned_scratch(ctx, router) : sp::BinnedScratch();
    uint64_t rdone = 0, rot = 0;
    for (uint32_t c = 0; rdone < round_n; ++c, ++j) {
      const uint32_t b = j & 1u;
      const uint64_t m = (round_n - rdone) < kStagingPairs ? (round_n - rdone) : kStagingPairs;
      const uint32_t* src = host_pairs + 2 * (done + rdone);
      if (cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_free[b], 0) != cudaSuccess ||
          cudaMemcpyAsync(ctx->staging[b], src, m * 8, cudaMemcpyHostToDevice, ctx->copy_stream) != cudaSuccess ||
          cudaEventRecord(ctx->ev_copied[b], ctx->copy_stream) != cudaSuccess ||
          cudaStreamWaitEvent(ctx->stream, ctx->ev_copied[b], 0) != cudaSuccess) return SP_ERR_CUDA;
      if (binned) {
        if (sp::binned_bin_chunk(ctx->d, ctx->seav(router), ctx->ldca(router), sp::bin_src_one(ctx->staging[b], m), s,
                                 cap, c > 0, (uint32_t)(rot % ctx->bs.ctas), ctx->stream) != cudaSuccess)
          return SP_ERR_CUDA;
        rot += (m + sp::binned_tile_pairs(ctx->bs.shape) - 1) / sp::binned_tile_pairs(ctx->bs.shape);
      } else if ((rc = do_update(ctx, router, ctx->staging[b], m)) != SP_OK) {
        return rc;
      }
      if (cudaEventRecord(ctx->ev_free[b], ctx->stream) != cudaSuccess) return SP_ERR_CUDA;
      rdone += m;
    }
    if (binned) {
      if (sp::binned_apply_round(ctx->d, s, cap, ctx->planes_dirty[router], ctx->stream) != cudaSuccess)
        return SP_ERR_CUDA;
      ctx->planes_dirty[router] = true;
    }
    done += round_n;
  }
  return SP_OK;
}

static bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// Uploads n entries of a batch table through the next pinned slot of the
// ring; *dev receives the slot's device copy.
// Gives a table slot room for n batches.  A slot that was never allocated
// costs no wait; growing a used one waits for the stream first, since a
// launch issued after its last upload may still read the old device copy.
static int grow_table_slot(sp_ctx* ctx, sp_ctx::TableSlot& t, uint32_t n) {
  if (n <= t.cap) return SP_OK;
  if (t.host) {
    const int wrc = wait_stream(ctx);
    if (wrc != SP_OK) return wrc;
    cudaFreeHost(t.host);
    cudaFree(t.dev);
    t.host = nullptr;
    t.dev = nullptr;
    t.cap = 0;
    t.pending = false;
  }
  const uint32_t cap = n < 1024 ? 1024 : n;
  if (cudaMallocHost(&t.host, cap * sizeof(sp_batch)) != cudaSuccess ||
      cudaMalloc(&t.dev, cap * sizeof(sp_batch)) != cudaSuccess) {
    cudaGetLastError();
    if (t.host) cudaFreeHost(t.host);
    t.host = nullptr;
    t.dev = nullptr;
    return SP_ERR_NOMEM;
  }
  t.cap = cap;
  if (!t.ev && cudaEventCreateWithFlags(&t.ev, cudaEventDisableTiming) != cudaSuccess) return SP_ERR_CUDA;
  return SP_OK;
}

static int upload_table(sp_ctx* ctx, const sp_batch* tab, uint32_t n, const sp_batch** dev) {
  sp_ctx::TableSlot& t = ctx->tables[ctx->table_next++ % sp_ctx::kTableRing];
  const int grc = grow_table_slot(ctx, t, n);
  if (grc != SP_OK) return grc;
  if (t.pending) {
    const int wrc = wait_event_bounded(ctx, t.ev);
    if (wrc != SP_OK) return wrc;
  }
  memcpy(t.host, tab, n * sizeof(sp_batch));
  if (cudaMemcpyAsync(t.dev, t.host, n * sizeof(sp_batch), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
      cudaEventRecord(t.ev, ctx->stream) != cudaSuccess) return SP_ERR_CUDA;
  t.pending = true;
  *dev = t.dev;
  return SP_OK;
}

static int launch_table(sp_ctx* ctx, const sp_batch* dev_tab, uint32_t n) {
  constexpr uint32_t kMaxTable = 8192;
  for (uint32_t i = 0; i < n; i += kMaxTable) {
    const uint32_t m = (n - i) < kMaxTable ? (n - i) : kMaxTable;
    if (sp::launch_scan_multi(ctx->d, ctx->sketches, ctx->stride, ctx->seav_pad, ctx->p.n_routers, dev_tab + i, m,
                              ctx->kerr, ctx->multi_threads, ctx->multi_grid, ctx->stream) != cudaSuccess)
      return SP_ERR_CUDA;
  }
  return SP_OK;
}

int sp_reserve(sp_ctx* ctx, uint32_t first, uint32_t count) {
  if (!ctx) return SP_ERR_PARAM;
  if (first > ctx->p.n_routers || count > ctx->p.n_routers - first) return SP_ERR_ROUTER;
  int rc = ensure_staging(ctx);
  for (int i = 0; rc == SP_OK && i < sp_ctx::kTableRing; ++i) rc = grow_table_slot(ctx, ctx->tables[i], 1);
  if (rc != SP_OK || !sp::binned_applicable(ctx->d)) return rc;
  for (uint32_t r = first; rc == SP_OK && r < first + count; ++r) rc = ensure_binned(ctx, r);
  return rc;
}

int sp_update_batched(sp_ctx* ctx, uint32_t n_batches, const uint32_t* routers,
                      const uint32_t* const* dev_pairs, const uint64_t* n_pairs) {
  if (!ctx) return SP_ERR_PARAM;
  if (n_batches == 0) return SP_OK;
  if (!routers || !dev_pairs || !n_pairs) return SP_ERR_PARAM;
  for (uint32_t b = 0; b < n_batches; ++b) {
    if (routers[b] >= ctx->p.n_routers) return SP_ERR_ROUTER;
    if (n_pairs[b] && (!dev_pairs[b] || ((uintptr_t)dev_pairs[b] & 7u))) return SP_ERR_PARAM;
  }
  if (capturing(ctx->stream)) return SP_ERR_STATE;
  const uint32_t R = ctx->p.n_routers;
  std::vector<uint64_t> total(R, 0);
  // the non-empty batches grouped by router, each group in call order (one counting pass)
  std::vector<uint32_t> first(R + 1, 0), order;
  for (uint32_t b = 0; b < n_batches; ++b) {
    total[routers[b]] += n_pairs[b];
    if (n_pairs[b]) ++first[routers[b] + 1];
  }
  for (uint32_t r = 0; r < R; ++r) first[r + 1] += first[r];
  order.resize(first[R]);
  {
    std::vector<uint32_t> fill(first.begin(), first.end() - 1);
    for (uint32_t b = 0; b < n_batches; ++b)
      if (n_pairs[b]) order[fill[routers[b]]++] = b;
  }
  for (uint32_t r = 0; r < R; ++r)
    if (total[r]) ctx->slice_dirty[r] = true;
  const uint32_t bins = 1u << ctx->p.k_log2;
  std::vector<sp_batch> rest;
  rest.reserve(n_batches);
  for (uint32_t r = 0; r < R; ++r) {
    if (total[r] == 0) continue;
    if (!use_binned(ctx, total[r])) {
      ctx->ldca_zero[r] = false;                         // direct form: bits straight into the LDCA
      for (uint32_t q = first[r]; q < first[r + 1]; ++q)
        rest.push_back(sp_batch{dev_pairs[order[q]], n_pairs[order[q]], r, 0u});
      continue;
    }
    int rc = ensure_binned(ctx, r);
    if (rc != SP_OK) return rc;
    // rounds of consecutive batches of router r, at most max_pairs each
    const std::vector<uint32_t> mine(order.begin() + first[r], order.begin() + first[r + 1]);
    size_t i = 0;
    while (i < mine.size()) {
      if (n_pairs[mine[i]] > ctx->bs.max_pairs) {          // a batch that is a round by itself
        if ((rc = do_update(ctx, r, dev_pairs[mine[i]], n_pairs[mine[i]])) != SP_OK) return rc;
        ++i;
        continue;
      }
      // a round ends before its pairs pass max_pairs or its list capacity
      // (which grows with the binning launches) passes the allocated one
      size_t j = i;
      uint64_t sum = 0;
      while (j < mine.size() && sum + n_pairs[mine[j]] <= ctx->bs.max_pairs) {
        const uint32_t l = (uint32_t)((j + 1 - i + sp::kBinMaxSrc - 1) / sp::kBinMaxSrc);
        if (j > i && sp::binned_list_cap(sum + n_pairs[mine[j]], bins, ctx->bs.shape, ctx->bs.ctas, l) >
                         ctx->bs.cap_alloc) break;
        sum += n_pairs[mine[j++]];
      }
      // the round's batches, up to kBinMaxSrc streams per binning launch
      const uint32_t launches = (uint32_t)((j - i + sp::kBinMaxSrc - 1) / sp::kBinMaxSrc);
      const uint32_t cap = sp::binned_list_cap(sum, bins, ctx->bs.shape, ctx->bs.ctas, launches);
      const sp::BinnedScratch s = binned_scratch(ctx, r);
      uint64_t rot = 0;
      for (size_t q0 = i; q0 < j; q0 += sp::kBinMaxSrc) {
        sp::BinSrc src{};
        uint64_t tiles = 0;
        for (size_t q = q0; q < j && q < q0 + sp::kBinMaxSrc; ++q) {
          src.ptr[src.count] = dev_pairs[mine[q]];
          src.n[src.count] = n_pairs[mine[q]];
          tiles += (n_pairs[mine[q]] + sp::binned_tile_pairs(ctx->bs.shape) - 1) / sp::binned_tile_pairs(ctx->bs.shape);
          ++src.count;
        }
        if (sp::binned_bin_chunk(ctx->d, ctx->seav(r), ctx->ldca(r), src, s, cap, q0 > i,
                                 (uint32_t)(rot % ctx->bs.ctas), ctx->stream) != cudaSuccess) return SP_ERR_CUDA;
        rot += tiles;
      }
      if (sp::binned_apply_round(ctx->d, s, cap, ctx->planes_dirty[r], ctx->stream) != cudaSuccess) return SP_ERR_CUDA;
      ctx->planes_dirty[r] = true;
      i = j;
    }
  }
  if (rest.empty()) return SP_OK;
  const sp_batch* dev_tab = nullptr;
  int rc = upload_table(ctx, rest.data(), (uint32_t)rest.size(), &dev_tab);
  if (rc != SP_OK) return rc;
  return launch_table(ctx, dev_tab, (uint32_t)rest.size());
}

int sp_update_batched_host(sp_ctx* ctx, uint32_t n_batches, const uint32_t* routers,
                           const uint32_t* const* host_pairs, const uint64_t* n_pairs, void* dev_arena,
                           uint64_t arena_bytes, void* copy_stream) {
  if (!ctx) return SP_ERR_PARAM;
  if (n_batches == 0) return SP_OK;
  if (!routers || !host_pairs || !n_pairs || !dev_arena || ((uintptr_t)dev_arena & 15u)) return SP_ERR_PARAM;
  // the batches' places in the arena: packed, each at a 16-byte boundary
  std::vector<const uint32_t*> dev(n_batches);
  uint64_t off = 0;
  for (uint32_t b = 0; b < n_batches; ++b) {
    if (routers[b] >= ctx->p.n_routers) return SP_ERR_ROUTER;
    if (n_pairs[b] && !host_pairs[b]) return SP_ERR_PARAM;
    dev[b] = reinterpret_cast<const uint32_t*>(static_cast<uint8_t*>(dev_arena) + off);
    off += align_up(n_pairs[b] * 8, 16);
    if (off > arena_bytes) return SP_ERR_PARAM;
  }
  if (!ctx->ev_arena && cudaEventCreateWithFlags(&ctx->ev_arena, cudaEventDisableTiming) != cudaSuccess)
    return SP_ERR_CUDA;
  cudaStream_t cs = static_cast<cudaStream_t>(copy_stream);
  for (uint32_t b = 0; b < n_batches; ++b)
    if (n_pairs[b] && cudaMemcpyAsync(const_cast<uint32_t*>(dev[b]), host_pairs[b], n_pairs[b] * 8,
                                      cudaMemcpyHostToDevice, cs) != cudaSuccess) return SP_ERR_CUDA;
  if (cudaEventRecord(ctx->ev_arena, cs) != cudaSuccess || cudaStreamWaitEvent(ctx->stream, ctx->ev_arena, 0) != cudaSuccess)
    return SP_ERR_CUDA;
  return sp_update_batched(ctx, n_batches, routers, dev.data(), n_pairs);
}

int sp_update_batched_device(sp_ctx* ctx, const sp_batch* dev_batches, uint32_t n_batches) {
  if (!ctx) return SP_ERR_PARAM;
  if (n_batches == 0) return SP_OK;
  if (!dev_batches || n_batches > 8192) return SP_ERR_PARAM;
  // the table is read on the device: any router may receive bits
  for (uint32_t r = 0; r < ctx->p.n_routers; ++r) {
    ctx->slice_dirty[r] = true;
    ctx->ldca_zero[r] = false;
  }
  return launch_table(ctx, dev_batches, n_batches);
}

int sp_autotune(sp_ctx* ctx, const uint32_t* dev_pairs, uint64_t n_pairs, uint32_t* best_threads,
                uint32_t* best_blocks) {
  if (!ctx || !dev_pairs || n_pairs == 0 || ((uintptr_t)dev_pairs & 7u)) return SP_ERR_PARAM;
  const sp_batch one{dev_pairs, n_pairs, 0u, 0u};
  const sp_batch* dev_tab = nullptr;
  ctx->ldca_zero[0] = false;                          // the trial scans write router 0 directly
  int rc = upload_table(ctx, &one, 1, &dev_tab);
  if (rc != SP_OK) return rc;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SP_ERR_CUDA;
  const int shapes[3] = {128, 256, 512};
  float best = 1e30f;
  int bt = ctx->multi_threads, bg = ctx->multi_grid;
  for (int t : shapes) {
    const int most = 2048 / t;
    const int per[4] = {1, 2, 4, most};
    for (int k = 0; k < 4; ++k) {
      if (per[k] > most || (k == 3 && (most == 1 || most == 2 || most == 4))) continue;
      ctx->multi_threads = t;
      ctx->multi_grid = sms * per[k];
      if ((rc = launch_table(ctx, dev_tab, 1)) != SP_OK) break;          // warm up
      cudaEventRecord(e0, ctx->stream);
      for (int it = 0; it < 3; ++it)
        if ((rc = launch_table(ctx, dev_tab, 1)) != SP_OK) break;
      cudaEventRecord(e1, ctx->stream);
      float ms = 0.f;
      if (rc == SP_OK) rc = wait_event_bounded(ctx, e1);
      if (rc == SP_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = SP_ERR_CUDA;
      if (rc != SP_OK) break;
      if (ms < best) { best = ms; bt = t; bg = ctx->multi_grid; }
    }
    if (rc != SP_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->multi_threads = bt;
  ctx->multi_grid = bg;
  if (rc != SP_OK) return rc;
  if (best_threads) *best_threads = (uint32_t)bt;
  if (best_blocks) *best_blocks = (uint32_t)(bg / (sms ? sms : 1));
  rc = sp_reset(ctx, 0);
  if (rc == SP_OK) rc = wait_stream(ctx);
  return rc;
}

static sp_binned_shape shape_record(uint32_t index) {
  const sp::BinShape h = sp::binned_shape((int)index);
  return sp_binned_shape{index, h.threads, h.stage, h.tpr, h.per_sm, h.apply_threads};
}

int sp_binned_shapes(sp_binned_shape* out, uint32_t cap, uint32_t* n) {
  if (!n || (cap && !out)) return SP_ERR_PARAM;
  *n = (uint32_t)sp::binned_shape_count();
  for (uint32_t i = 0; i < cap && i < *n; ++i) out[i] = shape_record(i);
  return SP_OK;
}

int sp_set_binned_shape(sp_ctx* ctx, uint32_t index) {
  if (!ctx || index >= (uint32_t)sp::binned_shape_count()) return SP_ERR_PARAM;
  ctx->bs_shape_index = index;
  if (ctx->bs.lists) set_binned_shape(ctx, (int)index);
  return SP_OK;
}

int sp_get_binned_shape(const sp_ctx* ctx, sp_binned_shape* out) {
  if (!ctx || !out) return SP_ERR_PARAM;
  *out = shape_record(ctx->bs_shape_index);
  return SP_OK;
}

int sp_autotune_binned(sp_ctx* ctx, const uint32_t* dev_pairs, uint64_t n_pairs, sp_binned_shape* best) {
  if (!ctx || !dev_pairs || n_pairs == 0 || ((uintptr_t)dev_pairs & 7u)) return SP_ERR_PARAM;
  if (!sp::binned_applicable(ctx->d)) return SP_ERR_STATE;
  int rc = ensure_binned(ctx, 0);
  if (rc != SP_OK) return rc;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return SP_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SP_ERR_CUDA;
  }
  const uint32_t before = ctx->bs_shape_index;
  uint32_t pick = before;
  float best_ms = 1e30f;
  auto scan = [&]() {
    const sp::BinnedScratch s = binned_scratch(ctx, 0);
    if (sp::launch_scan_binned(ctx->d, ctx->seav(0), ctx->ldca(0), dev_pairs, n_pairs, s, ctx->stream) != cudaSuccess)
      return SP_ERR_CUDA;
    ctx->planes_dirty[0] = true;
    return SP_OK;
  };
  for (int i = 0; i < sp::binned_shape_count() && rc == SP_OK; ++i) {
    set_binned_shape(ctx, i);
    if ((rc = scan()) != SP_OK) break;                                  // warm up
    if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) { rc = SP_ERR_CUDA; break; }
    for (int it = 0; it < 3 && rc == SP_OK; ++it) rc = scan();
    if (rc != SP_OK || cudaEventRecord(e1, ctx->stream) != cudaSuccess) { rc = rc != SP_OK ? rc : SP_ERR_CUDA; break; }
    float ms = 0.f;
    if ((rc = wait_event_bounded(ctx, e1)) != SP_OK) break;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { rc = SP_ERR_CUDA; break; }
    if (ms < best_ms) { best_ms = ms; pick = (uint32_t)i; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  set_binned_shape(ctx, (int)(rc == SP_OK ? pick : before));
  if (rc != SP_OK) return rc;
  if (best) *best = shape_record(pick);
  rc = sp_reset(ctx, 0);
  if (rc == SP_OK) rc = wait_stream(ctx);
  return rc;
}

int sp_merge(sp_ctx* ctx, const uint32_t* routers, uint32_t n, uint32_t dst_router) {
  if (!ctx || (n && !routers)) return SP_ERR_PARAM;
  if (dst_router >= ctx->p.n_routers) return SP_ERR_ROUTER;
  for (uint32_t i = 0; i < n; ++i)
    if (routers[i] >= ctx->p.n_routers) return SP_ERR_ROUTER;
  ctx->ldca_zero[dst_router] = false;
  std::vector<const uint8_t*> srcs;                // every listed router but dst (x | x = x)
  srcs.reserve(n);
  if (ctx->sliding) {
    for (uint32_t i = 0; i < n; ++i)
      if (ctx->slice[routers[i]] != ctx->slice[dst_router]) return SP_ERR_STATE;   // one slice clock
    int rc = commit(ctx, dst_router);
    for (uint32_t i = 0; i < n && rc == SP_OK; ++i) {
      rc = commit(ctx, routers[i]);
      if (routers[i] != dst_router) srcs.push_back(ctx->st_seav(routers[i]));
    }
    if (rc != SP_OK) return rc;
    return sp::launch_merge_stamp(ctx->st_seav(dst_router), srcs.data(), (uint32_t)srcs.size(), ctx->st_stride,
                                  ctx->dev_clock(dst_router), ctx->stream) == cudaSuccess ? SP_OK : SP_ERR_CUDA;
  }
  int rc = fold_router(ctx, dst_router);
  if (rc != SP_OK) return rc;
  for (uint32_t i = 0; i < n; ++i) {
    rc = fold_router(ctx, routers[i]);
    if (rc != SP_OK) return rc;
    if (routers[i] != dst_router) srcs.push_back(ctx->seav(routers[i]));
  }
  return sp::launch_merge(ctx->seav(dst_router), srcs.data(), (uint32_t)srcs.size(), ctx->stride, ctx->stream) ==
                 cudaSuccess ? SP_OK : SP_ERR_CUDA;
}

int sp_copy_sketch(sp_ctx* ctx, uint32_t router, void* dev_dst, uint64_t cap, uint64_t* n) {
  if (!ctx || !n) return SP_ERR_PARAM;
  if (router >= ctx->p.n_routers) return SP_ERR_ROUTER;
  *n = ctx->stride;
  if (!dev_dst) return SP_OK;
  if (cap < ctx->stride) return SP_ERR_TRUNCATED;
  if ((uintptr_t)dev_dst & 15u) return SP_ERR_PARAM;
  int frc = ctx->sliding ? commit_window(ctx, router) : fold_router(ctx, router);
  if (frc != SP_OK) return frc;
  const uint8_t* src = ctx->sliding ? ctx->wseav(router) : ctx->seav(router);
  return cudaMemcpyAsync(dev_dst, src, ctx->stride, cudaMemcpyDeviceToDevice, ctx->stream) == cudaSuccess
             ? SP_OK : SP_ERR_CUDA;
}

int sp_merge_device(sp_ctx* ctx, const void* const* dev_images, uint32_t n, uint32_t dst_router) {
  if (!ctx || (n && !dev_images)) return SP_ERR_PARAM;
  if (dst_router >= ctx->p.n_routers) return SP_ERR_ROUTER;
  if (ctx->sliding) return SP_ERR_STATE;      // an image holds window bits, not slice stamps
  std::vector<const uint8_t*> srcs(n);
  for (uint32_t i = 0; i < n; ++i) {
    if (!dev_images[i] || ((uintptr_t)dev_images[i] & 15u)) return SP_ERR_PARAM;
    srcs[i] = static_cast<const uint8_t*>(dev_images[i]);
  }
  const int rc = fold_router(ctx, dst_router);
  if (rc != SP_OK) return rc;
  ctx->ldca_zero[dst_router] = false;
  return sp::launch_merge(ctx->seav(dst_router), srcs.data(), n, ctx->stride, ctx->stream) == cudaSuccess
             ? SP_OK : SP_ERR_CUDA;
}

int sp_detect_async(sp_ctx* ctx, uint32_t router, uint32_t threshold) {
  if (!ctx) return SP_ERR_PARAM;
  if (router >= ctx->p.n_routers) return SP_ERR_ROUTER;
  if (threshold == 0) threshold = ctx->p.theta;
  const uint32_t zt = sp_z_theta(ctx->p.k_log2, threshold);
  int frc = ctx->sliding ? commit_seav_window(ctx, router) : fold_router(ctx, router);
  if (frc != SP_OK) return frc;
  if (cudaMemsetAsync(ctx->status, 0, sizeof(DetectStatus), ctx->stream) != cudaSuccess) return SP_ERR_CUDA;
  // a sliding router is detected on its window SEAV and, for the LDCA test of
  // each tested host, the active stamps and pending slice bits of its lines
  const cudaError_t de =
      ctx->sliding
          ? sp::launch_detect_sliding(ctx->d, ctx->wseav(router), ctx->ldca(router), ctx->st_ldca(router),
                                      ctx->dev_clock(router), ctx->p.window_slices, zt, ctx->keys, ctx->cap,
                                      ctx->p.max_join, ctx->status, ctx->stream)
          : sp::launch_detect(ctx->d, ctx->seav(router), ctx->ldca(router), zt, ctx->keys, ctx->cap,
                              ctx->p.max_join, ctx->status, ctx->stream);
  if (de != cudaSuccess) return SP_ERR_CUDA;
  if (sp::launch_sort_emit(ctx->keys, ctx->cap, ctx->status, ctx->est_table, ctx->p.k_log2,
                           ctx->records, ctx->stream) != cudaSuccess) return SP_ERR_CUDA;
  ctx->detect_issued = true;
  ctx->last_threshold = threshold;
  return threshold < ctx->p.theta ? SP_WARN_THETA_BELOW_INIT : SP_OK;
}

int sp_results(sp_ctx* ctx, sp_candidate* host_out, uint64_t cap, uint64_t* n_total) {
  if (!ctx || !n_total || (cap && !host_out)) return SP_ERR_PARAM;
  if (!ctx->detect_issued) return SP_ERR_STATE;
  // status, error word and a prefix of the records come back with one wait
  constexpr size_t kKerrAt = 64, kRecordsAt = 128;
  static_assert(sizeof(DetectStatus) <= kKerrAt, "status slot");
  if (!ctx->result_host &&
      cudaMallocHost(&ctx->result_host, kRecordsAt + (size_t)kResultPrefix * sizeof(sp_candidate)) != cudaSuccess) {
    cudaGetLastError();
    ctx->result_host = nullptr;
    return SP_ERR_NOMEM;
  }
  const uint64_t pre = ctx->cap < kResultPrefix ? ctx->cap : kResultPrefix;
  if (cudaMemcpyAsync(ctx->result_host, ctx->status, sizeof(DetectStatus), cudaMemcpyDeviceToHost,
                      ctx->stream) != cudaSuccess ||
      cudaMemcpyAsync(ctx->result_host + kKerrAt, ctx->kerr, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                      ctx->stream) != cudaSuccess ||
      (pre && cudaMemcpyAsync(ctx->result_host + kRecordsAt, ctx->records, pre * sizeof(sp_candidate),
                              cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)) return SP_ERR_CUDA;
  int wrc = wait_stream(ctx);
  if (wrc != SP_OK) return wrc;
  DetectStatus st;
  uint32_t kerr = 0;
  memcpy(&st, ctx->result_host, sizeof(st));
  memcpy(&kerr, ctx->result_host + kKerrAt, sizeof(kerr));
  if (kerr) {
    // a device batch table named a bad router or stream (the batch was skipped)
    cudaMemsetAsync(ctx->kerr, 0, sizeof(uint32_t), ctx->stream);
    *n_total = st.count;
    return SP_ERR_ROUTER;
  }
  *n_total = st.count;
  const uint64_t avail = st.count < ctx->cap ? st.count : ctx->cap;
  const uint64_t m = avail < cap ? avail : cap;
  const uint64_t staged = m < pre ? m : pre;
  if (staged) memcpy(host_out, ctx->result_host + kRecordsAt, staged * sizeof(sp_candidate));
  if (m > staged) {
    if (cudaMemcpyAsync(host_out + staged, ctx->records + staged, (m - staged) * sizeof(sp_candidate),
                        cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess) return SP_ERR_CUDA;
    if ((wrc = wait_stream(ctx)) != SP_OK) return wrc;
  }
  if (st.overflow) return SP_ERR_CANDIDATE_OVERFLOW;
  if (st.count > cap) return SP_ERR_TRUNCATED;
  return SP_OK;
}

int sp_results_async(sp_ctx* ctx, sp_candidate* host_out, uint64_t cap, uint32_t* host_status) {
  if (!ctx || !host_status || (cap && !host_out)) return SP_ERR_PARAM;
  if (!ctx->detect_issued) return SP_ERR_STATE;
  const uint64_t m = cap < ctx->cap ? cap : ctx->cap;
  if (cudaMemcpyAsync(host_status, ctx->status, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
    return SP_ERR_CUDA;
  if (m && cudaMemcpyAsync(host_out, ctx->records, m * sizeof(sp_candidate), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
    return SP_ERR_CUDA;
  return SP_OK;
}

int sp_detect(sp_ctx* ctx, uint32_t router, uint32_t threshold,
              sp_candidate* host_out, uint64_t cap, uint64_t* n_total) {
  int w = sp_detect_async(ctx, router, threshold);
  if (w < 0) return w;
  int rc = sp_results(ctx, host_out, cap, n_total);
  return rc != SP_OK ? rc : w;
}

int sp_results_device(sp_ctx* ctx, const sp_candidate** dev_records, const uint32_t** dev_count) {
  if (!ctx || !dev_records || !dev_count) return SP_ERR_PARAM;
  *dev_records = ctx->records;
  *dev_count = &ctx->status->count;
  return SP_OK;
}

int sp_slide(sp_ctx* ctx, uint32_t router) {
  if (!ctx) return SP_ERR_PARAM;
  if (router >= ctx->p.n_routers) return SP_ERR_ROUTER;
  if (!ctx->sliding) return sp_reset(ctx, router);   // discrete window: the next period starts empty
  int rc = commit(ctx, router);                       // slice t's bits carry id(t)
  if (rc != SP_OK) return rc;
  ctx->slice[router] += 1;
  // t += 1 on the device, then the sweep of segment (t mod M), M = 255 - k,
  // of the router's counters: every argument is fixed, so a graph that
  // recorded this call advances the window at each replay
  return sp::launch_tick_clean(ctx->st_seav(router), ctx->st_stride, ctx->dev_clock(router), ctx->p.window_slices,
                               ctx->stream) == cudaSuccess ? SP_OK : SP_ERR_CUDA;
}

int sp_export(sp_ctx* ctx, uint32_t router, void* host_buf, uint64_t cap, uint64_t* n) {
  if (!ctx || !n) return SP_ERR_PARAM;
  if (router >= ctx->p.n_routers) return SP_ERR_ROUTER;
  const uint64_t total = sizeof(ImageHeader) + ctx->seav_bytes + ctx->ldca_bytes + 8;
  *n = total;
  if (!host_buf) return SP_OK;
  if (cap < total) return SP_ERR_TRUNCATED;
  int frc = ctx->sliding ? commit_window(ctx, router) : fold_router(ctx, router);
  if (frc != SP_OK) return frc;
  const uint8_t* seav = ctx->sliding ? ctx->wseav(router) : ctx->seav(router);
  const uint32_t* ldca = ctx->sliding ? ctx->wldca(router) : ctx->ldca(router);
  ImageHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, "SPSKETCH", 8);
  h.version = 1;
  h.header_bytes = sizeof(ImageHeader);
  h.r = ctx->p.r; h.sr = ctx->p.sr;
  memcpy(h.isb, ctx->p.isb, sizeof(h.isb));
  memcpy(h.ibn, ctx->p.ibn, sizeof(h.ibn));
  h.k_log2 = ctx->p.k_log2; h.lr = ctx->p.lr; h.lc_log2 = ctx->p.lc_log2; h.theta = ctx->p.theta;
  h.seed = ctx->p.seed;
  h.seav_bytes = ctx->seav_bytes;
  h.ldca_bytes = ctx->ldca_bytes;
  uint8_t* out = static_cast<uint8_t*>(host_buf);
  memcpy(out, &h, sizeof(h));
  if (cudaMemcpyAsync(out + sizeof(h), seav, ctx->seav_bytes, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
      cudaMemcpyAsync(out + sizeof(h) + ctx->seav_bytes, ldca, ctx->ldca_bytes, cudaMemcpyDeviceToHost,
                      ctx->stream) != cudaSuccess) return SP_ERR_CUDA;
  const int wrc = wait_stream(ctx);
  if (wrc != SP_OK) return wrc;
  const uint64_t sum = fnv1a64(out, total - 8);
  memcpy(out + total - 8, &sum, 8);
  return SP_OK;
}

int sp_import(sp_ctx* ctx, uint32_t router, const void* host_buf, uint64_t n) {
  if (!ctx || !host_buf) return SP_ERR_PARAM;
  if (router >= ctx->p.n_routers) return SP_ERR_ROUTER;
  if (ctx->sliding) return SP_ERR_STATE;   // an image holds window bits, not slice stamps
  const uint64_t total = sizeof(ImageHeader) + ctx->seav_bytes + ctx->ldca_bytes + 8;
  if (n != total) return SP_ERR_CHECKSUM;
  const uint8_t* in = static_cast<const uint8_t*>(host_buf);
  uint64_t sum;
  memcpy(&sum, in + total - 8, 8);
  if (fnv1a64(in, total - 8) != sum) return SP_ERR_CHECKSUM;
  ImageHeader h;
  memcpy(&h, in, sizeof(h));
  if (memcmp(h.magic, "SPSKETCH", 8) != 0 || h.version != 1 || h.header_bytes != sizeof(ImageHeader) ||
      h.r != ctx->p.r || h.sr != ctx->p.sr || memcmp(h.isb, ctx->p.isb, sizeof(h.isb)) != 0 ||
      memcmp(h.ibn, ctx->p.ibn, sizeof(h.ibn)) != 0 || h.k_log2 != ctx->p.k_log2 || h.lr != ctx->p.lr ||
      h.lc_log2 != ctx->p.lc_log2 || h.theta != ctx->p.theta || h.seed != ctx->p.seed ||
      h.seav_bytes != ctx->seav_bytes || h.ldca_bytes != ctx->ldca_bytes)
    return SP_ERR_CHECKSUM;
  ctx->planes_dirty[router] = false;
  ctx->ldca_zero[router] = false;
  if (cudaMemcpyAsync(ctx->seav(router), in + sizeof(h), ctx->seav_bytes, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
      cudaMemcpyAsync(ctx->ldca(router), in + sizeof(h) + ctx->seav_bytes, ctx->ldca_bytes, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
    return SP_ERR_CUDA;
  return wait_stream(ctx);
}

}  // extern "C"
