// sp_noalloc.cu -- detect without any device allocation.
//
// sp_detect_noalloc runs the same restore-and-filter kernels as
// sp_detect_async, but on a sketch the caller already holds in device memory
// and with all of its scratch (the unsorted result keys, the status word and
// the estimate tables) taken from one fixed array in this file instead of
// from a context.  It exists for callers that may not allocate device memory
// at the point where they detect: processes whose device memory is owned by
// another allocator (a framework's caching allocator, a partition fixed at
// start-up) or budgeted up front, and real-time loops that cannot afford an
// allocation, or its failure, on their critical path.
#include <math.h>
#include <string.h>

#include <mutex>

#include "sp_internal.h"

namespace {

// Scratch layout, in 64-bit words:
//   [0, kKeys)                unsorted (ip << 32 | z0) keys, a power of two
//   [kKeys, kKeys + kEstAll)  estimate tables -k ln(z / k), z = 0 .. k (doubles),
//                             one per k_log2 = 5 .. SP_NOALLOC_MAX_K_LOG2,
//                             written once per device at set-up
//   [kKeys + kEstAll, + 2)    DetectStatus
constexpr uint32_t kKeys = SP_NOALLOC_MAX_RESULTS;            // 65536
constexpr uint32_t kMinKLog2 = 5;
// table of k_log2 = q starts at sum over q' < q of (2^q' + 1) doubles
constexpr uint32_t est_offset(uint32_t q) { return ((1u << q) - (1u << kMinKLog2)) + (q - kMinKLog2); }
constexpr uint32_t kEstAll = est_offset(SP_NOALLOC_MAX_K_LOG2 + 1);   // 8168
constexpr uint32_t kWords = kKeys + kEstAll + 2;

// Every GPU that loads the library holds this array (about 576 KiB) until
// the process exits.  All calls on a device share it.
static __device__ __align__(256) uint64_t sp_noalloc_scratch[kWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint64_t* g_scratch[kMaxDevices] = {};     // device address of the array, per device
double g_tables[kEstAll];                  // host copy of the estimate tables (static storage)
bool g_tables_ready = false;

// The host-side name sp_noalloc_scratch is only a stand-in; the device
// address comes from cudaGetSymbolAddress, once per device, with that device
// current.  The same set-up writes the estimate tables of every supported k
// into the array (one synchronous copy from static host memory), so later
// calls copy nothing from the host.
int scratch_for_current_device(uint64_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SP_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    if (!g_tables_ready) {
      for (uint32_t q = kMinKLog2; q <= SP_NOALLOC_MAX_K_LOG2; ++q) {
        double* t = g_tables + est_offset(q);
        const uint32_t k = 1u << q;
        t[0] = (double)k * log((double)k);   // saturated union: reported as k ln k
        for (uint32_t z = 1; z <= k; ++z) t[z] = -(double)k * log((double)z / (double)k);   // Eq. 4
      }
      g_tables_ready = true;
    }
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, sp_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SP_ERR_CUDA;
    }
    uint64_t* base = static_cast<uint64_t*>(p);
    if (cudaMemcpy(base + kKeys, g_tables, sizeof(g_tables), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      return SP_ERR_CUDA;
    }
    g_scratch[dev] = base;
  }
  *out = g_scratch[dev];
  return SP_OK;
}

uint64_t splitmix64_step(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" int sp_detect_noalloc(const sp_params* p, const uint8_t* dev_seav, const uint32_t* dev_ldca,
                                 uint32_t threshold, sp_candidate* dev_out, uint32_t cap,
                                 uint32_t* dev_status, void* cuda_stream) {
  if (!p || !dev_seav || !dev_ldca || !dev_status || (cap && !dev_out)) return SP_ERR_PARAM;
  if (sp_check_params(p) != SP_OK) return SP_ERR_PARAM;
  if (p->window_slices != 1) return SP_ERR_PARAM;                 // bits only, no stamps
  if (cap > SP_NOALLOC_MAX_RESULTS || p->k_log2 > SP_NOALLOC_MAX_K_LOG2) return SP_ERR_PARAM;
  if (((uintptr_t)dev_ldca & 15u) != 0 || ((uintptr_t)dev_status & 3u) != 0) return SP_ERR_PARAM;
  uint64_t* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != SP_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  // the kernel parameter block, as sp_create derives it
  sp::DevParams d;
  memset(&d, 0, sizeof(d));
  uint64_t s = p->seed;
  for (uint32_t i = 0; i < 2 + p->lr; ++i) {
    d.ha[i] = splitmix64_step(&s);
    d.hb[i] = splitmix64_step(&s);
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
  sp_sketch_bytes(p, &d.seav_bytes, &d.ldca_words);
  d.ldca_words /= 4;

  uint64_t* keys = scratch;
  const double* est = reinterpret_cast<const double*>(scratch + kKeys) + est_offset(p->k_log2);
  sp::DetectStatus* status = reinterpret_cast<sp::DetectStatus*>(scratch + kKeys + kEstAll);

  // the array keeps the previous call's contents: reset the status word (keys
  // are written before they are read, up to the count in the status word;
  // the estimate tables never change after set-up)
  if (cudaMemsetAsync(status, 0, sizeof(sp::DetectStatus), st) != cudaSuccess) return SP_ERR_CUDA;
  if (cap == 0) cap = 1;   // the kernels need room for one key; nothing is copied out
  const uint32_t zt = sp_z_theta(p->k_log2, threshold ? threshold : p->theta);
  const uint64_t max_join = p->max_join ? p->max_join : (1ull << 26);
  if (sp::launch_detect(d, dev_seav, dev_ldca, zt, keys, cap, max_join, status, st) != cudaSuccess) return SP_ERR_CUDA;
  if (dev_out &&
      sp::launch_sort_emit(keys, cap, status, est, p->k_log2, dev_out, st) != cudaSuccess) return SP_ERR_CUDA;
  // count and overflow flags to the caller's two words
  if (cudaMemcpyAsync(dev_status, status, 2 * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SP_ERR_CUDA;
  return (threshold && threshold < p->theta) ? SP_WARN_THETA_BELOW_INIT : SP_OK;
}
