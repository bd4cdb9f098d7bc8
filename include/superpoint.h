/*
 * superpoint.h -- C ABI of the GB300 super point detection library.
 *
 * The library implements the data-parallel path of the SLGA scheme of
 * Xu, Ding and Hu, "Most memory efficient distributed super points detection
 * on core networks" (arXiv 1901.07306):
 *
 *   scan      every <hip, oip> pair sets bits in the short estimator array
 *             vector (SEAV, Sec. 3.1-3.2) and the long estimator array
 *             (LDCA, Sec. 3.3) of one watch point (WP, Sec. 4.1);
 *   merge     the WPs' sketches are combined into the global ones (Sec. 4.2);
 *   detect    hot SEs -> candidate index sets -> SEU test -> LP/IP
 *             reconstruction (Eq. 3) -> LDCA union filter (Eq. 4), Sec. 3.2-3.3.
 *
 * Conventions shared by every call:
 *   - A pair stream is an array of uint32_t, two per pair: element 2j is the
 *     monitored host hip (source IP), element 2j+1 its opposite IP oip
 *     (Def. 1).  Addresses are plain host-order 32-bit integers.
 *   - "dev_" pointers are CUDA device pointers of the current device;
 *     "host_" pointers are host memory (pinned memory gives overlapped
 *     copies, pageable memory works but copies synchronously).
 *   - All GPU work of a context is issued on the context's stream.  Calls
 *     marked "async" return once the work is enqueued; the caller keeps
 *     inputs alive until the stream has passed that work.
 *   - Every call returns SP_OK (0), a positive warning, or a negative error
 *     code; sp_strerror() names it.  No call aborts the process.
 *   - The library owns all sketch, staging and scratch memory of a context;
 *     it is allocated in sp_create() and released by sp_destroy().
 *   - A context is not thread safe: one host thread at a time.
 *   - Every call that waits for the context's stream waits at most the
 *     context's bound (sp_set_timeout, default 60 s) and then returns
 *     SP_ERR_TIMEOUT with the work still in flight; only sp_destroy waits
 *     without a bound.
 */
#ifndef SUPERPOINT_H
#define SUPERPOINT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SP_API __attribute__((visibility("default")))
#else
#define SP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define SP_OK 0
#define SP_WARN_THETA_BELOW_INIT 1   /* detect threshold < params.theta (see sp_detect_async) */
#define SP_ERR_PARAM (-1)            /* invalid argument or parameter set */
#define SP_ERR_ROUTER (-2)           /* router index out of range */
#define SP_ERR_TRUNCATED (-3)        /* more results than the caller's cap; first cap written */
#define SP_ERR_CANDIDATE_OVERFLOW (-4) /* device result or join bound exceeded; list incomplete */
#define SP_ERR_CUDA (-5)             /* a CUDA runtime call failed */
#define SP_ERR_TIMEOUT (-6)          /* a wait for the stream passed the context's bound */
#define SP_ERR_CHECKSUM (-7)         /* imported sketch image is corrupt or mismatched */
#define SP_ERR_NOMEM (-8)            /* device or host allocation failed */
#define SP_ERR_STATE (-9)            /* call not valid in the context's current state */

/* sp_params.scan_mode */
#define SP_SCAN_AUTO 0u
#define SP_SCAN_DIRECT 1u
#define SP_SCAN_BINNED 2u

/* sp_candidate.flags */
#define SP_FLAG_SATURATED 1u         /* z0 == 0: the LDC union is full; est = k ln k */

/*
 * Parameters (Sec. 3.1-3.3; defaults by sp_default_params()).
 *
 * SEAV (Sec. 3.2): 2^r SEAs selected by RP = the low r bits of hip; each SEA
 * has sr rows, row i holding SC(i) = 2^ibn[i] one-byte SEs (g = 8 bits,
 * Sec. 3.1) indexed by Idx(i, LP) (Eq. 2) with LP = hip >> r.  The rows must
 * cover every LP bit (Sec. 3.2 constraint 1) and row i must share at least one
 * LP bit with row (i + 1) mod sr (constraint 2, read as an overlap).  Library
 * limits: r <= 24, 1 <= sr <= 8, 1 <= ibn[i] <= 12, isb[i] < 32 - r, and the
 * bytes of one SEA (sum of SC(i)) at most 4096.
 *
 * LDCA (Sec. 3.3): lr rows x 2^lc_log2 columns of LDCs of k = 2^k_log2 bits;
 * 5 <= k_log2 <= 16, 1 <= lr <= 8, lc_log2 <= 24, lr * 2^lc_log2 * k <= 2^32.
 *
 * theta fixes the SE sampling level tau = ceil(log2(theta / 8)) (Eq. 1) at
 * scan time; theta >= 1.
 *
 * n_routers sketches (one per simulated watch point) are held by the context.
 * window_slices = 1 is the discrete window of Sec. 3; 2 .. 128 selects the
 * sliding window W(t, k) of Sec. 5 over k = window_slices time slices: every
 * SEAV/LDCA bit gets a one-byte slice stamp (8x the sketch memory, plus a
 * second bit sketch: the router's bit sketch collects the current slice, the
 * other holds the window's bits for detect and export), a bit is active in
 * W(t, k) iff it was set in one of the slices t-k+1 .. t, and sp_slide()
 * advances t (see there).
 * max_candidates bounds the detect result buffer (0 = 1 << 20).
 * max_join bounds the LPs that reach the LDCA test in one detect (0 = 1 << 26).
 * scan_mode selects how the LDCA bits of a scan reach memory (results are
 * identical): SP_SCAN_AUTO (0) picks the binned form for updates of at least
 * 2^22 pairs when it applies (k <= 1024, LC >= 32, lr * LC <= 2^20), else the
 * direct form; SP_SCAN_DIRECT (1) sets every bit with an L2 atomic OR;
 * SP_SCAN_BINNED (2) groups the pairs' hips into lists by LDC bit position,
 * sets the bits of each bit plane with shared-memory atomics and folds the
 * planes into the LDCA before the next detect, merge or export (when it
 * applies).
 * seed seeds the hash family: multiply-add-shift hashes whose (a, b) words are
 * consecutive SplitMix64 outputs for H1, H3, LH_0 .. LH_{lr-1}.
 */
typedef struct sp_params {
  uint32_t r;
  uint32_t sr;
  uint32_t isb[8];
  uint32_t ibn[8];
  uint32_t k_log2;
  uint32_t lr;
  uint32_t lc_log2;
  uint32_t theta;
  uint32_t n_routers;
  uint32_t window_slices;
  uint32_t max_candidates;
  uint32_t scan_mode;
  uint64_t seed;
  uint64_t max_join;
} sp_params;

/* One detected super point (Def. 2 via Sec. 3.2-3.3).  z0 = zero bits of the
 * host's LDC union; est = -k ln(z0 / k) (Eq. 4), k ln k when saturated. */
typedef struct sp_candidate {
  uint32_t ip;
  uint32_t z0;
  double est;
  uint32_t flags;
  uint32_t pad;
} sp_candidate;

typedef struct sp_ctx sp_ctx;

/* Fills *out with the default profile: r = 14, sr = 4, isb = {0, 5, 10, 15},
 * ibn = 7 (the Sec. 3.2 rule IBN = ceil(L / SR) + a, ISB(i) = i ceil(L / SR)
 * with L = 18, a = 2), k = 1024, lr = 4, LC = 2^16, theta = 1024, one router,
 * discrete window.  SEAV = 8 MiB, LDCA = 32 MiB. */
SP_API int sp_default_params(sp_params* out);

/* Validates *p against the Sec. 3.2 constraints and the library limits above.
 * Returns SP_OK or SP_ERR_PARAM. */
SP_API int sp_check_params(const sp_params* p);

/* Bytes of one router's SEAV and LDCA for *p (the logical layout that
 * sp_export writes).  Either output may be NULL. */
SP_API int sp_sketch_bytes(const sp_params* p, uint64_t* seav_bytes, uint64_t* ldca_bytes);

/* tau of Eq. 1 and Z_theta = max{ z in [0, k] : -k ln(z / k) >= threshold }
 * (Eq. 4 as an integer test), as the library computes them. */
SP_API uint32_t sp_tau(uint32_t theta);
SP_API uint32_t sp_z_theta(uint32_t k_log2, uint32_t threshold);

/* Lemma 1 (Sec. 3.4): probability that a bit of a host's LDC union (the AND
 * over the lr rows) is 1 when n_pairs distinct pairs are spread uniformly over
 * the 2^lc_log2 columns of each row: (1 - (1 - 1/k)^(n / LC))^lr. */
SP_API double sp_psu(uint64_t n_pairs, uint32_t k_log2, uint32_t lr, uint32_t lc_log2);

/* LDCA sizing (Sec. 3.4, Lemma 1 and Theorem 1) for an expected n_pairs
 * distinct pairs per window and a budget of ldc_budget LDCs of k = 2^k_log2
 * bits: *lr and *lc_log2 receive the layout (lr in 1..8, LC a power of two,
 * lr * LC <= ldc_budget, within the library limits) with the smallest Psu,
 * fewer rows on ties; *psu its Psu; *lr_star Theorem 1's continuous optimum
 * -V ln 2 / (n ln(1 - 1/k)) for V = ldc_budget.  Any output may be NULL.
 * Errors: SP_ERR_PARAM (n_pairs = 0, k_log2 out of 5..16, ldc_budget = 0). */
SP_API int sp_size_ldca(uint64_t n_pairs, uint32_t k_log2, uint64_t ldc_budget, uint32_t* lr,
                        uint32_t* lc_log2, double* psu, double* lr_star);

/* Creates a context on the current CUDA device.  cuda_stream is a
 * cudaStream_t (NULL = the legacy default stream); the context issues all
 * its work there.  Allocates and zeroes n_routers sketches plus scratch.
 * Errors: SP_ERR_PARAM, SP_ERR_NOMEM, SP_ERR_CUDA.  *out is NULL on error. */
SP_API int sp_create(const sp_params* p, void* cuda_stream, sp_ctx** out);

/* Releases every resource of ctx after draining its stream (this wait has no
 * bound).  NULL is a no-op. */
SP_API void sp_destroy(sp_ctx* ctx);

/* Replaces the context's stream (work already issued stays ordered on the old
 * one; the caller synchronises if needed). */
SP_API int sp_set_stream(sp_ctx* ctx, void* cuda_stream);

/* Bound of every wait of the context on its stream (sp_results, sp_detect,
 * sp_export, sp_import, sp_autotune, and sp_update_batched when its ring of
 * batch tables is full): a wait that has not seen the stream's work complete
 * after timeout_ms milliseconds returns SP_ERR_TIMEOUT, leaving the work in
 * flight (a later call may wait for it again; buffers the work reads or
 * writes stay in use until it completes).  0 = wait without a bound.  The
 * default of sp_create is 60,000 ms.  The paper has no counterpart: this is
 * the failure detection of a watch point whose GPU stopped making progress,
 * done on the host (the library's kernels never wait on a flag).  Errors:
 * SP_ERR_PARAM (ctx NULL). */
SP_API int sp_set_timeout(sp_ctx* ctx, uint32_t timeout_ms);

/* Allocates now the device and pinned host buffers that updates of routers
 * first .. first + count - 1 would otherwise allocate on first use: the two
 * staging buffers of sp_update_host, the ring of batch tables of
 * sp_update_batched (room for 1,024 batches per call each), and, where the
 * binned scan applies to the parameter set, its bin lists and the routers'
 * accumulator planes.  A loop that must not stall on an allocation (a server
 * acknowledging batches) calls it once before it starts.  Optional: every
 * update still allocates what is missing.  Synchronous on the host (it
 * allocates), issues no stream work.  Errors: SP_ERR_PARAM (ctx NULL),
 * SP_ERR_ROUTER (range outside the context), SP_ERR_NOMEM, SP_ERR_CUDA. */
SP_API int sp_reserve(sp_ctx* ctx, uint32_t first, uint32_t count);

/* Copy of the parameters the context was created with. */
SP_API int sp_get_params(const sp_ctx* ctx, sp_params* out);

/* Starts a new discrete window for one router (Sec. 3: every bit is 0 at the
 * beginning of a time period): zeroes its SEAV and LDCA.  Async.
 * In a sliding context it also forgets every slice.  Errors: SP_ERR_ROUTER. */
SP_API int sp_reset(sp_ctx* ctx, uint32_t router);

/* sp_reset for routers first .. first + count - 1 (a new discrete window for
 * every watch point at once, Sec. 3): their sketches are contiguous, so one
 * zeroing launch covers them.  Async.  Errors: SP_ERR_ROUTER (range outside
 * the context). */
SP_API int sp_reset_range(sp_ctx* ctx, uint32_t first, uint32_t count);

/* Scan (Sec. 3.1-3.3, Sec. 4.1): for every pair of dev_pairs[0 .. 2 n_pairs),
 * sets bit H2(oip) of the SE at Idx(i, LP(hip)) in every row i of SEA RP(hip)
 * when lsb(H1(oip)) >= tau, and bit H3(oip) of LDC LH_i(hip) in every LDCA
 * row i.  dev_pairs is borrowed until the stream passes the work; it must be
 * 8-byte aligned.  n_pairs = 0 is a no-op.  Bit setting is idempotent and
 * order independent (Sec. 3.4), so updates may be split arbitrarily.
 * In a sliding context the bits go to the router's slice sketch, whose set
 * bits are stamped with the current slice (and the sketch cleared) before the
 * slice closes and before a detect, merge or export reads the window.  Async.
 * Errors: SP_ERR_ROUTER, SP_ERR_PARAM (NULL or misaligned pointer), SP_ERR_CUDA. */
SP_API int sp_update(sp_ctx* ctx, uint32_t router, const uint32_t* dev_pairs, uint64_t n_pairs);

/* The watch point's host path of Sec. 4.1: host_pairs are copied to the GPU
 * in fixed-size chunks through two device staging buffers, the copy of chunk
 * j + 1 overlapping the scan of chunk j.  Returns when every chunk is
 * enqueued; host_pairs must stay valid until the stream has passed them.
 * Same semantics and errors as sp_update. */
SP_API int sp_update_host(sp_ctx* ctx, uint32_t router, const uint32_t* host_pairs, uint64_t n_pairs);

/* One batch of a batched scan: n_pairs pairs for one router (8-byte aligned
 * device stream).  The device form of the table is read by the kernels. */
typedef struct sp_batch {
  const uint32_t* pairs;
  uint64_t n_pairs;
  uint32_t router;
  uint32_t reserved;
} sp_batch;

/* Batched scan (the WPs of Sec. 4.1 fed together): n_batches
 * (router, pairs, n_pairs) triples of device streams of uneven sizes, given as
 * three host arrays; routers[b] may repeat.  Routers whose batches add up to
 * at least 2^22 pairs take the binned scan (one binning launch per batch, one
 * plane launch per router); all other batches are scanned by ONE persistent
 * launch over a batch table, whose block shape comes from sp_autotune (or a
 * default).  Same per-batch semantics and errors as sp_update.  A stream may
 * also be page-locked host memory mapped into the device's address space
 * (cudaHostAlloc or cudaHostRegister; under unified addressing the host
 * pointer is the device pointer): the kernels then read it in place across
 * the host link (NVLink-C2C on a Grace-Blackwell node), with no staging copy.
 * Async; the table goes to the device through a context-owned pinned buffer,
 * so the call is not valid inside a stream capture (SP_ERR_STATE): capture
 * sp_update_batched_device instead. */
SP_API int sp_update_batched(sp_ctx* ctx, uint32_t n_batches, const uint32_t* routers,
                             const uint32_t* const* dev_pairs, const uint64_t* n_pairs);

/* Batched scan of batches in host memory (the serving path of many watch
 * points, Sec. 4.1): copies batch b (host_pairs[b], n_pairs[b] pairs; pinned
 * memory makes the copies asynchronous) into dev_arena -- caller-owned device
 * memory of arena_bytes, 16-byte aligned; the batches are packed in order,
 * each at a 16-byte boundary -- on copy_stream (a cudaStream_t, NULL = the
 * legacy default stream), makes the context's stream wait for the copies, and
 * scans them as sp_update_batched does.  One call per engine step, the copy
 * loop in C.  The caller orders copy_stream after the last scan that read the
 * arena, and keeps the host buffers and the arena alive until the stream has
 * passed the scan.  Async.  Errors: SP_ERR_PARAM (NULL or misaligned arena,
 * the batches do not fit it), SP_ERR_ROUTER, SP_ERR_STATE (inside a stream
 * capture), SP_ERR_CUDA. */
SP_API int sp_update_batched_host(sp_ctx* ctx, uint32_t n_batches, const uint32_t* routers,
                                  const uint32_t* const* host_pairs, const uint64_t* n_pairs, void* dev_arena,
                                  uint64_t arena_bytes, void* copy_stream);

/* Batched scan over a table that already lives in device memory
 * (dev_batches[0 .. n_batches), n_batches <= 8192), always by the one
 * persistent launch (direct form).  The kernel reads sizes and pointers when it
 * runs, so a CUDA graph that captured this call can be replayed after the
 * caller rewrites the table.  A batch whose router is out of range or whose
 * stream is misaligned is skipped and makes the next sp_results return
 * SP_ERR_ROUTER.  In a sliding context every router counts as updated (its
 * slice sketch is committed at the next slide, detect, merge or export).
 * Async. */
SP_API int sp_update_batched_device(sp_ctx* ctx, const sp_batch* dev_batches, uint32_t n_batches);

/* Autotuner of the batched launch: times every compiled block shape
 * (128 / 256 / 512 threads) at 1, 2 and 4 blocks per SM (and the most that fit)
 * on router 0 with the caller's sample stream dev_pairs[0 .. 2 n_pairs)
 * (scanned repeatedly; router 0's sketch is reset afterwards), keeps the
 * fastest for this context and reports it.  Synchronises the stream.
 * Either output may be NULL. */
SP_API int sp_autotune(sp_ctx* ctx, const uint32_t* dev_pairs, uint64_t n_pairs,
                       uint32_t* best_threads, uint32_t* best_blocks);

/* Staging shape of the binned scan (an implementation choice; the paper's
 * per-pair update of Sec. 3.3 fixes only the bits, which every shape gives
 * exactly): the binning block size, the hips a bin's shared-memory row
 * holds, the tiles binned between two flushes of the rows to the lists, the
 * binning blocks per SM, and the block size of the plane pass. */
typedef struct sp_binned_shape {
  uint32_t index;                /* position in the compiled list */
  uint32_t bin_threads;
  uint32_t bin_stage;
  uint32_t bin_tiles_per_round;
  uint32_t bin_blocks_per_sm;
  uint32_t apply_threads;
} sp_binned_shape;

/* The compiled staging shapes: *n receives their number, out[0 .. min(cap, *n))
 * their description (out may be NULL when cap = 0).  Shape 0 is the default. */
SP_API int sp_binned_shapes(sp_binned_shape* out, uint32_t cap, uint32_t* n);

/* Selects staging shape `index` for the context's later binned scans (results
 * are identical for every shape).  Errors: SP_ERR_PARAM (index out of range). */
SP_API int sp_set_binned_shape(sp_ctx* ctx, uint32_t index);

/* The context's current staging shape. */
SP_API int sp_get_binned_shape(const sp_ctx* ctx, sp_binned_shape* out);

/* Autotuner of the binned scan: times every compiled staging shape on router
 * 0 with the caller's sample stream dev_pairs[0 .. 2 n_pairs) (a binned scan
 * of it, 3 times after a warm-up), keeps the fastest for this context and
 * reports it in *best (may be NULL).  Router 0's sketch is reset afterwards.
 * Synchronises the stream.  Errors: SP_ERR_PARAM (NULL, empty or misaligned
 * sample), SP_ERR_STATE (the parameters rule the binned scan out: k > 1024,
 * LC < 32 or lr * LC > 2^20), SP_ERR_NOMEM, SP_ERR_CUDA, SP_ERR_TIMEOUT. */
SP_API int sp_autotune_binned(sp_ctx* ctx, const uint32_t* dev_pairs, uint64_t n_pairs, sp_binned_shape* best);

/* Global SEAV/LDCA of Sec. 4.2: dst |= src for every source router, bitwise
 * OR over both structures (the OR of the WPs' sketches equals the sketch of
 * the union of their streams).  routers is a host array of n indices; it may
 * contain dst_router.  In a sliding context every listed router must be at
 * the same slice as dst (else SP_ERR_STATE) and each stamp becomes the
 * youngest of the routers' stamps, which ORs every window.  Async.
 * Errors: SP_ERR_ROUTER, SP_ERR_PARAM, SP_ERR_STATE. */
SP_API int sp_merge(sp_ctx* ctx, const uint32_t* routers, uint32_t n, uint32_t dst_router);

/* Device image of one router for a WP -> GS shipment that stays in device
 * memory (Sec. 4.2 over NCCL or another device transport): copies the
 * router's sketch to dev_dst (device memory, 16-byte aligned) on the stream,
 * in the context's device layout -- the SEAV bytes [2^r][sum SC(i)], zero
 * padding to a multiple of 256 bytes, the LDCA words [lr][LC][k / 32], zero
 * padding to a multiple of 256 bytes -- which is the same for every context
 * with the same parameters.  Pending binned-scan planes are folded first; a
 * sliding context copies the bits of its current window.  With dev_dst NULL
 * *n receives the image size.  Async.  Errors: SP_ERR_TRUNCATED (cap too
 * small), SP_ERR_ROUTER, SP_ERR_PARAM (misaligned dev_dst), SP_ERR_CUDA. */
SP_API int sp_copy_sketch(sp_ctx* ctx, uint32_t router, void* dev_dst, uint64_t cap, uint64_t* n);

/* Global SEAV/LDCA of Sec. 4.2 from images in device memory: dst |= every
 * image of dev_images[0 .. n) (a host array of device pointers, each image
 * 16-byte aligned, written by sp_copy_sketch of a context with the same
 * parameters -- e.g. gathered from other GPUs), bitwise OR over the whole
 * image on the GPU.  The images are read when the stream reaches the merge.
 * Async.  Discrete contexts only (SP_ERR_STATE in a sliding context).
 * Errors: SP_ERR_ROUTER, SP_ERR_PARAM (NULL or misaligned image), SP_ERR_CUDA. */
SP_API int sp_merge_device(sp_ctx* ctx, const void* const* dev_images, uint32_t n, uint32_t dst_router);

/* Restore + filter (Sec. 3.2-3.3) on one router's sketch, enqueued on the
 * stream: HSE(i) = SEs of weight >= 3; every candidate index set of the
 * cartesian product whose rows agree on their shared LP bits and whose SEU
 * (AND of the chosen SEs) has weight >= 3 gives LP by Eq. 3 and
 * ip = LP << r | RP; ip is kept when the AND of its LDCs over all LDCA rows has
 * z0 <= Z_theta(threshold) zero bits.  Results are sorted by ascending ip and
 * stay on the device until sp_results().  threshold 0 means params.theta.
 * Returns SP_WARN_THETA_BELOW_INIT when threshold < params.theta (tau, and so
 * the SE sensitivity, was fixed at scan time).  Errors: SP_ERR_ROUTER,
 * SP_ERR_CUDA. */
SP_API int sp_detect_async(sp_ctx* ctx, uint32_t router, uint32_t threshold);

/* Waits for the stream, then copies the last detect's results:
 * *n_total = number of super points found; the first
 * min(*n_total, max_candidates, cap) records, in ascending ip order, go to
 * host_out (may be NULL when cap = 0).  Errors: SP_ERR_TRUNCATED when
 * *n_total > cap; SP_ERR_CANDIDATE_OVERFLOW when the device result buffer
 * (max_candidates) or the join bound (max_join) overflowed, in which case the
 * list is incomplete; SP_ERR_ROUTER when a device batch table named a bad
 * router or stream since the last check (that batch was skipped);
 * SP_ERR_TIMEOUT when the wait for the stream passed the context's bound
 * (sp_set_timeout; nothing was written, the detect is still in flight and a
 * later sp_results may collect it); SP_ERR_STATE when no detect was issued;
 * SP_ERR_CUDA. */
SP_API int sp_results(sp_ctx* ctx, sp_candidate* host_out, uint64_t cap, uint64_t* n_total);

/* Non-blocking form of sp_results for pipelines: enqueues on the stream the
 * copies of the last detect's status -- host_status[0] = super points found,
 * host_status[1] = overflow flags (1: result buffer, 2: join bound) -- and of
 * the first min(cap, max_candidates) result slots to host_out; only the first
 * min(host_status[0], cap) of them are valid.  Pinned host memory makes the
 * copies asynchronous; the caller waits on the stream (or an event) before
 * reading.  Errors: SP_ERR_STATE when no detect was issued, SP_ERR_PARAM,
 * SP_ERR_CUDA. */
SP_API int sp_results_async(sp_ctx* ctx, sp_candidate* host_out, uint64_t cap, uint32_t* host_status);

/* sp_detect_async followed by sp_results. */
SP_API int sp_detect(sp_ctx* ctx, uint32_t router, uint32_t threshold,
              sp_candidate* host_out, uint64_t cap, uint64_t* n_total);

/* Device view of the last detect's sorted results (valid until the next
 * detect): *dev_records points at max_candidates sp_candidate slots,
 * *dev_count at the uint32 count of valid ones (which may exceed
 * max_candidates on overflow).  No synchronisation. */
SP_API int sp_results_device(sp_ctx* ctx, const sp_candidate** dev_records, const uint32_t** dev_count);

/* Sliding window (Sec. 5): closes the current time slice t of one router of a
 * sliding context and opens slice t + 1 (t starts at 0 after sp_create or
 * sp_reset); bits last set more than window_slices - 1 slices ago become
 * inactive ("0") for detect, merge and export.  Each call also sweeps one of
 * 255 - window_slices segments of the router's stamps (the per-slice counter
 * maintenance of Sec. 5.2), so a call costs 1/(255 - k) of a pass over them.
 * The slice clock t lives in device memory and the kernels read it there, so
 * the per-slice step -- sp_slide, sp_update_batched_device on a table the
 * caller rewrites, sp_detect_async -- can be recorded once in a CUDA graph
 * and replayed slice after slice (each replay advances t).  The library's
 * host-side count of sp_slide calls (sp_merge's same-slice check) does not
 * see replays.  Async.  In a discrete context (window_slices = 1) it equals
 * sp_reset.  Errors: SP_ERR_ROUTER. */
SP_API int sp_slide(sp_ctx* ctx, uint32_t router);

/* Checkpoint / WP->GS shipment (Sec. 4.2): a self-describing image of one
 * router's sketch in the logical layout -- header, SEAV bytes
 * [2^r][sum SC(i)], LDCA words [lr][LC][k / 32] (bit b of an LDC is bit
 * b % 32 of word b / 32) -- followed by a 64-bit checksum.  With host_buf NULL
 * *n receives the image size.  A sliding context exports the bits of its
 * current window.  Synchronises the stream.
 * Errors: SP_ERR_TRUNCATED (cap too small), SP_ERR_ROUTER, SP_ERR_CUDA,
 * SP_ERR_TIMEOUT (the copies into host_buf are still in flight: it stays in
 * use until the stream passes them, and it holds no checksum). */
SP_API int sp_export(sp_ctx* ctx, uint32_t router, void* host_buf, uint64_t cap, uint64_t* n);

/* Loads an image written by sp_export into a router, replacing its sketch.
 * Rejects an image with a bad checksum or parameters other than the
 * context's (SP_ERR_CHECKSUM) without touching the router.  A sliding context
 * cannot import window bits (SP_ERR_STATE).  Synchronises the stream;
 * SP_ERR_TIMEOUT leaves the copies from host_buf in flight (it stays in use
 * until the stream passes them). */
SP_API int sp_import(sp_ctx* ctx, uint32_t router, const void* host_buf, uint64_t n);

/* Limits of sp_detect_noalloc. */
#define SP_NOALLOC_MAX_RESULTS 65536u
#define SP_NOALLOC_MAX_K_LOG2 12u

/* Detect without allocating.  The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory when they detect --
 * programs whose device memory is owned by another allocator (a framework's
 * caching allocator, a partition fixed at start-up) or budgeted up front, and
 * latency-critical loops that cannot take an allocation, or its failure, on
 * their path.  It runs the same restore and filter as sp_detect_async on a
 * sketch the caller holds:
 *   p          parameters the sketch was built with (validated; discrete
 *              window only; k_log2 <= SP_NOALLOC_MAX_K_LOG2)
 *   dev_seav   one router's SEAV, device memory, the sp_export layout
 *   dev_ldca   its LDCA, device memory, 16-byte aligned, the sp_export layout
 *   threshold  0 means p->theta
 *   dev_out    device array of cap records, sorted by ascending ip
 *              (min(count, cap) are written); may be NULL when cap = 0
 *   cap        at most SP_NOALLOC_MAX_RESULTS
 *   dev_status two device uint32 words: [0] = super points found (may exceed
 *              cap; then the list holds an unspecified subset), [1] = overflow
 *              flags (1: more than cap found, 2: the join bound was hit)
 *   cuda_stream the stream the work is enqueued on (async)
 * It calls no cudaMalloc, cudaFree or other allocating routine.  Its scratch
 * is one fixed array of about 576 KiB in the library's device image, held by
 * every GPU that loads the library until the process exits.  The first call
 * on each device sets the array up: it looks up the array's device address
 * (cudaGetSymbolAddress, with the device current) and writes the estimate
 * tables of every supported k into it with one synchronous copy, so make that
 * first call before any stream capture begins.  Later calls copy nothing
 * from the host.  All calls on a device share the array and it keeps the
 * last call's contents (each call resets what must start from zero): calls
 * that overlap on the GPU -- on different streams, or from different host
 * threads -- race and give undefined results.  Errors: SP_ERR_PARAM (a limit above exceeded,
 * invalid parameters, misaligned pointer), SP_ERR_CUDA; returns
 * SP_WARN_THETA_BELOW_INIT like sp_detect_async. */
SP_API int sp_detect_noalloc(const sp_params* p, const uint8_t* dev_seav, const uint32_t* dev_ldca,
                             uint32_t threshold, sp_candidate* dev_out, uint32_t cap,
                             uint32_t* dev_status, void* cuda_stream);

/* Human-readable name of a status code (static storage). */
SP_API const char* sp_strerror(int code);

/* Library version as MAJOR * 10000 + MINOR * 100 + PATCH. */
SP_API int sp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SUPERPOINT_H */
