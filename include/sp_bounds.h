/*
 * sp_bounds.h -- hardware probes behind the scan's roofline figures.
 *
 * The paper has no counterpart: these kernels measure the three rates that
 * bound the per-pair scan of Sec. 3.1-3.3 on the GPU running it -- streaming
 * reads from HBM (the pair stream), random 32-bit atomic ORs into an
 * L2-resident array (one per LDCA bit in the direct scan), and random 32-bit
 * atomic ORs into shared memory (one per LDCA bit in the binned scan's plane
 * pass).  Each call only enqueues one kernel on cuda_stream; the caller times
 * it (CUDA events on that stream).  Built into libspbounds.so, separate from
 * the detection library.
 *
 * Errors: 0 on success, -1 for an invalid argument, -5 when the launch
 * failed (the codes of superpoint.h).
 */
#ifndef SP_BOUNDS_H
#define SP_BOUNDS_H

#include <stdint.h>

#if defined(__GNUC__)
#define SPB_API __attribute__((visibility("default")))
#else
#define SPB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Reads dev_buf[0 .. bytes) once with 16-byte loads (bytes a multiple of 16,
 * dev_buf 16-byte aligned) and writes one XOR word per block to dev_sink
 * (grid words, so the loads are not optimised away).  grid blocks of 256
 * threads; grid = 0 picks 8 per SM. */
SPB_API int sp_probe_stream_read(const void* dev_buf, uint64_t bytes, uint32_t* dev_sink, uint32_t grid,
                                 void* cuda_stream);

/* ops_per_thread random atomic ORs of one bit into dev_words[0 .. 2^words_log2)
 * per thread, from grid blocks of 256 threads (grid = 0: 8 per SM); word
 * indices from a per-thread linear congruential sequence seeded by seed. */
SPB_API int sp_probe_l2_red(uint32_t* dev_words, uint32_t words_log2, uint32_t ops_per_thread, uint32_t grid,
                            uint32_t seed, void* cuda_stream);

/* ops_per_thread random atomic ORs of one bit into a shared-memory array of
 * 2^words_log2 32-bit words (words_log2 <= 13, 32 KiB) per block, grid
 * blocks of 512 threads (grid = 0: 4 per SM); each block ORs its array into
 * dev_sink[0 .. 2^words_log2) at the end.  The same index sequence as
 * sp_probe_l2_red. */
SPB_API int sp_probe_smem_atomic(uint32_t* dev_sink, uint32_t words_log2, uint32_t ops_per_thread, uint32_t grid,
                                 uint32_t seed, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SP_BOUNDS_H */
