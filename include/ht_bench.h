/*
 * ht_bench.h -- measurement helpers of libht.so (no counterpart in the paper).
 *
 * The evaluation and tracking kernels are bound by the FP64 pipe; the driver's
 * peak table has no FP64 figure, so the benchmark measures it live with this
 * call and reports kernel throughput as a fraction of it.
 */
#ifndef HT_BENCH_H
#define HT_BENCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * ht_bench_fp64_rate -- FP64 instruction throughput of the current device.
 * Runs independent fused multiply-add chains on every SM (enough warps to fill
 * the FP64 pipe), timed with CUDA events on `stream`, and writes the rate in
 * FP64 instructions per second (one DFMA per lane = one instruction; a DADD or
 * DMUL issues at the same rate on this pipe) to *ops_per_s.  Blocks until done.
 * Takes about `iters` x 20 microseconds.  Errors: HT_EINVAL (NULL output or
 * iters < 1), HT_ECUDA.
 */
int ht_bench_fp64_rate(int iters, double* ops_per_s, void* stream);

/*
 * ht_bench_imad_rate -- throughput of 32 x 32 -> 64-bit integer multiply-adds
 * (IMAD.WIDE, the limb product of the integer evaluation variant) on the
 * current device, in lane operations per second, measured like
 * ht_bench_fp64_rate.
 */
int ht_bench_imad_rate(int iters, double* ops_per_s, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HT_BENCH_H */
