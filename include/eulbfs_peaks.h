/*
 * eulbfs_peaks.h -- measured arithmetic throughput of the GPU, the
 * denominators of the EULBFS step's arithmetic rooflines.  The paper has no
 * counterpart: it states no hardware.  Exported by libeulbfs.so.
 *
 * Each call times one launch of a kernel in which every thread advances 32
 * independent FMA chains (a = a * b + c) for `iters` iterations, with the
 * grid filling every SM at full occupancy, so the FMA pipe, not latency or
 * memory, sets the rate.  One FMA counts as 2 floating-point operations.
 */
#ifndef EULBFS_PEAKS_H
#define EULBFS_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EULBFS_PEAK_FP32 = 0,      /* scalar FP32 FMA (one per lane per instruction) */
    EULBFS_PEAK_FP32X2 = 1,    /* packed FP32 FMA on float pairs (fma.rn.f32x2: two per lane) */
    EULBFS_PEAK_FP64 = 2       /* FP64 FMA */
} eulbfs_peak_kind;

/* Launch the FMA-chain kernel of `kind` for `iters` >= 1 iterations on
 * `stream` (a cudaStream_t, NULL: the legacy default stream), wait for it and
 * report the operations per second (*flops_per_s, 2 per FMA), the launch time
 * measured with CUDA events on that stream (*ms) and the warp instructions
 * per second that issued FMAs (*fma_warp_inst_per_s).  Allocates and frees a
 * small output buffer (one value per thread).  Errors: EULBFS_EINVAL (1) for
 * an unknown kind, iters < 1 or null outputs; EULBFS_ECUDA (3) for a CUDA
 * failure (the message is in eulbfs_last_error()). */
int eulbfs_peak_fma(int kind, long long iters, void* stream, double* flops_per_s, double* ms,
                    double* fma_warp_inst_per_s);

#ifdef __cplusplus
}
#endif
#endif
