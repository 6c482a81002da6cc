/*
 * qhd_probe.h -- arithmetic throughput probe of the current GPU, built as its
 * own library (libqhd_probe.so) beside the simulator.  It has no counterpart in
 * the paper and is not part of the simulator's ABI (qhd.h): the benchmark uses
 * it to state the roofline peaks that no datasheet gives for this part.
 */
#ifndef QHD_PROBE_H
#define QHD_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Timed loops of eight independent dependency chains per thread on every SM
 * (16 blocks of 256 threads per SM, CUDA events, one warm-up run each).
 * out (4 doubles, host): [0] FP32 FMAs/s, [1] 32 x 32 -> 64-bit integer
 * multiply-adds/s, [2] FP64 FMAs/s, [3] hardware sine approximations/s.
 * Allocates nothing; runs on the legacy default stream of the current device
 * and synchronises it.  Returns 0 on success, 1 for a NULL out, 4 for a failed
 * launch or event (the values of qhd_status in qhd.h). */
int qhd_probe_alu_rates(double *out);

#ifdef __cplusplus
}
#endif

#endif /* QHD_PROBE_H */
