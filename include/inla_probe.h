/*
 * inla_probe.h -- measurement utilities of the benchmark (libinla_probe.so).
 *
 * No counterpart in the paper.  These functions time register-resident
 * arithmetic loops over every SM of one GPU, so that roofline fractions can be
 * quoted against throughputs measured on the same device and in the same run.
 * They are not part of the evaluation library (libinla_gpu.so) and read or
 * write none of its state.  Each allocates and frees a small device buffer
 * (one value per thread, so the compiler keeps the loops), synchronises the
 * device, and returns 0 on success or an inla_status code from inla_gpu.h
 * (INLA_ERR_ARG for a NULL output, INLA_ERR_CUDA / INLA_ERR_OOM when a CUDA call
 * fails), with a message from inla_probe_last_error().
 */
#ifndef INLA_PROBE_H
#define INLA_PROBE_H

#include "inla_gpu.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Sustained FP64 throughput of device `device` in TFLOP/s (2 flops per FMA):
 * use_tensor = 0 times scalar FMA, 1 the warp-level double-precision MMA
 * instruction (m8n8k4), 2 both at once (half the warps each), which shows
 * whether the two FP64 paths share one pipe.  Result in *tflops (HOST). */
int inla_measure_fp64_peak(int device, int use_tensor, double *tflops);

/* Sustained FP32 scalar FMA throughput of device `device` in TFLOP/s. */
int inla_measure_fp32_peak(int device, double *tflops);

/* Message of the last non-OK return of a probe on this thread ("" if none). */
const char *inla_probe_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* INLA_PROBE_H */
