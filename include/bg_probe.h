/* bg_probe.h -- C ABI of libbg_probe.so, a measurement utility shipped beside
 * libbg.so (not part of the method, and not part of libbg.so).
 *
 * bgprobe_fma launches a kernel of independent fused multiply-adds on
 * `blocks` blocks of 256 threads, `iters` iterations of 16 FMAs per thread,
 * in FP32 (f32 != 0) or FP64, on `stream` (a cudaStream_t, NULL = the legacy
 * default stream), and stores in *flops (HOST) the number of floating-point
 * operations the kernel performs (2 per FMA).  Timing it with events on the
 * same stream measures the device's FMA pipe peak.  Returns 0 on success, 1
 * for invalid arguments (blocks < 1, iters < 1, flops NULL), 3 if the launch
 * failed.  Asynchronous: the kernel may still run when the call returns. */
#ifndef BG_PROBE_H
#define BG_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

int bgprobe_fma(int f32, int blocks, int iters, double* flops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BG_PROBE_H */
