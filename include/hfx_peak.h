/*
 * libhfx -- arithmetic peak of this GPU, measured, for the rooflines of the ALU-bound kernels
 * (the FP64 exchange path, the SIN(R) updates, the FP64 ACE contractions).
 *
 * The paper has no counterpart: it is measurement support.  The rate is taken, not assumed, because
 * the FP64 rate of this part is a small fraction of its FP32 rate and the nominal figures differ
 * between documents.
 */
#ifndef HFX_PEAK_H_
#define HFX_PEAK_H_

#include <stdint.h>

#include "hfx.h"

#ifdef __cplusplus
extern "C" {
#endif

/* hfx_fma_peak -- fused multiply-add throughput of the current device in TFLOP/s (2 flops per
 * FMA): every resident thread runs 8 independent FMA chains for `iters` iterations (FP64 when fp64
 * is nonzero, else FP32), timed with CUDA events on cuda_stream; *tflops receives the rate.
 * Synchronises the stream.  Allocates a small device buffer for the chains' results (so the
 * compiler keeps them) and frees it.  Returns HFX_ERR_INVALID_ARG (iters < 1, NULL tflops) or
 * HFX_ERR_CUDA.  (Measurement support; the paper has no counterpart.) */
hfx_status hfx_fma_peak(int32_t fp64, int32_t iters, double* tflops, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* HFX_PEAK_H_ */
