/* gr_measure.h -- measurement helpers of libgr.so (not part of the rendering
 * method; the paper has no counterpart).  Conventions as in gr.h. */
#ifndef GR_MEASURE_H
#define GR_MEASURE_H

#include "gr.h"

#ifdef __cplusplus
extern "C" {
#endif

/* FP32 FMA throughput of the current device, the denominator of the ALU
 * roofline of the BVH traversal kernels (which are FP32 slab and edge-function
 * arithmetic): 16 independent fmaf chains per thread, 64 warps per SM, one
 * warm-up launch then the best of three, timed with CUDA events on
 * cuda_stream (a cudaStream_t, NULL = legacy default stream); synchronises
 * that stream.  Writes TFLOP/s (2 FLOP per fmaf) to *tflops_out and the
 * fastest launch's milliseconds to *ms_out.  Allocates and frees a small
 * device buffer on the stream.  GR_E_INVALID for null out-pointers,
 * GR_E_CUDA (message in gr_last_error) for a CUDA failure. */
gr_status gr_measure_fp32_peak(void* cuda_stream, double* tflops_out, double* ms_out);

#ifdef __cplusplus
}
#endif

#endif /* GR_MEASURE_H */
