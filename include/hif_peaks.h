/*
 * hif_peaks.h -- arithmetic peaks of the current GPU, measured.
 *
 * The paper has no counterpart: this is the measuring stick of the
 * benchmark.  The roofline fraction of a kernel of the factorization is its
 * algorithmic rate divided by the rate the same units reach in a loop that
 * does nothing else, so the denominators of the FMA-bound and tensor-bound
 * kernels are measured on the device they run on instead of taken from
 * data sheets.
 */
#ifndef HIF_PEAKS_H_
#define HIF_PEAKS_H_

#include "hif.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int sm_count;              /* multiprocessors of the current device */
  int sm_clock_khz;          /* its maximum SM clock (device attribute) */
  double fp32_fma_tflops;    /* dense FP32 FMA loop, every SM, 2 flops per FMA */
  double fp64_fma_tflops;    /* the same loop in FP64 */
  double tf32_mma_tflops;    /* tcgen05.mma kind::tf32, M = 128, N = 256, operands
                                in shared memory, FP32 accumulator in tensor memory */
  double bf16_mma_tflops;    /* the same with kind::f16 and BF16 operands (a
                                cross-check against a library GEMM's BF16 rate) */
  double seconds;            /* wall time the measurement took */
} hif_peaks;

/*
 * hif_measure_peaks -- time each loop with CUDA events on `stream` (each
 * launch sized to run for about 20-40 ms, best of three after a warm-up) and
 * fill *out.  Changes no clock or other device setting.  Every tensor-core
 * wait has an iteration limit; an expired wait returns HIF_ERR_TIMEOUT.
 * Errors: INVALID_ARG (out NULL), TIMEOUT, CUDA.
 */
hif_status hif_measure_peaks(hif_peaks* out, hif_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* HIF_PEAKS_H_ */
