/*
 * tsallis_testing.h -- test hooks of the thresholding library.
 *
 * Not part of the method's boundary. These entry points expose internal
 * arithmetic so that tests can check it against independent results.
 */
#ifndef TSALLIS_TESTING_H
#define TSALLIS_TESTING_H

#include "tsallis.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * For each of the n counts d_h[i] (device, uint32), writes the double-float
 * power (d_h[i] / N)^q used by the search, rounded to double, to d_pow[i]
 * (0 when d_h[i] is 0 or above N), and log2(d_h[i]) to d_log2[i] (0 for 0).
 * The double-float log2/exp2 behind both are documented to stay within a
 * relative error of 1e-12 for counts below 2^31 and 0 < q <= 4; this hook
 * exists so tests can hold them to that. Errors: TSALLIS_ERR_INVALID_ARG for
 * null pointers, n < 0, N == 0 or q outside (0, 4].
 */
tsallis_status tsallis_probe_dfmath(tsallis_ctx* ctx, const uint32_t* d_h, int64_t n, uint32_t N, float q,
                                   double* d_pow, double* d_log2, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* TSALLIS_TESTING_H */
