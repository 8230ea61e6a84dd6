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

/*
 * The proposer's top-k selection on caller data: for each of the B rows of
 * d_logits [B][4096] (device, float), the indices of its k largest values in
 * descending order, equal values ranked by the smaller index, into d_out
 * [B][k] (device). 1 <= k <= 256. Errors: TSALLIS_ERR_INVALID_ARG.
 */
tsallis_status tsallis_probe_topk(tsallis_ctx* ctx, const float* d_logits, int32_t B, int32_t k, int32_t* d_out,
                                  cudaStream_t stream);

/*
 * Predicted first-pass kernel: with on = 1 its prediction phase publishes no
 * prediction, so nothing is binarised in the first pass and every slice is
 * binarised after its search; results must be unchanged (statuses then lack
 * TSALLIS_STATUS_FIRST_PASS_EXACT). on = 0 restores normal operation.
 * TSALLIS_ERR_INVALID_ARG for a null context or another value of on.
 */
tsallis_status tsallis_test_withhold_predictions(tsallis_ctx* ctx, int32_t on);

/*
 * Checked build only (the library compiled with -DTSALLIS_CHECKED): the
 * kernels test the indices they compute against the extents of the buffers
 * they address, skip an access that fails and record the first failing
 * site. This call waits for the device, writes that site number to *site (0:
 * every check passed since the last call) and clears it. In normal builds it
 * returns TSALLIS_ERR_UNIMPLEMENTED. Site numbers: 101-103 the tile kernel
 * (group, tile, binarise queue), 201-206 pre-processing (staged word, voxel
 * read, disk window, intermediate word, output voxel, histogram level),
 * 301-303 the 2-D search (table entries, candidate cell, brute-force row),
 * 401-402 the predicted first-pass kernel (job slice, rewritten position).
 */
tsallis_status tsallis_check_status(tsallis_ctx* ctx, uint32_t* site);

#ifdef __cplusplus
}
#endif
#endif /* TSALLIS_TESTING_H */
