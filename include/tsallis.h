/*
 * tsallis.h -- C ABI of the GB300 maximum-Tsallis-entropy thresholding path.
 *
 * The method (Chang & Sheu, "GPU acceleration of a patient-specific airway
 * image segmentation and its assessment", section II-C "Segmentation"):
 *   1. histogram of grey levels (section I "Thresholding", Fig. 2), or the
 *      2-D histogram of grey level x 3x3(x3) floor-mean level (section II-C,
 *      "Tsallis entropy", the mean-image and h(i, j) equations);
 *   2. class masses P_1, P_2 and class Tsallis entropies H_1^alpha, H_2^alpha
 *      for every threshold t (or pair (t, s));
 *   3. the pseudo-additive objective
 *          phi_alpha = H_1 + H_2 + (1 - alpha) H_1 H_2,
 *      maximised over all thresholds;
 *   4. Algorithm 1 (thresholding kernel): every voxel is set to 1 or 0 by
 *      comparing its level with the chosen threshold.
 * alpha is called q below.
 *
 * Conventions shared by every entry point:
 *   - All device pointers are plain CUDA device addresses owned by the
 *     caller. The library never frees them and keeps no reference after the
 *     call returns. Work is enqueued on the given stream and runs
 *     asynchronously; results are valid after the stream is synchronised.
 *   - Volumes are int16 Hounsfield values laid out [nz][ny][nx], x fastest,
 *     contiguous. Masks are uint8 [nz][ny][nx] holding 0 or 1.
 *   - Volume and mask base pointers must be 16-byte aligned (any cudaMalloc
 *     result is) unless an entry point states its own rule
 *     (tsallis_preprocess, tsallis_segment_host); otherwise
 *     TSALLIS_ERR_ALIGNMENT is returned. Any nx, ny, nz is accepted; ragged
 *     tails are handled inside the kernels.
 *   - Argument, size and alignment errors are returned synchronously, before
 *     anything is enqueued. Data-dependent outcomes (no valid threshold, a
 *     device wait that ran out) are written per histogram to d_status and are
 *     read after synchronising.
 *   - A context owns scratch memory on its device. Calls on one context must
 *     not overlap in time on different streams (they share that scratch).
 *     Contexts are independent of each other.
 */
#ifndef TSALLIS_H
#define TSALLIS_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TSALLIS_OK = 0,
    TSALLIS_ERR_INVALID_ARG = 1,       /* null pointer, bad size, q outside (0, 4], ... */
    TSALLIS_ERR_ALIGNMENT = 2,         /* a volume or mask pointer is not 16-byte aligned */
    TSALLIS_ERR_CUDA = 3,              /* a CUDA runtime call failed */
    TSALLIS_ERR_NO_VALID_THRESHOLD = 4,/* per histogram: fewer than two non-empty levels */
    TSALLIS_ERR_TIMEOUT = 5,           /* per histogram: a bounded device wait ran out */
    TSALLIS_ERR_OOM = 6,               /* scratch allocation failed */
    TSALLIS_ERR_UNIMPLEMENTED = 7
} tsallis_status;

/* Extra bits OR-ed into d_status entries (low byte holds a tsallis_status). */
#define TSALLIS_STATUS_RERANKED 0x100  /* FP64 re-rank decided between near-tied candidates */
#define TSALLIS_STATUS_WINDOW_HIT 0x400    /* window search: the maximiser was among the
                                            proposed candidates */
#define TSALLIS_STATUS_FALLBACK_SHIFT 16   /* window search: bits 16..23 hold how many
                                              64-level blocks (1-D) or 4x4-pair cells (2-D,
                                              saturating at 255) beyond the proposals were
                                              searched exhaustively */
#define TSALLIS_STATUS_FIRST_PASS_EXACT 0x200  /* the mask written in the histogram pass with a
                                                  predicted threshold was already exact, so the
                                                  group was not read a second time */

typedef enum {
    TSALLIS_PER_SLICE = 0,    /* one histogram and threshold per z slice */
    TSALLIS_WHOLE_VOLUME = 1  /* one histogram and threshold for the whole volume */
} tsallis_mode;

typedef enum {
    TSALLIS_MASK_LOW = 0,  /* mask = 1 where level <= t (class 1: the low-HU lumen) */
    TSALLIS_MASK_HIGH = 1  /* mask = 1 where level >= t + 1 (Algorithm 1 with T = t + 1) */
} tsallis_polarity;

/* Debug flags (tests only). */
#define TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL 0x1u /* tile and cluster kernels (and
                                                tsallis_segment_static): the first histogram
                                                tile never reports arrival, so waits on its
                                                histogram run out and its group reports
                                                TSALLIS_ERR_TIMEOUT; predicted first-pass kernel:
                                                one block never arrives at the grid barrier
                                                after the streaming phase, the barrier's wait
                                                runs out and every slice of the call reports
                                                TSALLIS_ERR_TIMEOUT; pipelined kernel: the
                                                first chunk never arrives on its slice's
                                                counter, the wait for that slice's threshold
                                                runs out and every slice of the call reports
                                                TSALLIS_ERR_TIMEOUT */
/* tsallis_segment_batch, whole-volume mode: binarise in the histogram pass
 * with a threshold predicted from the histogram of the middle sixteenth of
 * each volume's slices, by the proposer (PREDICT_PROPOSER; needs one, see
 * tsallis_proposer_set) or by the exhaustive search of that histogram
 * (PREDICT_SUBSAMPLE). When no voxel of a volume has a level between the
 * predicted and the exact threshold, the mask written in the histogram pass
 * is kept (3 bytes per voxel plus the sixteenth, instead of 5); otherwise the
 * volume is binarised again. Results are those of the exhaustive path; only
 * the memory traffic changes. Statuses of volumes finished without a second
 * read carry TSALLIS_STATUS_FIRST_PASS_EXACT. */
#define TSALLIS_FLAG_PREDICT_PROPOSER 0x2u
#define TSALLIS_FLAG_PREDICT_SUBSAMPLE 0x4u
/* 2-D form only (two_d = 1, else TSALLIS_ERR_INVALID_ARG): search as the
 * paper's GPU code does (section III, Table 4), one thread per threshold
 * pair (t, s) summing its quadrants directly, O(L2^2) per pair, instead of
 * through summed-area tables. Counts are exact; terms are pairs of floats
 * summed with compensation, row by row, and the rows in FP64, so each pair's
 * objective (formed in FP64) carries a bound of about 1e-9 relative; the
 * pairs whose bounds reach the largest lower bound are evaluated again in
 * plain FP64 and the largest wins. Same outputs, tie rule (smallest t, then
 * s) and curve as the default search; statuses never carry
 * TSALLIS_STATUS_RERANKED. A comparison point: far slower than the default
 * search. */
#define TSALLIS_FLAG_BRUTE_FORCE_2D 0x8u

typedef struct {
    int32_t lo;       /* Hounsfield value of level 0, -32768..32767; default -1024 */
    int32_t nbins;    /* L, number of 1-D levels, 2..4096; default 4096. Level of a
                         voxel v is b = clamp(v - lo, 0, L - 1). */
    float q;          /* Tsallis index (alpha), 0 < q <= 4; q == 1 selects the
                         Shannon (Kapur) limit. Default 0.8 */
    int32_t mode;     /* tsallis_mode; default TSALLIS_PER_SLICE */
    int32_t polarity; /* tsallis_polarity; default TSALLIS_MASK_LOW */
    int32_t two_d;    /* 0: 1-D form; 1: 2-D grey x mean form. Default 0 */
    int32_t shift;    /* 2-D only: grey level = b >> shift, giving L2 = nbins >> shift
                         levels (2..256); default 4 */
    int32_t topk;     /* 0: exhaustive search (default); 1..256: window search of the
                         proposer's topk candidates, certified by per-block bounds;
                         1-D: nbins 4096 and proposer slot 0; 2-D: 256 grey levels and
                         slot 1 (see tsallis_proposer_set and tsallis_proposer_select) */
    uint32_t flags;   /* TSALLIS_FLAG_* */
} tsallis_params;

typedef struct tsallis_ctx tsallis_ctx;

/* Fills p with the defaults listed above. */
tsallis_status tsallis_params_default(tsallis_params* p);

/* Human-readable name of a status code (the low byte of d_status entries). */
const char* tsallis_status_string(int32_t status);

/* Creates a context bound to CUDA device `device`. *ctx receives the handle.
 * Allocates a few kilobytes of constant tables on the device; scratch for
 * the kernels is allocated by the first call that needs it. */
tsallis_status tsallis_create(tsallis_ctx** ctx, int device);

/* Releases the context's scratch memory. Safe with NULL. The caller must
 * make sure no work of this context is still running. */
void tsallis_destroy(tsallis_ctx* ctx);

/* Limit, in nanoseconds, on every device-side wait of this context
 * (default 1e9). A wait that runs out writes TSALLIS_ERR_TIMEOUT. */
tsallis_status tsallis_set_wait_timeout(tsallis_ctx* ctx, uint64_t ns);

/*
 * Launch shape of the persistent kernels (the counterpart of the grid/block
 * tuning in the paper's Table 4): voxels per work tile (a multiple of 8 in
 * 4096..2^22; default 131072) and resident blocks per SM used for the grid
 * (0 = as many as fit). Returns TSALLIS_ERR_INVALID_ARG outside those ranges.
 */
tsallis_status tsallis_set_launch_shape(tsallis_ctx* ctx, int32_t tile_vox, int32_t blocks_per_sm);

/*
 * Kernel used by tsallis_segment for per-slice 1-D work (the paper has one
 * GPU design; these are GB300 designs of the same steps, with equal
 * results):
 *   TSALLIS_SLICE_KERNEL_AUTO (default): the cluster kernel where it applies
 *     (below) for volumes of at most twice as many slices as 8-CTA
 *     clusters fit on the device at once (38 on a 152-SM part), else the
 *     persistent tile kernel;
 *   TSALLIS_SLICE_KERNEL_TILES: the persistent tile kernel;
 *   TSALLIS_SLICE_KERNEL_CLUSTER: the cluster kernel where it applies
 *     (slices of at most 262144 voxels whose voxel count is a multiple of
 *     8), else the tile kernel. Returns TSALLIS_ERR_UNIMPLEMENTED if the
 *     device cannot run 8-CTA clusters.
 *   TSALLIS_SLICE_KERNEL_PREDICT: the predicted first-pass kernel where it
 *     applies (slices whose voxel count is a multiple of 8 and at most
 *     2^24; topk = 0), else the tile kernel.
 *   TSALLIS_SLICE_KERNEL_PIPELINE: the pipelined kernel where it applies
 *     (slices whose voxel count is a multiple of 8; topk = 0), else the tile
 *     kernel.
 * The pipelined kernel cuts the slices into chunks (at most 8 a slice, at
 * least 131072 voxels) taken in slice order; the block that counts a slice's
 * last chunk runs its search at once, and each block binarises the chunks it
 * counted as soon as their slices' thresholds are out, a few microseconds
 * after it read them, so the second read comes from L2. A wait for a
 * threshold that runs out (TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL: one chunk never
 * arrives) makes every slice of the call report TSALLIS_ERR_TIMEOUT.
 * The predicted first-pass kernel reads every voxel once in the usual case:
 * a predicted threshold t^ per slice (the exhaustive search, in FP32, of
 * the histogram of every 16th row of the slice; see tsallis_set_prediction)
 * lets the histogram pass also write the mask (Algorithm 1 at t^) and list
 * the voxels whose level lies within the prediction window of t^; after the
 * slice's exact search gives t, the listed voxels whose side changes are
 * rewritten. A slice is read a second time only when t lies outside the
 * window, the subsample has fewer than two non-empty levels, or a warp's
 * list overflows (a warp keeps up to max(256, 1/16 of the voxels it counts)
 * entries; a grid barrier that runs out of time makes every slice of the
 * call report TSALLIS_ERR_TIMEOUT instead). Slices whose mask needed
 * no second read carry TSALLIS_STATUS_FIRST_PASS_EXACT. The tile kernel
 * reads each slice twice, the second time mostly from L2 when it comes soon
 * enough. The cluster kernel holds each slice in the shared memory of an
 * 8-CTA thread-block cluster between its histogram and its binarisation,
 * so the volume is read from memory once; it is slower than the others
 * (each cluster waits for its slice's search before taking the next).
 */
#define TSALLIS_SLICE_KERNEL_AUTO 0
#define TSALLIS_SLICE_KERNEL_TILES 1
#define TSALLIS_SLICE_KERNEL_CLUSTER 2
#define TSALLIS_SLICE_KERNEL_PREDICT 3
#define TSALLIS_SLICE_KERNEL_PIPELINE 4
tsallis_status tsallis_set_slice_kernel(tsallis_ctx* ctx, int32_t kind);

/*
 * First-pass binarisation with a predicted threshold in the tile kernel
 * (off by default; on = 1). With it on, a histogram tile of a group also writes the
 * group's mask with a predicted threshold t^ (the threshold of the group
 * whose search finished most recently in the same call; groups that start
 * before any search has finished get no prediction). Once the group's
 * search gives t, the mask is exact if no voxel of the group has a level
 * between t^ and t, or (per-slice groups of at most 2^20 voxels) when every
 * voxel that lies between them is among those the first pass listed (levels
 * within 8 of t^), which are then rewritten; the group's status carries
 * TSALLIS_STATUS_FIRST_PASS_EXACT and the group is not read again.
 * Otherwise the group is binarised again with t. Results are identical
 * either way; only the memory traffic differs.
 */
tsallis_status tsallis_set_speculation(tsallis_ctx* ctx, int32_t on);

/*
 * Settings of the predicted first-pass kernel (TSALLIS_SLICE_KERNEL_PREDICT):
 * the prediction histograms every row_stride-th row of a slice (1..4096,
 * default 16; a slice of fewer rows uses its middle row), and the voxels the
 * first pass lists are those whose level lies in (t^ - window, t^ + window]
 * (1..127, default 8). Both only trade memory traffic against work; results
 * are the same for every setting. TSALLIS_ERR_INVALID_ARG outside the ranges.
 */
tsallis_status tsallis_set_prediction(tsallis_ctx* ctx, int32_t row_stride, int32_t window);

/*
 * Step 1: histogram (section I "Thresholding", Fig. 2; 2-D: section II-C,
 * mean image g and h(i, j)).
 *   d_vol   [nz][ny][nx] int16, device.
 *   d_hist  out, int32, device: 1-D: [nh][nbins]; 2-D: [nh][L2][L2] indexed
 *           [grey][mean]. nh = nz (per slice) or 1 (whole volume).
 *           Overwritten (zeroed first).
 * 2-D per-slice mode uses the 3x3 in-slice mean (the paper's form); 2-D
 * whole-volume mode uses the 3x3x3 mean when nz > 1. Both clamp indices at
 * the borders. Counts per histogram must stay below 2^31.
 */
tsallis_status tsallis_histogram(tsallis_ctx* ctx, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                                 const tsallis_params* p, int32_t* d_hist, cudaStream_t stream);

/*
 * Steps 2-3: objective over every threshold and its maximiser (section II-C,
 * class-mass, class-entropy and phi_alpha equations), for nh histograms.
 *   d_hist    [nh][nbins] (1-D) or [nh][L2][L2] (2-D) int32, device.
 *   d_t       out, int32: 1-D: [nh] threshold t; 2-D: [nh][2] pairs (t, s).
 *             t = -1 when no threshold is valid.
 *   d_phi     out, float [nh]: maximum objective value.
 *   d_status  out, int32 [nh]: tsallis_status | TSALLIS_STATUS_* bits.
 *   d_curve   optional out (may be NULL), float: 1-D [nh][nbins-1] phi(t);
 *             2-D [nh][L2-1][L2-1] phi(t, s). NaN where a class is empty.
 * t (then s) is the smallest maximiser. Objective values are FP32 with
 * compensated sums; candidates within the FP32 error band of the maximum are
 * re-ranked in FP64.
 */
tsallis_status tsallis_search(tsallis_ctx* ctx, const int32_t* d_hist, int64_t nh, const tsallis_params* p,
                              int32_t* d_t, float* d_phi, int32_t* d_status, float* d_curve,
                              cudaStream_t stream);

/*
 * Step 4: Algorithm 1 (thresholding kernel) with thresholds from d_t
 * (per slice: [nz]; whole volume: [1]; 2-D: pairs, only t is used, applied
 * to the grey level b >> shift). t = -1 gives an all-zero mask.
 *   d_mask  out, uint8 [nz][ny][nx], device.
 */
tsallis_status tsallis_binarize(tsallis_ctx* ctx, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                                const int32_t* d_t, const tsallis_params* p, uint8_t* d_mask,
                                cudaStream_t stream);

/*
 * Steps 1-4 fused in one persistent kernel (1-D form): per-slice histograms
 * are built, searched by the last tile to arrive, and the slice is binarised
 * by the same launch (its second read can hit L2 when it comes soon enough
 * after the first; on large volumes most of it comes from memory).
 *   d_mask out [nz][ny][nx]; d_t, d_phi, d_status out [nh] as in
 *   tsallis_search (nh = nz per slice, 1 whole volume).
 * The 2-D form is dispatched to its own kernels by the same call.
 */
tsallis_status tsallis_segment(tsallis_ctx* ctx, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                               const tsallis_params* p, uint8_t* d_mask, int32_t* d_t, float* d_phi,
                               int32_t* d_status, cudaStream_t stream);

/*
 * tsallis_segment from and to HOST memory: h_vol (int16 [nz][ny][nx]) is
 * read and h_mask (uint8, same shape), h_t, h_phi, h_status (as for
 * tsallis_segment) are written by the call's copies. In the per-slice 1-D
 * form the volume is pipelined in chunks of about 2^24 voxels (whole slices)
 * through two device buffers on internal streams, so that copying chunk i+1
 * in, segmenting chunk i and copying the mask of chunk i-1 out overlap; the
 * other forms copy the volume in, segment it and copy the results out. The
 * context owns the device buffers (grown on demand). Asynchronous: the work
 * is ordered after what `stream` already holds and `stream` waits for all of
 * it, so the host buffers may be read after synchronising `stream`. The copies
 * overlap only when the host buffers are page-locked (cudaHostAlloc or
 * cudaHostRegister); pageable memory works, more slowly. Errors as for
 * tsallis_segment (no alignment rule for the host buffers).
 */
tsallis_status tsallis_segment_host(tsallis_ctx* ctx, const int16_t* h_vol, int64_t nx, int64_t ny, int64_t nz,
                                    const tsallis_params* p, uint8_t* h_mask, int32_t* h_t, float* h_phi,
                                    int32_t* h_status, cudaStream_t stream);

/* One volume of a batch: device pointers and its shape. */
typedef struct {
    const int16_t* vol;
    uint8_t* mask;
    int64_t nx, ny, nz;
} tsallis_volume;

/*
 * Steps 1-4 for nvol volumes of uneven depth in one persistent launch, one
 * histogram and threshold per volume (whole-volume mode) or per slice
 * (per-slice mode, slices of all volumes numbered consecutively).
 *   h_vols   host array of nvol descriptors (read during the call only);
 *            each volume and mask 16-byte aligned, nz >= 1.
 *   d_t, d_phi, d_status  out, one entry per histogram, in volume order.
 * The volumes' group table is written on the device by a small kernel
 * whose arguments carry the descriptors, so the whole call (two or more
 * launches, no host copies) can be captured in a CUDA graph once a first
 * call has sized the context's scratch. Per histogram at most 2^31 - 1
 * voxels; in all at most 2^20 - 2 histograms. The 2-D form runs volume by
 * volume. Errors as for tsallis_segment.
 */
tsallis_status tsallis_segment_batch(tsallis_ctx* ctx, const tsallis_volume* h_vols, int32_t nvol,
                                     const tsallis_params* p, int32_t* d_t, float* d_phi, int32_t* d_status,
                                     cudaStream_t stream);

/*
 * Learned threshold proposer (an addition: the paper's search is exhaustive).
 * A network reads x_k = log1p(counts of levels 16k..16k+15) / log1p(N),
 * k < 256, of a 4096-level histogram and gives 4096 logits, one per
 * threshold: z1 = W1 x + b1, a1 = GELU(z1), z2 = W2 a1 + b2, a2 = GELU(z2),
 * z3 = W3 a2 + b3, with W1, W2 256 x 256 and W3 4096 x 256. Its parameters
 * are one flat float vector of TSALLIS_PROPOSER_PARAMS values in the order
 * W1, b1, W2, b2, W3, b3 (matrices row-major [out][in]); the GPU multiplies
 * with bfloat16 copies of the matrices and accumulates in FP32. With
 * params.topk = k > 0, tsallis_search, tsallis_segment and
 * tsallis_segment_batch evaluate the objective first at the canonical
 * thresholds of the k highest logits, then exhaustively in every block of
 * 64 levels whose bound (from the class sums at its ends) could still reach
 * that maximum: the result is that of the exhaustive search; the statuses
 * report whether the window held the maximiser (TSALLIS_STATUS_WINDOW_HIT)
 * and how many blocks were searched (bits TSALLIS_STATUS_FALLBACK_SHIFT..+7).
 *
 * tsallis_proposer_set / _get: copy the parameter vector to / from the
 *   context (host memory, n must equal TSALLIS_PROPOSER_PARAMS; synchronous).
 *   Setting also clears the optimiser state.
 * tsallis_proposer_load / _save: the same through a file (8-byte magic
 *   "TSPROP01", int64 count, the floats).
 * tsallis_proposer_features: x [nh][256] (device) from histograms [nh][4096]
 *   (slot 1: from 2-D histograms [nh][256][256]).
 * tsallis_proposer_forward: logits [B][4096] (device) from x [B][256].
 * tsallis_proposer_train_step: forward pass, mean cross-entropy of
 *   softmax(logits) against target distributions y [B][4096] into *d_loss,
 *   backward pass, and (update != 0) one Adam step (beta 0.9, 0.999,
 *   eps 1e-8) with learning rate lr; d_grad (nullable) receives the
 *   gradient [TSALLIS_PROPOSER_PARAMS]. Steps on one context are ordered on
 *   the stream.
 */
#define TSALLIS_PROPOSER_PARAMS 1184256
/*
 * Two proposers live in a context: slot 0 (the 1-D searches, described
 * above) and slot 1 (the 2-D search). tsallis_proposer_select chooses the
 * slot that tsallis_proposer_set, _get, _load, _save, _checkpoint_save,
 * _checkpoint_load, _features,
 * _forward and _train_step act on (0 by default); the searches always use their
 * own slot. Slot 1 has the same network and parameter layout; its features
 * come from a 2-D histogram of 256 x 256 grey x mean levels:
 * x_f = log1p(count of 16 x 16 block f) / log1p(N), f = 16 * (grey block) +
 * (mean block), and its 4096 logits score cells of 4 x 4 threshold pairs,
 * cell 64 * (t / 4) + s / 4. With params.two_d = 1, nbins >> shift = 256 and
 * topk = k > 0, tsallis_search / tsallis_segment / tsallis_segment_batch
 * evaluate the objective at every pair of the k best cells, bound every other
 * cell from the summed-area tables at its corners (the class counts and term
 * sums grow with t and s in quadrant 1 and shrink in quadrant 2) and evaluate
 * the cells whose bound reaches that maximum: the result is the exhaustive
 * search's. Statuses carry TSALLIS_STATUS_WINDOW_HIT and the number of
 * searched non-candidate cells (bits 16..23, saturating at 255). Needs slot 1
 * set; not with TSALLIS_FLAG_BRUTE_FORCE_2D nor a curve output.
 */
tsallis_status tsallis_proposer_select(tsallis_ctx* ctx, int32_t slot);
/*
 * Training checkpoints: tsallis_proposer_checkpoint_save writes the FP32
 * parameters, both Adam moments and the number of Adam steps taken, with a
 * header (magic "TSCKPT01", version 1, the layer sizes) and, after the
 * moments, user_bytes bytes of the caller's own state (for example its data
 * sampler's random state), closed by a CRC-32 of everything before it.
 * tsallis_proposer_checkpoint_load restores parameters, moments and step
 * count (training then continues exactly as if uninterrupted, given the same
 * batches) and copies the caller's state into user (at most user_cap bytes;
 * *user_bytes receives its length). A damaged, truncated or foreign file, or
 * a user state longer than user_cap, gives TSALLIS_ERR_INVALID_ARG and leaves
 * the context unchanged. Both are synchronous.
 */
tsallis_status tsallis_proposer_checkpoint_save(tsallis_ctx* ctx, const char* path, const void* user,
                                                int64_t user_bytes);
tsallis_status tsallis_proposer_checkpoint_load(tsallis_ctx* ctx, const char* path, void* user, int64_t user_cap,
                                                int64_t* user_bytes);
tsallis_status tsallis_proposer_set(tsallis_ctx* ctx, const float* h_params, int64_t n);
tsallis_status tsallis_proposer_get(tsallis_ctx* ctx, float* h_params, int64_t n);
tsallis_status tsallis_proposer_load(tsallis_ctx* ctx, const char* path);
tsallis_status tsallis_proposer_save(tsallis_ctx* ctx, const char* path);
tsallis_status tsallis_proposer_features(tsallis_ctx* ctx, const int32_t* d_hist, int64_t nh, float* d_x,
                                         cudaStream_t stream);
tsallis_status tsallis_proposer_forward(tsallis_ctx* ctx, const float* d_x, int32_t B, float* d_logits,
                                        cudaStream_t stream);
tsallis_status tsallis_proposer_train_step(tsallis_ctx* ctx, const float* d_x, const float* d_y, int32_t B,
                                           float lr, int32_t update, float* d_loss, float* d_grad,
                                           cudaStream_t stream);

/*
 * Autotuner for tsallis_segment_batch (the counterpart of the paper's
 * grid/block-size experiment, Table 4): runs the batch with every work-tile
 * size in {16384, 32768, 65536, 131072, 262144} voxels and every resident
 * block count per SM the kernel allows, timing the best of three passes
 * each, and keeps the fastest as the context's launch shape (see
 * tsallis_set_launch_shape). Synchronous; the outputs hold the last pass's
 * results. The chosen shape and time go to *tile_vox, *blocks_per_sm and
 * *best_ms (each may be NULL). 1-D form only.
 */
tsallis_status tsallis_autotune_batch(tsallis_ctx* ctx, const tsallis_volume* h_vols, int32_t nvol,
                                      const tsallis_params* p, int32_t* d_t, float* d_phi, int32_t* d_status,
                                      cudaStream_t stream, int32_t* tile_vox, int32_t* blocks_per_sm,
                                      float* best_ms);

/*
 * tsallis_segment_static: tsallis_segment for callers that cannot allocate
 * device memory. The paper has no counterpart; it exists for code whose
 * device memory is all owned by someone else (a framework's memory pool, a
 * pipeline that forbids allocation after start-up) or that must avoid the
 * implicit synchronisation of cudaMalloc/cudaFree. tsallis_segment needs a
 * context, and creating one allocates; this entry point takes no context and
 * calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * Its scratch is one fixed __device__ array inside the library (about 8.2 MB,
 * held on every GPU that loads the library until the process exits). Limits
 * that follow from it: at most 512 histograms per call (slices in per-slice
 * mode) and at most 16384 work tiles of 65536 voxels (about 1.07e9 voxels in
 * whole-volume mode); 1-D form only (two_d must be 0) and exhaustive only
 * (topk must be 0: there is no proposer without a context). Calls beyond those
 * limits return TSALLIS_ERR_INVALID_ARG before anything is enqueued. Other
 * arguments, outputs and statuses are as for tsallis_segment; the device is
 * the current CUDA device.
 *
 * The first call on a device does a synchronous set-up (looks up the array's
 * device address, clears it, writes constant tables, sets kernel
 * attributes); make that first call before any stream capture. Later calls
 * only enqueue one kernel. Every call uses the same array, which keeps the
 * state the previous call left (the kernel leaves it ready for the next
 * call), so calls that overlap in time on the GPU (on different streams, or
 * from different threads) race and must not be issued.
 */
tsallis_status tsallis_segment_static(const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                                      const tsallis_params* p, uint8_t* d_mask, int32_t* d_t, float* d_phi,
                                      int32_t* d_status, cudaStream_t stream);

/*
 * Pre-processing and chest-mask morphology: the steps of the paper that come
 * before the threshold (section II-B "Pre-processing", section II-C
 * "Morphology"), in one pass over the volume.
 *
 *   level   each CT number v becomes an 8-bit grey level: 0 when
 *           v <= background (the detector background, -2000 HU), otherwise
 *           v is clamped to [hu_min, hu_max] and mapped linearly onto 0..255,
 *           rounded to nearest with halves up:
 *           g = floor((clamp(v) - hu_min) * 255 / (hu_max - hu_min) + 1/2).
 *   morph   flat grey morphology of each z slice as a 2-D image with the
 *           digital disk of radius `radius` (offsets dx^2 + dy^2 <= r^2;
 *           offsets that leave the slice are not part of the window):
 *           erosion = minimum over the disk, dilation = maximum, opening =
 *           dilation of the erosion, closing = erosion of the dilation.
 *   op      the output: TSALLIS_MORPH_CHEST_MASK = g - opening(g), the
 *           chest-mask subtraction (the paper opens with a disk of size 10
 *           and subtracts; an opening never exceeds the image, so the
 *           difference is taken in the order that keeps it non-negative);
 *           TSALLIS_MORPH_BLACK_TOPHAT = closing(g) - g; or the erosion,
 *           dilation, opening, closing, or g itself (TSALLIS_MORPH_NONE).
 *
 * d_vol   device int16 [nz][ny][nx] (x fastest), 4-byte aligned
 *         (TSALLIS_ERR_ALIGNMENT otherwise).
 * d_out   device int16 [nz][ny][nx] receiving the result as levels 0..255
 *         (nullable); the same layout the other calls read, so that
 *         tsallis_search / tsallis_binarize / tsallis_segment with lo = 0,
 *         nbins = 256 threshold it. Must not overlap d_vol.
 * d_hist  device int32, 256 counts of the result's levels per slice
 *         ([nz][256], per_slice = 1) or for the volume ([256]); nullable;
 *         zeroed and filled by the call.
 * Limits: radius 0..15; hu_min < hu_max <= hu_min + 65535; nx, ny >= 1,
 * nz >= 0, at most 2^31 - 1 tiles of 128 x 64 pixels; d_out and d_hist not both
 * null (unless nz = 0, which writes nothing but the zeroed volume histogram).
 * Violations return TSALLIS_ERR_INVALID_ARG before anything is enqueued.
 * Asynchronous on `stream`; no scratch memory.
 */
typedef enum {
    TSALLIS_MORPH_NONE = 0,
    TSALLIS_MORPH_ERODE = 1,
    TSALLIS_MORPH_DILATE = 2,
    TSALLIS_MORPH_OPEN = 3,
    TSALLIS_MORPH_CLOSE = 4,
    TSALLIS_MORPH_CHEST_MASK = 5,
    TSALLIS_MORPH_BLACK_TOPHAT = 6
} tsallis_morph_op;

typedef struct {
    int32_t background; /* -2000 */
    int32_t hu_min;     /* -2000 */
    int32_t hu_max;     /* 2500 */
    int32_t radius;     /* 10 */
    int32_t op;         /* TSALLIS_MORPH_CHEST_MASK */
    int32_t per_slice;  /* 1 */
} tsallis_preprocess_params;

tsallis_status tsallis_preprocess_params_default(tsallis_preprocess_params* pp);
tsallis_status tsallis_preprocess(tsallis_ctx* ctx, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                                  const tsallis_preprocess_params* pp, int16_t* d_out, int32_t* d_hist,
                                  cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* TSALLIS_H */
