// Internal interface between the C-ABI layer (api.cu) and the kernel
// translation units. Host-side only declarations plus the argument structs
// that are passed by value to the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tsl {

constexpr int kMaxLevels = 4096;  // largest 1-D histogram

// Scratch header that lives at the start of a context's device scratch.
// It starts zeroed and every launch leaves it as it found it (the last block
// to finish resets the ticket and done counters and bumps the epoch), so no
// memset is needed between launches and CUDA-graph replays are safe.
struct ScratchHeader {
    unsigned int h_next;  // next histogram work item
    unsigned int b_next;  // next binarise queue position to claim
    unsigned int b_tail;  // binarise queue positions reserved by published groups
    unsigned int done;    // blocks that have finished
    int epoch;            // launches so far; flags are compared to epoch + 1
    int err;              // a device wait ran out or an arrival was skipped
    unsigned long long latest;   // (epoch + 1) << 32 | (t + 1): the threshold found
                                 // most recently in this launch (a prediction)
    unsigned int gcount;     // predicted first pass: grid barrier arrivals
    int pad0;
    unsigned long long serial;   // pipelined per-slice kernel: launches so far (readiness tags)
    unsigned long long pipe_latest;   // pipelined kernel: (serial + 1) << 13 | (t + 1), the latest threshold
    int pad[2];
};

enum Phase : int { kPhaseHist = 1, kPhaseSearch = 2, kPhaseBin = 4 };

// A group (one histogram) of a batch: its voxels, its mask, and where its
// tiles start in the batch's sequence of histogram work items.
struct GroupDesc {
    const int16_t* vol;
    uint8_t* mask;
    long long nvox;
    int ntiles;
    int tile_off;
};

struct SegArgs {
    const int16_t* vol;     // uniform groups: group g starts at vol + g * group_vox
    uint8_t* mask;
    long long group_vox;
    int ngroups;
    int ntiles;             // tiles per group (uniform groups)
    int tile_vox;           // voxels per tile, multiple of 8
    unsigned int ntotal;    // histogram (or binarise) work items in total
    const GroupDesc* groups;   // non-null: batch of uneven groups
    int lo, L;
    float q;
    int polarity;
    int bin_shift;          // threshold applies to level >> bin_shift (2-D grey levels)
    int phases;
    unsigned int flags;
    unsigned long long timeout_ns;
    ScratchHeader* hdr;
    int* arrive;            // [ngroups] histogram tiles added so far
    int* done_flag;         // [ngroups] epoch + 1 once the threshold is published
    int* bdone;             // [ngroups] binarise tiles finished
    unsigned long long* that;  // [ngroups] (epoch + 1) << 32 | (t^ + 1): the predicted
                               // threshold the group's first pass binarised with
    int spec;               // 1: histogram tiles also binarise with a predicted threshold
    // exceptions of the first pass: voxels whose level lies within exc_w of the
    // predicted threshold, (position in group << 16) | (level - (t^ - exc_w + 1));
    // group g owns the pool entries from (first tile * tile_vox) / 32 on, as
    // many as 1/32 of the voxels its tiles span; exc_w = 0: none are kept
    unsigned long long* exc;
    int* exc_n;             // [ngroups] entries appended (more than the region: overflowed)
    int exc_w;
    const int* hint;        // optional [ngroups]: predicted thresholds (else the latest found)
    unsigned long long* bq; // [ntotal] binarise queue (launch tag | group | tile)
    int* ghist;             // [ngroups][L]: histogram target (scratch or caller's)
    const int* t_in;        // binarise-only: caller's thresholds
    int t_stride;           // entries between consecutive groups' thresholds in t_in
    int* t_out;
    float* phi_out;
    int* status;
    float* curve;           // optional [ngroups][L-1]
    const void* df_tables;  // double-float log2/exp2 tables (device)
    const float2* ptab;     // optional: terms 2^64 (n / ptab_n)^q (q = 1: n log2 n) for n = 0..ptab_n;
    long long ptab_n;       // groups of exactly ptab_n voxels are searched with it
    unsigned* check;        // checked build: first failing index check (checked.cuh)
};

// A volume of a batch as the descriptor-expansion kernel receives it: its
// groups (one per slice, or the whole volume) are consecutive.
struct BatchVolDesc {
    const int16_t* vol;
    uint8_t* mask;
    long long gvox;         // voxels per group
    int ngroups;            // groups of this volume
    int ntiles;             // tiles per group
    int group_off;          // first group of this volume in the batch
    int tile_off;           // first histogram work item of this volume
};
constexpr int kExpandVols = 48;     // volumes per expansion launch (kernel parameter space)
struct ExpandArgs {
    BatchVolDesc v[kExpandVols];
    int nvol;
    int ngroups;            // groups of these volumes
    GroupDesc* out;         // the batch's group table (written from v[0].group_off on)
};
cudaError_t launch_expand_groups(const ExpandArgs& a, cudaStream_t s);

// Kernel launchers (seg1d.cu).
cudaError_t launch_segment1d(const SegArgs& a, int grid, int copies, cudaStream_t s);
cudaError_t launch_search1d(const int32_t* hist, long long nh, int L, float q, int32_t* t, float* phi,
                            int32_t* status, float* curve, const void* tables, cudaStream_t s);
cudaError_t launch_probe_dfmath(const unsigned* h, long long n, unsigned N, float q, double* pw, double* lg,
                                const void* tables, cudaStream_t s);
size_t df_tables_bytes();
// log2_table: device array of (log2_table_max + 1) float2 entries, filled by
// build_log2_table once the tables themselves are on the device.
void df_tables_fill(void* host, const void* log2_table, int log2_table_max);
cudaError_t build_log2_table(void* lt, int n, const void* tables, cudaStream_t s);
constexpr int kLog2TableMax = 1 << 18;
int segment1d_threads();
int segment1d_smem_bytes(int L, int copies);
cudaError_t segment1d_occupancy(int copies, int L, int* blocks_per_sm);
cudaError_t segment1d_prepare();
// Term table of the table search for groups of n_max voxels, on stream s.
cudaError_t build_pow_table(float2* tab, long long n_max, float q, const void* tables, cudaStream_t s);
constexpr long long kPowTableMax = 1ll << 22;   // largest group size given a term table
constexpr int kExcWindow = 8;      // levels on each side of the predicted threshold

// Per-slice 1-D form with the slice held in a cluster's shared memory
// (seg_cluster.cu): a cluster of kClusterCtas CTAs owns one slice, each CTA
// at most kClusterPartVox voxels of it.
constexpr int kClusterCtas = 8;
constexpr int kClusterPartVox = 32768;
struct ClusterArgs {
    const int16_t* vol;     // [nz][slice_vox], 16-byte aligned, slice_vox % 8 == 0
    uint8_t* mask;
    long long slice_vox;    // N, voxels per slice (<= kClusterCtas * kClusterPartVox)
    long long part_vox;     // voxels per CTA part: ceil(N / kClusterCtas) rounded up to 8
    int nz;
    int lo, L;
    float q;
    int polarity;
    unsigned int flags;
    unsigned long long timeout_ns;
    ScratchHeader* hdr;     // h_next: next slice; done: finished CTAs (both reset by the kernel)
    int* t_out;
    float* phi_out;
    int* status;
    const void* df_tables;
};
cudaError_t slice_cluster_prepare();
cudaError_t slice_cluster_occupancy(int* max_clusters);
cudaError_t launch_slice_cluster(const ClusterArgs& a, int nclusters, cudaStream_t s);

// Per-slice 1-D form that reads each voxel once (seg_spec.cu): a predicted
// threshold per slice from a row subsample, Algorithm 1 in the histogram
// pass, the voxels near the prediction listed, and corrected after the
// exact search.
struct SpecArgs {
    const int16_t* vol;     // [nz][slice_vox], 16-byte aligned, slice_vox % 8 == 0
    uint8_t* mask;
    long long slice_vox;    // S = nx * ny <= kSpecMaxSlice
    long long nvox;         // nz * S
    int nx, ny, nz;
    int nseg;               // slices a block's range can meet (list bookkeeping per block)
    int wcap;               // list entries a warp can keep (its region of exc)
    int piece_vox;          // voxels per piece of a second pass (a multiple of 8)
    int npiece;             // pieces per slice (< 4096)
    int sub_stride;         // prediction: every sub_stride-th row
    int win;                // list window: levels (t^ - win, t^ + win], 1 <= win <= kSpecMaxWin
    int lo, L;
    float q;
    int polarity;
    unsigned int flags;     // TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL, kSpecDebugNoPrediction
    unsigned long long timeout_ns;
    ScratchHeader* hdr;     // gcount, b_next, b_tail, done, err, epoch (reset by the last block)
    int* ghist;             // [nz][kMaxLevels] slice histograms, left zeroed
    unsigned long long* pred;  // [nz] kPredReady | (t^ + 1), left zeroed
    int* sflag;             // [nz] bit 0: the slice needs a second pass, left zeroed
    int* toff;              // [grid][nseg][16] where each warp's list of a part of a slice starts
    int* tcnt;              // [grid][nseg][16] its length (-1: incomplete)
    unsigned* exc;          // [grid][16][wcap]: (position in slice << 8) | (level - (t^ - win + 1))
    unsigned* rbq;          // [nz * npiece] second-pass queue: z << 12 | piece
    int* t_out;
    float* phi_out;
    int* status;
    const void* df_tables;
    const float2* ptab;     // optional term table (2^64 (n / ptab_n)^q) for slices of ptab_n voxels
    long long ptab_n;
    unsigned* check;
};
constexpr long long kSpecMaxSlice = 1ll << 24;   // positions fit 24 bits of a list entry
constexpr int kSpecMaxWin = 127;                 // levels fit 8 bits
constexpr int kSpecWarpList = 256;               // list entries one warp holds for a tile
constexpr int kSpecWarps = 16;                   // streaming warps of a block
constexpr unsigned kSpecDebugNoPrediction = 1u << 16;   // test hook: prediction jobs publish nothing
int slice_spec_smem_bytes();
cudaError_t slice_spec_prepare();
cudaError_t slice_spec_occupancy(int* blocks_per_sm);
cudaError_t launch_slice_spec(const SpecArgs& a, int grid, cudaStream_t s);

// Per-slice 1-D form in one pipelined pass (seg_pipe.cu): chunks counted in
// slice order, each slice searched by the block that counts its last chunk,
// and each chunk binarised by the block that counted it (from L2).
struct PipeArgs {
    const int16_t* vol;     // [nz][slice_vox], 16-byte aligned, slice_vox % 8 == 0
    uint8_t* mask;
    long long slice_vox;    // S
    long long chunk_vox;    // voxels per chunk (a multiple of 8; the last chunk of a slice may be shorter)
    int chunks_per_slice;   // <= 8
    int nz;
    int lo, L;
    float q;
    int polarity;
    unsigned int flags;     // TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL
    unsigned long long timeout_ns;
    ScratchHeader* hdr;     // h_next, done, err, serial (restored by the last block)
    int* ghist;             // [nz][kMaxLevels] slice histograms, left zeroed
    int* parts;             // [nz] chunks of the slice counted, left zeroed
    unsigned long long* ready;   // [nz] (serial + 1) << 13 | (t + 1) once the slice is searched
    int win;                // list window: levels (t^ - win, t^ + win], 1 <= win <= kSpecMaxWin
    int wcap;               // list entries a warp keeps for one chunk
    unsigned* exc;          // [grid][kPipeRing][16][wcap]: index in the chunk of a listed 16-byte group
    int* t_out;
    float* phi_out;
    int* status;
    const void* df_tables;
    const float2* ptab;     // optional term table (2^64 (n / ptab_n)^q) for slices of ptab_n voxels
    long long ptab_n;
    unsigned* check;
};
constexpr int kPipeRing = 12;                           // chunks a block counts before finishing them
constexpr long long kPipeMaxSlice = 1ll << 27;          // 8 chunks of at most 2^24 voxels (list positions)
constexpr unsigned kPipeDebugNoPrediction = 1u << 16;   // test hook: chunks are counted without a prediction
int slice_pipe_smem_bytes();
cudaError_t slice_pipe_prepare();
cudaError_t slice_pipe_occupancy(int* blocks_per_sm);
int pipe_chunks_per_slice(long long slice_vox, long long* chunk_vox);
cudaError_t launch_slice_pipe(const PipeArgs& a, int grid, cudaStream_t s);

// Learned threshold proposer (mlp.cu): 256 features -> 256 -> 256 -> 4096.
constexpr int kMlpIn = 256, kMlpHid = 256, kMlpOut = 4096, kMlpGroup = 16;
constexpr long long kOffW1 = 0, kOffB1 = kOffW1 + (long long)kMlpHid * kMlpIn;
constexpr long long kOffW2 = kOffB1 + kMlpHid, kOffB2 = kOffW2 + (long long)kMlpHid * kMlpHid;
constexpr long long kOffW3 = kOffB2 + kMlpHid, kOffB3 = kOffW3 + (long long)kMlpOut * kMlpHid;
constexpr long long kMlpParams = kOffB3 + kMlpOut;   // 1,184,256
struct MlpBuffers {
    float* p32;      // [kMlpParams] optimiser copy (biases are read from here)
    void* p16;       // [kMlpParams] bfloat16 copy (matrices are read from here)
    float* grad;     // [kMlpParams]
    float* m;        // Adam moments
    float* v;
    // activations for up to `cap` rows
    float *z1, *a1, *z2, *a2;   // [cap][256]
    float *z3, *d3;             // [cap][4096]
    float *da, *dz;             // [cap][256]
    int cap;
};
cudaError_t mlp_features(const int32_t* hist, long long nh, float* x, cudaStream_t s);
cudaError_t mlp_features2d(const int32_t* hist, long long nh, float* x, cudaStream_t s);   // [nh][256][256]
cudaError_t mlp_to_bf16(const float* p, void* p16, long long n, cudaStream_t s);
cudaError_t mlp_forward(const MlpBuffers& b, const float* x, int B, cudaStream_t s);   // logits in b.z3
cudaError_t mlp_backward(const MlpBuffers& b, const float* x, const float* y, int B, float* loss, cudaStream_t s);
cudaError_t mlp_adam(const MlpBuffers& b, float lr, int step, cudaStream_t s);
cudaError_t mlp_topk(const float* z, int B, int k, int32_t* out, cudaStream_t s);
// Inference of up to kMlpInferRows rows in one launch: (hist given) the
// features into xw, the three layers (logits in b.z3), then (k > 0) the top
// k of each row into cand. sync: three words, zero between launches.
constexpr int kMlpInferRows = 64;
cudaError_t mlp_prepare();
cudaError_t mlp_infer(const MlpBuffers& b, const int32_t* hist, const float* x, float* xw, int B, int k,
                      int32_t* cand, unsigned* sync, unsigned long long timeout_ns, cudaStream_t s);
// Window search (seg1d.cu): nh histograms, k candidate levels each.
cudaError_t launch_search1d_window(const int32_t* hist, long long nh, int L, float q, const int32_t* cand, int k,
                                   int32_t* t, float* phi, int32_t* status, const void* tables, cudaStream_t s);

// 2-D form (seg2d.cu).
struct Hist2dLaunch {
    const int16_t* vol;
    int nx, ny, nz;
    int lo, L, shift;
    int per_slice;          // 1: one histogram per slice, 3x3 window; 0: one histogram, 3x3x3 window (nz > 1)
    int* hist;              // [nh][L2][L2], zeroed by the caller
    int sm_count, blocks_per_sm;
};
// 2-D window search: cells of 4 x 4 pairs, 64 x 64 of them for 256 levels.
constexpr int kCell2d = 4;
constexpr int kCells2d = 4096;
struct Search2dLaunch {
    const int* hist;        // [K][L2][L2]
    long long K;
    int L2;
    float q;
    const void* tables;
    void* scratch;          // search2d_scratch_bytes(L2, K)
    float* curve;           // optional [K][L2-1][L2-1]
    int* t;                 // [K][2]
    int* t_bin;             // optional [K]
    float* phi;
    int* status;
    // window search (optional): per histogram, the proposer's candidate
    // cells [K][topk], a flag per cell [K][kCells2d] (0 skip, 1 bound
    // reaches the window, 2 candidate) and the number of flag-1 cells [K]
    const int* cand;
    int topk;
    unsigned char* cellflag;
    int* winfo;
    unsigned* check;        // checked build: first failing index check (checked.cuh)
};
cudaError_t seg2d_prepare();
cudaError_t hist2d_occupancy(int* blocks_per_sm);
cudaError_t launch_hist2d(const Hist2dLaunch& p, cudaStream_t s);
size_t search2d_scratch_bytes(int L2, long long K);
cudaError_t launch_search2d(const Search2dLaunch& p, cudaStream_t s);
// the same in phases: tables (row and column scans), then, for a window
// search, the cell flags, then evaluation and the final maximum
cudaError_t launch_search2d_tables(const Search2dLaunch& p, cudaStream_t s);
cudaError_t launch_search2d_window(const Search2dLaunch& p, cudaStream_t s);
cudaError_t launch_search2d_finish(const Search2dLaunch& p, cudaStream_t s);
// One thread per pair, quadrants summed directly (seg2d_brute.cu).
size_t search2d_brute_scratch_bytes(int L2, long long K);
cudaError_t launch_search2d_brute(const Search2dLaunch& p, cudaStream_t s);

// Pre-processing and morphology (preproc.cu); arguments in preproc_args.h.
struct PreArgs;
int preproc_tile_w();
int preproc_tile_h();
cudaError_t preproc_prepare();
cudaError_t launch_preprocess(const PreArgs& a, cudaStream_t s);

}  // namespace tsl
