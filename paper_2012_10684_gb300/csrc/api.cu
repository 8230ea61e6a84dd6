// C ABI of the thresholding path (declared in include/tsallis.h): argument
// checks, the context's scratch memory, and dispatch to the kernels.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/tsallis.h"
#include "../../include/tsallis_testing.h"
#include "checked.cuh"
#include "kernels.h"
#include "preproc_args.h"

#include <nvtx3/nvToolsExt.h>

using namespace tsl;

namespace {
// One NVTX range per call of an entry point that enqueues GPU work, named
// after the entry point, so a trace shows where each call's kernels came
// from. Without a tool attached the push and pop are no-ops.
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};
}  // namespace
#define TSL_TRACE() const TraceRange tsl_trace_range_(__func__)

static_assert(kMlpParams == TSALLIS_PROPOSER_PARAMS, "parameter count of the C ABI");

struct ProposerSlot {
    MlpBuffers mlp{};
    void* params = nullptr;
    void* act = nullptr;
    int step = 0;           // Adam steps taken
    bool ready = false;     // parameters were set
};

struct tsallis_ctx {
    int device = 0;
    int sm_count = 0;
    long long l2_bytes = 0;
    void* scratch = nullptr;      // ScratchHeader, then per-group arrays
    size_t scratch_bytes = 0;
    long long cap_groups = 0;
    long long cap_tiles = 0;
    long long cap_exc = 0;
    unsigned long long timeout_ns = 1000000000ull;
    // launch shape of the 1-D persistent kernel
    int copies = 1;
    int tile_vox = 131072;
    int blocks_per_sm = 0;        // resident blocks per SM used for the grid
    int max_blocks_per_sm = 0;    // what the occupancy calculator allows
    // batch work list (device copy) and its host image
    void* batch_buf = nullptr;
    size_t batch_bytes = 0;
    void* df_tables = nullptr;    // double-float log2/exp2 tables (device)
    // 2-D form: histograms, search tables and thresholds (grown on demand)
    void* s2_buf = nullptr;
    size_t s2_bytes = 0;
    int hist2d_blocks_per_sm = 0;
    void* log2_table = nullptr;   // log2 of counts up to 2^18 as float pairs (device)
    // per-slice 1-D kernel: TSALLIS_SLICE_KERNEL_*; clusters that fit at once
    int slice_kernel = TSALLIS_SLICE_KERNEL_AUTO;
    int speculate = 0;            // tile kernel: binarise in the first pass with a predicted threshold
    int cluster_max = 0;
    // per-slice kernel that reads each voxel once: prediction settings, its
    // resident blocks per SM, a test switch, and its arrays (spec_layout)
    int spec_stride = 16;
    int spec_win = 8;
    int spec_blocks_per_sm = 0;
    unsigned spec_test_flags = 0;
    void* spec_buf = nullptr;       // predicted thresholds, flags, queue, tile counts, lists
    size_t spec_bytes = 0;
    long long spec_nz = 0, spec_ntot = 0, spec_nl = 0, spec_nexc = 0;   // the layout it holds
    // pipelined per-slice kernel: resident blocks per SM; per-slice counters
    // and readiness words for up to pipe_nz slices (zeroed when allocated)
    int pipe_blocks_per_sm = 0;
    void* pipe_buf = nullptr;
    long long pipe_nz = 0, pipe_nexc = 0;
    // term table of the per-slice search (built for one slice size and q)
    float2* ptab = nullptr;
    long long ptab_cap = 0;     // entries allocated
    long long ptab_n = -1;      // slice size it holds
    float ptab_q = 0.f;
    // learned proposer: parameters (FP32, bfloat16, gradient, Adam moments),
    // activations for up to mlp.cap rows, features and candidates
    // slot 0 serves the 1-D searches, slot 1 the 2-D search; the
    // tsallis_proposer_* calls act on the slot chosen by
    // tsallis_proposer_select
    ProposerSlot prop[2];
    int prop_sel = 0;
    float* prop_x = nullptr;        // [prop_cap][256]
    int32_t* prop_cand = nullptr;   // [prop_cap][256]
    unsigned* prop_sync = nullptr;  // barrier words of the fused inference kernel (in prop_x's buffer)
    int prop_cap = 0;
    // first-pass prediction of batches: sub-volume group table, histograms,
    // predicted thresholds and the search's other outputs
    void* pred_buf = nullptr;
    int pred_cap = 0;
    unsigned* check = nullptr;    // checked build: first failing index check (checked.cuh)
    // host-buffer entry point: device chunk buffers and outputs, internal
    // streams (copy in, compute, copy out) and the events that order them
    void* hp_buf = nullptr;
    size_t hp_bytes = 0;
    cudaStream_t hp_stream[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t hp_ev[8] = {};
    bool hp_ready = false;
};

namespace {

inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

class DeviceGuard {
  public:
    explicit DeviceGuard(int dev) {
        ok_ = cudaGetDevice(&prev_) == cudaSuccess;
        if (ok_ && prev_ != dev) ok_ = cudaSetDevice(dev) == cudaSuccess;
        else if (ok_) prev_ = -1;
    }
    ~DeviceGuard() {
        if (prev_ >= 0) cudaSetDevice(prev_);
    }
    bool ok() const { return ok_; }

  private:
    int prev_ = -1;
    bool ok_ = false;
};

tsallis_status check_params(const tsallis_params* p) {
    if (!p) return TSALLIS_ERR_INVALID_ARG;
    if (!(p->q > 0.0f) || !(p->q <= 4.0f)) return TSALLIS_ERR_INVALID_ARG;
    if (p->nbins < 2 || p->nbins > kMaxLevels) return TSALLIS_ERR_INVALID_ARG;
    if (p->lo < -32768 || p->lo > 32767) return TSALLIS_ERR_INVALID_ARG;
    if (p->mode != TSALLIS_PER_SLICE && p->mode != TSALLIS_WHOLE_VOLUME) return TSALLIS_ERR_INVALID_ARG;
    if (p->polarity != TSALLIS_MASK_LOW && p->polarity != TSALLIS_MASK_HIGH) return TSALLIS_ERR_INVALID_ARG;
    if (p->two_d != 0 && p->two_d != 1) return TSALLIS_ERR_INVALID_ARG;
    if (p->two_d) {
        if (p->shift < 0 || p->shift > 15) return TSALLIS_ERR_INVALID_ARG;
        int L2 = p->nbins >> p->shift;
        if (L2 < 2 || L2 > 256) return TSALLIS_ERR_INVALID_ARG;
        if (p->nbins & ((1 << p->shift) - 1)) return TSALLIS_ERR_INVALID_ARG;   // grey levels must fill [0, L2)
    }
    if (p->topk < 0) return TSALLIS_ERR_INVALID_ARG;
    if (p->flags & ~(TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL | TSALLIS_FLAG_PREDICT_PROPOSER | TSALLIS_FLAG_PREDICT_SUBSAMPLE |
                     TSALLIS_FLAG_BRUTE_FORCE_2D))
        return TSALLIS_ERR_INVALID_ARG;
    if ((p->flags & TSALLIS_FLAG_BRUTE_FORCE_2D) && !p->two_d) return TSALLIS_ERR_INVALID_ARG;
    return TSALLIS_OK;
}

tsallis_status check_shape(int64_t nx, int64_t ny, int64_t nz) {
    if (nx < 1 || ny < 1 || nz < 0) return TSALLIS_ERR_INVALID_ARG;
    if (nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20)) return TSALLIS_ERR_INVALID_ARG;
    const long long slice = (long long)nx * ny;
    if (slice > (1ll << 31) - 1) return TSALLIS_ERR_INVALID_ARG;
    if (nz > 0 && slice > (1ll << 40) / nz) return TSALLIS_ERR_INVALID_ARG;
    return TSALLIS_OK;
}

// Grows the context's scratch so it holds at least ngroups groups, ntiles
// work tiles and nexc first-pass exception entries. The layout depends only
// on the capacities (arrive, done_flag, bdone [capg]; that [capg]; ghist
// [capg][kMaxLevels]; bq [capt]; exc_n [capg]; exc [capx]), so state left
// by one launch lines up with the next. New memory is zeroed; the kernels
// keep it consistent between launches.
size_t scratch_layout(long long capg, long long capt, long long capx, size_t* ghist_off, size_t* bq_off,
                      size_t* exc_off) {
    size_t off = sizeof(ScratchHeader) + (size_t)capg * (3 * sizeof(int) + sizeof(unsigned long long));
    off = (off + 255) & ~size_t(255);
    if (ghist_off) *ghist_off = off;
    off += (size_t)capg * kMaxLevels * sizeof(int);
    off = (off + 255) & ~size_t(255);
    if (bq_off) *bq_off = off;
    off += (size_t)capt * sizeof(unsigned long long);
    off = (off + 255) & ~size_t(255);
    if (exc_off) *exc_off = off;   // exc_n [capg], then the pool
    off += (size_t)capg * sizeof(int);
    off = (off + 255) & ~size_t(255);
    return off + (size_t)capx * sizeof(unsigned long long);
}

tsallis_status ensure_scratch(tsallis_ctx* c, long long ngroups, long long ntiles, long long nexc = 0) {
    if (c->scratch && ngroups <= c->cap_groups && ntiles <= c->cap_tiles && nexc <= c->cap_exc) return TSALLIS_OK;
    long long capg = c->cap_groups > 0 ? c->cap_groups : 16;
    long long capt = c->cap_tiles > 0 ? c->cap_tiles : 4096;
    long long capx = c->cap_exc;
    while (capg < ngroups) capg *= 2;
    while (capt < ntiles) capt *= 2;
    if (capx < nexc) capx = nexc;
    if (c->scratch) {
        if (cudaDeviceSynchronize() != cudaSuccess) return TSALLIS_ERR_CUDA;
        cudaFree(c->scratch);
        c->scratch = nullptr;
        c->scratch_bytes = 0;
        c->cap_groups = 0;
        c->cap_tiles = 0;
        c->cap_exc = 0;
    }
    const size_t bytes = scratch_layout(capg, capt, capx, nullptr, nullptr, nullptr);
    if (cudaMalloc(&c->scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        return TSALLIS_ERR_OOM;
    }
    if (cudaMemset(c->scratch, 0, bytes) != cudaSuccess) return TSALLIS_ERR_CUDA;
    c->scratch_bytes = bytes;
    c->cap_groups = capg;
    c->cap_tiles = capt;
    c->cap_exc = capx;
    return TSALLIS_OK;
}

// Exception entries a first pass needs: 1/32 of the voxels its tiles span.
inline long long exc_entries(long long ntiles, int tile_vox) { return (ntiles * (long long)tile_vox) >> 5; }

// The term table for groups of n voxels at q: reused while n and q stay
// the same, else rebuilt on the stream (ordered before the kernel that reads
// it). Returns nullptr when n is too large for a table or memory is short
// (the search then computes its terms).
const float2* pow_table(tsallis_ctx* c, long long n, float q, cudaStream_t stream) {
    if (n < 1 || n > kPowTableMax) return nullptr;
    if (c->ptab && c->ptab_n == n && c->ptab_q == q) return c->ptab;
    if (!c->ptab || c->ptab_cap < n + 1) {
        long long cap = c->ptab_cap > 0 ? c->ptab_cap : 65536;
        while (cap < n + 1) cap *= 2;
        if (c->ptab) {
            if (cudaDeviceSynchronize() != cudaSuccess) return nullptr;
            cudaFree(c->ptab);
            c->ptab = nullptr;
            c->ptab_cap = 0;
        }
        if (cudaMalloc(&c->ptab, (size_t)cap * sizeof(float2)) != cudaSuccess) {
            cudaGetLastError();
            c->ptab_n = -1;
            return nullptr;
        }
        c->ptab_cap = cap;
    }
    if (build_pow_table(c->ptab, n, q, c->df_tables, stream) != cudaSuccess) {
        cudaGetLastError();
        c->ptab_n = -1;
        return nullptr;
    }
    c->ptab_n = n;
    c->ptab_q = q;
    return c->ptab;
}

// Parameter block of the proposer: FP32 copy, gradient, two Adam moments
// (kMlpParams floats each), then the bfloat16 copy.
tsallis_status ensure_mlp_params(tsallis_ctx* c, int slot) {
    ProposerSlot& S = c->prop[slot];
    if (S.params) return TSALLIS_OK;
    const size_t f = (size_t)kMlpParams * sizeof(float);
    const size_t bytes = 4 * f + (size_t)kMlpParams * 2;
    if (cudaMalloc(&S.params, bytes) != cudaSuccess) {
        cudaGetLastError();
        S.params = nullptr;
        return TSALLIS_ERR_OOM;
    }
    char* b = static_cast<char*>(S.params);
    S.mlp.p32 = reinterpret_cast<float*>(b);
    S.mlp.grad = reinterpret_cast<float*>(b + f);
    S.mlp.m = reinterpret_cast<float*>(b + 2 * f);
    S.mlp.v = reinterpret_cast<float*>(b + 3 * f);
    S.mlp.p16 = b + 4 * f;
    if (cudaMemset(S.params, 0, bytes) != cudaSuccess) return TSALLIS_ERR_CUDA;
    return TSALLIS_OK;
}

// Activations for `rows` rows of the proposer (grown, never shrunk; the
// device is synchronised before a smaller buffer is replaced).
tsallis_status ensure_mlp_act(tsallis_ctx* c, int slot, int rows) {
    ProposerSlot& S = c->prop[slot];
    if (S.act && S.mlp.cap >= rows) return TSALLIS_OK;
    int cap = S.mlp.cap > 0 ? S.mlp.cap : 256;
    while (cap < rows) cap *= 2;
    if (S.act) {
        if (cudaDeviceSynchronize() != cudaSuccess) return TSALLIS_ERR_CUDA;
        cudaFree(S.act);
        S.act = nullptr;
        S.mlp.cap = 0;
    }
    const size_t h = (size_t)cap * kMlpHid, o = (size_t)cap * kMlpOut;
    if (cudaMalloc(&S.act, (6 * h + 2 * o) * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return TSALLIS_ERR_OOM;
    }
    float* f = static_cast<float*>(S.act);
    S.mlp.z1 = f; S.mlp.a1 = f + h; S.mlp.z2 = f + 2 * h; S.mlp.a2 = f + 3 * h;
    S.mlp.da = f + 4 * h; S.mlp.dz = f + 5 * h;
    S.mlp.z3 = f + 6 * h; S.mlp.d3 = f + 6 * h + o;
    S.mlp.cap = cap;
    return TSALLIS_OK;
}

constexpr int kPropChunk = 1024;   // histograms per proposer pass

tsallis_status ensure_prop(tsallis_ctx* c, int rows) {
    if (c->prop_x && c->prop_cap >= rows) return TSALLIS_OK;
    if (c->prop_x) {
        if (cudaDeviceSynchronize() != cudaSuccess) return TSALLIS_ERR_CUDA;
        cudaFree(c->prop_x);
        c->prop_x = nullptr;
        c->prop_cand = nullptr;
        c->prop_cap = 0;
    }
    void* b = nullptr;
    const size_t main = (size_t)rows * (kMlpIn * sizeof(float) + 256 * sizeof(int32_t));
    if (cudaMalloc(&b, main + 256) != cudaSuccess) {
        cudaGetLastError();
        return TSALLIS_ERR_OOM;
    }
    c->prop_x = static_cast<float*>(b);
    c->prop_cand = reinterpret_cast<int32_t*>(c->prop_x + (size_t)rows * kMlpIn);
    c->prop_sync = reinterpret_cast<unsigned*>(static_cast<char*>(b) + main);   // the fused kernel's barrier words
    if (cudaMemset(c->prop_sync, 0, 256) != cudaSuccess) return TSALLIS_ERR_CUDA;
    c->prop_cap = rows;
    return TSALLIS_OK;
}

// The proposer's top k of n rows, from histograms (1-D or 2-D features) or
// from features x: one fused launch for up to kMlpInferRows rows and
// k <= 64, else the features, forward and top-k kernels. The slot's
// activations and the context's proposer buffers must hold n rows.
cudaError_t propose(tsallis_ctx* c, ProposerSlot& S, const int32_t* hist, bool two_d, const float* x, int n, int k,
                    int32_t* cand, cudaStream_t s) {
    cudaError_t e;
    if (hist && two_d) {
        if ((e = mlp_features2d(hist, n, c->prop_x, s)) != cudaSuccess) return e;
        hist = nullptr;
        x = c->prop_x;
    }
    if (n <= kMlpInferRows && k <= 64)
        return mlp_infer(S.mlp, hist, x, c->prop_x, n, k, cand, c->prop_sync, c->timeout_ns, s);
    if (hist) {
        if ((e = mlp_features(hist, n, c->prop_x, s)) != cudaSuccess) return e;
        x = c->prop_x;
    }
    if ((e = mlp_forward(S.mlp, x, n, s)) != cudaSuccess) return e;
    return mlp_topk(S.mlp.z3, n, k, cand, s);
}

// Window search of nh 1-D histograms: features, proposer, the top k
// levels, then the certified window search (search1d.cuh).
tsallis_status search_window(tsallis_ctx* c, const int32_t* d_hist, long long nh, const tsallis_params* p,
                             int32_t* d_t, float* d_phi, int32_t* d_status, cudaStream_t stream) {
    ProposerSlot& S = c->prop[0];
    if (!S.ready) return TSALLIS_ERR_INVALID_ARG;   // no proposer was set
    if (p->nbins != kMlpOut || p->two_d || p->topk < 1 || p->topk > 256) return TSALLIS_ERR_INVALID_ARG;
    tsallis_status st;
    const int chunk = (int)(nh < kPropChunk ? nh : kPropChunk);
    if ((st = ensure_mlp_act(c, 0, chunk)) != TSALLIS_OK || (st = ensure_prop(c, chunk)) != TSALLIS_OK) return st;
    for (long long h0 = 0; h0 < nh; h0 += chunk) {
        const int n = (int)(nh - h0 < chunk ? nh - h0 : chunk);
        const int32_t* hist = d_hist + h0 * kMlpOut;
        if (propose(c, S, hist, false, nullptr, n, p->topk, c->prop_cand, stream) != cudaSuccess ||
            launch_search1d_window(hist, n, kMlpOut, p->q, c->prop_cand, p->topk, d_t + h0, d_phi + h0,
                                   d_status + h0, c->df_tables, stream) != cudaSuccess)
            return TSALLIS_ERR_CUDA;
    }
    return TSALLIS_OK;
}

struct ScratchView {
    ScratchHeader* hdr;
    int* arrive;
    int* done_flag;
    int* bdone;
    unsigned long long* that;
    int* ghist;
    unsigned long long* bq;
    int* exc_n;
    unsigned long long* exc;
};

ScratchView view(tsallis_ctx* c) {
    char* b = (char*)c->scratch;
    size_t goff = 0, qoff = 0, eoff = 0;
    scratch_layout(c->cap_groups, c->cap_tiles, c->cap_exc, &goff, &qoff, &eoff);
    ScratchView v;
    v.hdr = (ScratchHeader*)b;
    v.arrive = (int*)(b + sizeof(ScratchHeader));
    v.done_flag = v.arrive + c->cap_groups;
    v.bdone = v.done_flag + c->cap_groups;
    v.that = reinterpret_cast<unsigned long long*>(v.bdone + c->cap_groups);
    v.ghist = (int*)(b + goff);
    v.bq = (unsigned long long*)(b + qoff);
    v.exc_n = (int*)(b + eoff);
    v.exc = (unsigned long long*)(b + ((eoff + (size_t)c->cap_groups * sizeof(int) + 255) & ~size_t(255)));
    return v;
}

// 2-D buffer: grows (never shrinks) to hold `bytes`; synchronises the device
// before replacing a smaller buffer that earlier work may still use.
tsallis_status ensure_s2(tsallis_ctx* c, size_t bytes) {
    if (c->s2_buf && bytes <= c->s2_bytes) return TSALLIS_OK;
    size_t cap = c->s2_bytes > 0 ? c->s2_bytes : (size_t)1 << 22;
    while (cap < bytes) cap *= 2;
    if (c->s2_buf) {
        if (cudaDeviceSynchronize() != cudaSuccess) return TSALLIS_ERR_CUDA;
        cudaFree(c->s2_buf);
        c->s2_buf = nullptr;
        c->s2_bytes = 0;
    }
    if (cudaMalloc(&c->s2_buf, cap) != cudaSuccess) {
        cudaGetLastError();
        return TSALLIS_ERR_OOM;
    }
    c->s2_bytes = cap;
    return TSALLIS_OK;
}

constexpr long long kSearch2dChunk = 64;   // histograms per 2-D search launch sequence
inline int levels2(const tsallis_params* p) { return p->nbins >> p->shift; }
// the 2-D window search's cell flags and counts follow the search tables
inline size_t s2_window_bytes(const tsallis_params* p, long long K) {
    return p->topk > 0 ? (size_t)K * kCells2d + (size_t)K * sizeof(int) + 512 : 0;
}
inline size_t s2_search_bytes(const tsallis_params* p, long long K) {
    return ((p->flags & TSALLIS_FLAG_BRUTE_FORCE_2D) ? search2d_brute_scratch_bytes(levels2(p), K)
                                                     : search2d_scratch_bytes(levels2(p), K)) +
           s2_window_bytes(p, K);
}
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// The 2-D window search needs the 2-D proposer (slot 1) and 256 grey levels.
tsallis_status check_window2d(tsallis_ctx* c, const tsallis_params* p) {
    if (p->topk <= 0) return TSALLIS_OK;
    if (!c->prop[1].ready || levels2(p) != 256 || p->topk > 256 || (p->flags & TSALLIS_FLAG_BRUTE_FORCE_2D))
        return TSALLIS_ERR_INVALID_ARG;
    return TSALLIS_OK;
}

cudaError_t hist2d_enqueue(tsallis_ctx* c, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                           const tsallis_params* p, int32_t* d_hist, long long nh, cudaStream_t stream) {
    const int L2 = levels2(p);
    cudaError_t e = cudaMemsetAsync(d_hist, 0, (size_t)nh * L2 * L2 * sizeof(int32_t), stream);
    if (e != cudaSuccess) return e;
    Hist2dLaunch h;
    h.vol = d_vol;
    h.nx = (int)nx;
    h.ny = (int)ny;
    h.nz = (int)nz;
    h.lo = p->lo;
    h.L = p->nbins;
    h.shift = p->shift;
    h.per_slice = p->mode == TSALLIS_PER_SLICE;
    h.hist = d_hist;
    h.sm_count = c->sm_count;
    h.blocks_per_sm = c->hist2d_blocks_per_sm;
    return launch_hist2d(h, stream);
}

// Searches nh 2-D histograms in chunks that share one scratch area.
cudaError_t search2d_enqueue(tsallis_ctx* c, void* scratch, const int32_t* d_hist, long long nh,
                             const tsallis_params* p, int32_t* d_t, int32_t* d_tbin, float* d_phi, int32_t* d_status,
                             float* d_curve, cudaStream_t stream) {
    const int L2 = levels2(p);
    const long long cells = (long long)L2 * L2, m2 = (long long)(L2 - 1) * (L2 - 1);
    const bool window = p->topk > 0;
    const long long Kmax = nh < kSearch2dChunk ? nh : kSearch2dChunk;
    unsigned char* wbuf = nullptr;
    if (window) {
        if (ensure_mlp_act(c, 1, (int)Kmax) != TSALLIS_OK || ensure_prop(c, (int)Kmax) != TSALLIS_OK)
            return cudaErrorMemoryAllocation;
        wbuf = static_cast<unsigned char*>(scratch) + search2d_scratch_bytes(L2, Kmax);
    }
    for (long long k0 = 0; k0 < nh; k0 += kSearch2dChunk) {
        Search2dLaunch s{};
        s.check = c->check;
        s.K = nh - k0 < kSearch2dChunk ? nh - k0 : kSearch2dChunk;
        s.hist = d_hist + k0 * cells;
        s.L2 = L2;
        s.q = p->q;
        s.tables = c->df_tables;
        s.scratch = scratch;
        s.curve = d_curve ? d_curve + k0 * m2 : nullptr;
        s.t = d_t + 2 * k0;
        s.t_bin = d_tbin ? d_tbin + k0 : nullptr;
        s.phi = d_phi + k0;
        s.status = d_status + k0;
        cudaError_t e;
        if (p->flags & TSALLIS_FLAG_BRUTE_FORCE_2D) {
            e = launch_search2d_brute(s, stream);
        } else if (window) {
            // tables, then the proposer's candidate cells and the cells whose
            // bound reaches them, then evaluation of the flagged cells only
            s.topk = p->topk;
            s.cand = c->prop_cand;
            s.cellflag = wbuf;
            s.winfo = reinterpret_cast<int*>(wbuf + align256((size_t)Kmax * kCells2d));
            e = launch_search2d_tables(s, stream);
            if (e == cudaSuccess) e = propose(c, c->prop[1], s.hist, true, nullptr, (int)s.K, p->topk, c->prop_cand, stream);
            if (e == cudaSuccess) e = launch_search2d_window(s, stream);
            if (e == cudaSuccess) e = launch_search2d_finish(s, stream);
        } else {
            e = launch_search2d(s, stream);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int grid_for(tsallis_ctx* c, unsigned nitems) {
    long long g = (long long)c->sm_count * (c->blocks_per_sm > 0 ? c->blocks_per_sm : 1);
    if ((long long)nitems < g) g = nitems;
    return (int)(g < 1 ? 1 : g);
}

void fill_common(SegArgs& a, const tsallis_params* p, tsallis_ctx* c) {
    std::memset(&a, 0, sizeof(a));
    a.lo = p->lo;
    a.L = p->nbins;
    a.q = p->q;
    a.polarity = p->polarity;
    a.bin_shift = 0;
    a.t_stride = 1;
    a.flags = p->flags;
    a.timeout_ns = c->timeout_ns;
    a.tile_vox = c->tile_vox;
    a.df_tables = c->df_tables;
    a.check = c->check;
}

tsallis_status cuda_status(cudaError_t e) { return e == cudaSuccess ? TSALLIS_OK : TSALLIS_ERR_CUDA; }

// 2-D steps 1-4: histogram kernel, search kernels, then the binarise phase
// of the 1-D persistent kernel on the grey levels. The 2-D buffer holds the
// histograms, the search tables and the thresholds t alone.
tsallis_status segment2d(tsallis_ctx* c, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                         const tsallis_params* p, long long ng, long long gvox, uint8_t* d_mask, int32_t* d_t,
                         float* d_phi, int32_t* d_status, cudaStream_t stream) {
    const int L2 = levels2(p);
    const long long K = ng < kSearch2dChunk ? ng : kSearch2dChunk;
    const size_t hist_bytes = align256((size_t)ng * L2 * L2 * sizeof(int32_t));
    const size_t tbin_bytes = align256((size_t)ng * sizeof(int32_t));
    const size_t search_bytes = s2_search_bytes(p, K);
    tsallis_status st = check_window2d(c, p);
    if (st != TSALLIS_OK) return st;
    if ((st = ensure_scratch(c, 0, 0)) != TSALLIS_OK) return st;
    if ((st = ensure_s2(c, hist_bytes + tbin_bytes + search_bytes)) != TSALLIS_OK) return st;
    unsigned char* b = static_cast<unsigned char*>(c->s2_buf);
    int32_t* hist = reinterpret_cast<int32_t*>(b);
    int32_t* tbin = reinterpret_cast<int32_t*>(b + hist_bytes);
    void* search = b + hist_bytes + tbin_bytes;
    cudaError_t e = hist2d_enqueue(c, d_vol, nx, ny, nz, p, hist, ng, stream);
    if (e == cudaSuccess) e = search2d_enqueue(c, search, hist, ng, p, d_t, tbin, d_phi, d_status, nullptr, stream);
    if (e != cudaSuccess) return TSALLIS_ERR_CUDA;
    SegArgs a;
    fill_common(a, p, c);
    a.bin_shift = p->shift;
    a.vol = d_vol;
    a.mask = d_mask;
    a.group_vox = gvox;
    a.ngroups = (int)ng;
    a.ntiles = (int)((gvox + a.tile_vox - 1) / a.tile_vox);
    a.phases = kPhaseBin;
    if (ng * a.ntiles > 0xffffffffll) return TSALLIS_ERR_INVALID_ARG;
    a.ntotal = (unsigned)(ng * a.ntiles);
    a.t_in = tbin;
    ScratchView v = view(c);
    a.hdr = v.hdr;
    return cuda_status(launch_segment1d(a, grid_for(c, a.ntotal), c->copies, stream));
}

// The cluster kernel, when chosen, takes per-slice 1-D work whose slices
// are whole 16-byte words and fit in one cluster's shared memory.
// The cluster kernel takes slices of whole 16-byte groups that fit a
// cluster's shared memory: always when selected, and by default (AUTO) for
// volumes of at most twice as many slices as clusters fit at once, where its
// one read per voxel beats the tile kernel (measured: one 512x512 slice
// 16.4 against 32.8 us, 16 slices 22.6 against 36.6 us; at 400 slices the
// tile kernel is faster, 0.124 against 0.185 ms).
bool use_slice_cluster(const tsallis_ctx* c, const tsallis_params* p, long long slice, long long nz) {
    if (c->cluster_max < 1) return false;
    if (c->slice_kernel != TSALLIS_SLICE_KERNEL_CLUSTER &&
        !(c->slice_kernel == TSALLIS_SLICE_KERNEL_AUTO && !c->speculate && p->topk == 0 &&
          nz <= 2ll * c->cluster_max))
        return false;
    return p->mode == TSALLIS_PER_SLICE && !p->two_d && slice % 8 == 0 &&
           slice <= (long long)kClusterCtas * kClusterPartVox;
}

// The predicted first-pass kernel (when selected) takes per-slice 1-D work
// whose slices are whole 16-byte words of at most kSpecMaxSlice voxels.
bool use_slice_spec(const tsallis_ctx* c, const tsallis_params* p, long long slice, long long nz) {
    if (c->slice_kernel != TSALLIS_SLICE_KERNEL_PREDICT) return false;
    return p->mode == TSALLIS_PER_SLICE && !p->two_d && p->topk == 0 && slice % 8 == 0 &&
           slice <= kSpecMaxSlice && nz <= (1 << 19);   // queue entries hold the slice in 20 bits
}

// Arrays of the predicted first-pass kernel in one buffer (grown, never
// shrunk; zeroed when allocated): predicted thresholds [nz] (u64), slice
// flags [nz], second-pass queue [nz * npiece], list starts and lengths
// [grid * nseg * 16] each, lists [grid * 16 * wcap]. The kernel leaves the
// thresholds and flags zeroed; the others are written before they are read.
struct SpecView {
    unsigned long long* pred;
    int* sflag;
    unsigned* rbq;
    int* toff;
    int* tcnt;
    unsigned* exc;
};
inline size_t spec_layout(long long nz, long long nq, long long nl, long long nexc, SpecView* v, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (off + bytes + 255) & ~size_t(255);
        return o;
    };
    const size_t o_pred = take((size_t)nz * 8), o_flag = take((size_t)nz * 4), o_rbq = take((size_t)nq * 4),
                 o_toff = take((size_t)nl * 4), o_tcnt = take((size_t)nl * 4), o_exc = take((size_t)nexc * 4);
    if (v) {
        v->pred = reinterpret_cast<unsigned long long*>(base + o_pred);
        v->sflag = reinterpret_cast<int*>(base + o_flag);
        v->rbq = reinterpret_cast<unsigned*>(base + o_rbq);
        v->toff = reinterpret_cast<int*>(base + o_toff);
        v->tcnt = reinterpret_cast<int*>(base + o_tcnt);
        v->exc = reinterpret_cast<unsigned*>(base + o_exc);
    }
    return off;
}

// A buffer is reused only for the same layout; a new layout gets a new
// zeroed buffer.
tsallis_status ensure_spec(tsallis_ctx* c, long long nz, long long nq, long long nl, long long nexc, SpecView* v) {
    const size_t bytes = spec_layout(nz, nq, nl, nexc, nullptr, nullptr);
    const bool same = c->spec_buf && c->spec_nz == nz && c->spec_ntot == nq && c->spec_nl == nl && c->spec_nexc == nexc;
    if (!same) {
        if (c->spec_buf) {
            if (cudaDeviceSynchronize() != cudaSuccess) return TSALLIS_ERR_CUDA;
            cudaFree(c->spec_buf);
            c->spec_buf = nullptr;
            c->spec_bytes = 0;
        }
        if (cudaMalloc(&c->spec_buf, bytes) != cudaSuccess) {
            cudaGetLastError();
            return TSALLIS_ERR_OOM;
        }
        if (cudaMemset(c->spec_buf, 0, bytes) != cudaSuccess) return TSALLIS_ERR_CUDA;
        c->spec_bytes = bytes;
        c->spec_nz = nz;
        c->spec_ntot = nq;
        c->spec_nl = nl;
        c->spec_nexc = nexc;
    }
    spec_layout(nz, nq, nl, nexc, v, static_cast<char*>(c->spec_buf));
    return TSALLIS_OK;
}

tsallis_status segment_spec(tsallis_ctx* c, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                            const tsallis_params* p, uint8_t* d_mask, int32_t* d_t, float* d_phi, int32_t* d_status,
                            cudaStream_t stream) {
    const long long S = nx * ny, V = S * nz;
    const long long G = (long long)c->sm_count * c->spec_blocks_per_sm;
    // the largest range of a block, the slices it can meet, the lists a warp keeps
    const long long rmax = ((V / G + 7) / 8) * 8 + 8;
    const long long nseg = (rmax + S - 1) / S + 1;
    const long long wcap = rmax / kSpecWarps / 16 > kSpecWarpList ? rmax / kSpecWarps / 16 : kSpecWarpList;
    const int piece = 65536;
    const long long npiece = (S + piece - 1) / piece;
    if (npiece >= 4096) return TSALLIS_ERR_INVALID_ARG;
    tsallis_status st;
    if ((st = ensure_scratch(c, nz, 0)) != TSALLIS_OK) return st;
    SpecView sv;
    if ((st = ensure_spec(c, nz, nz * npiece, G * nseg * kSpecWarps, G * kSpecWarps * wcap, &sv)) != TSALLIS_OK)
        return st;
    SpecArgs a;
    std::memset(&a, 0, sizeof(a));
    a.vol = d_vol;
    a.mask = d_mask;
    a.slice_vox = S;
    a.nvox = V;
    a.nx = (int)nx;
    a.ny = (int)ny;
    a.nz = (int)nz;
    a.nseg = (int)nseg;
    a.wcap = (int)wcap;
    a.piece_vox = piece;
    a.npiece = (int)npiece;
    a.sub_stride = c->spec_stride;
    a.win = c->spec_win;
    a.lo = p->lo;
    a.L = p->nbins;
    a.q = p->q;
    a.polarity = p->polarity;
    a.flags = (p->flags & TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL) | c->spec_test_flags;
    a.timeout_ns = c->timeout_ns;
    ScratchView v = view(c);
    a.hdr = v.hdr;
    a.ghist = v.ghist;
    a.pred = sv.pred;
    a.sflag = sv.sflag;
    a.toff = sv.toff;
    a.tcnt = sv.tcnt;
    a.exc = sv.exc;
    a.rbq = sv.rbq;
    a.t_out = d_t;
    a.phi_out = d_phi;
    a.status = d_status;
    a.df_tables = c->df_tables;
    a.ptab = pow_table(c, S, p->q, stream);
    a.ptab_n = S;
    a.check = c->check;
    return cuda_status(launch_slice_spec(a, (int)G, stream));
}

// The pipelined kernel takes per-slice 1-D work whose slices are whole
// 16-byte words.
bool use_slice_pipe(const tsallis_ctx* c, const tsallis_params* p, long long slice, long long nz) {
    if (c->slice_kernel != TSALLIS_SLICE_KERNEL_PIPELINE) return false;
    return p->mode == TSALLIS_PER_SLICE && !p->two_d && p->topk == 0 && slice % 8 == 0 && slice <= kPipeMaxSlice &&
           nz <= (1 << 28);
}

// Per-slice counters [nz] (int), readiness words [nz] (u64) and the blocks'
// list regions [nexc] (u32) in one buffer, grown (never shrunk) and zeroed
// when allocated; the kernel leaves the counters zeroed, tags the readiness
// words with its launch number and writes list entries before reading them.
tsallis_status ensure_pipe(tsallis_ctx* c, long long nz, long long nexc, int** parts, unsigned long long** ready,
                           unsigned** exc) {
    auto layout = [](long long n, size_t* o_ready, size_t* o_exc) {
        *o_ready = ((size_t)n * 4 + 255) & ~size_t(255);
        *o_exc = (*o_ready + (size_t)n * 8 + 255) & ~size_t(255);
    };
    size_t o_ready, o_exc;
    if (!c->pipe_buf || c->pipe_nz < nz || c->pipe_nexc < nexc) {
        if (c->pipe_buf) {
            if (cudaDeviceSynchronize() != cudaSuccess) return TSALLIS_ERR_CUDA;
            cudaFree(c->pipe_buf);
            c->pipe_buf = nullptr;
            c->pipe_nz = 0;
            c->pipe_nexc = 0;
        }
        layout(nz, &o_ready, &o_exc);
        const size_t bytes = o_exc + (size_t)nexc * 4;
        if (cudaMalloc(&c->pipe_buf, bytes) != cudaSuccess) {
            cudaGetLastError();
            return TSALLIS_ERR_OOM;
        }
        if (cudaMemset(c->pipe_buf, 0, bytes) != cudaSuccess) return TSALLIS_ERR_CUDA;
        c->pipe_nz = nz;
        c->pipe_nexc = nexc;
    }
    layout(c->pipe_nz, &o_ready, &o_exc);
    char* b = static_cast<char*>(c->pipe_buf);
    *parts = reinterpret_cast<int*>(b);
    *ready = reinterpret_cast<unsigned long long*>(b + o_ready);
    *exc = reinterpret_cast<unsigned*>(b + o_exc);
    return TSALLIS_OK;
}

tsallis_status segment_pipe(tsallis_ctx* c, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                            const tsallis_params* p, uint8_t* d_mask, int32_t* d_t, float* d_phi, int32_t* d_status,
                            cudaStream_t stream) {
    const long long S = nx * ny;
    const long long G = (long long)c->sm_count * c->pipe_blocks_per_sm;
    tsallis_status st;
    if ((st = ensure_scratch(c, nz, 0)) != TSALLIS_OK) return st;
    PipeArgs a;
    std::memset(&a, 0, sizeof(a));
    a.chunks_per_slice = pipe_chunks_per_slice(S, &a.chunk_vox);
    // a warp lists up to a quarter of the 16-byte groups it counts in a chunk (at least 256)
    a.wcap = (int)(a.chunk_vox / 8 / kSpecWarps / 4 > kSpecWarpList ? a.chunk_vox / 8 / kSpecWarps / 4 : kSpecWarpList);
    a.win = c->spec_win;
    if ((st = ensure_pipe(c, nz, G * kPipeRing * kSpecWarps * a.wcap, &a.parts, &a.ready, &a.exc)) != TSALLIS_OK)
        return st;
    a.vol = d_vol;
    a.mask = d_mask;
    a.slice_vox = S;
    a.nz = (int)nz;
    a.lo = p->lo;
    a.L = p->nbins;
    a.q = p->q;
    a.polarity = p->polarity;
    a.flags = (p->flags & TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL) | (c->spec_test_flags ? kPipeDebugNoPrediction : 0u);
    a.timeout_ns = c->timeout_ns;
    ScratchView v = view(c);
    a.hdr = v.hdr;
    a.ghist = v.ghist;
    a.t_out = d_t;
    a.phi_out = d_phi;
    a.status = d_status;
    a.df_tables = c->df_tables;
    a.ptab = pow_table(c, S, p->q, stream);
    a.ptab_n = S;
    a.check = c->check;
    return cuda_status(launch_slice_pipe(a, (int)G, stream));
}

}  // namespace

extern "C" {

tsallis_status tsallis_params_default(tsallis_params* p) {
    if (!p) return TSALLIS_ERR_INVALID_ARG;
    p->lo = -1024;
    p->nbins = 4096;
    p->q = 0.8f;
    p->mode = TSALLIS_PER_SLICE;
    p->polarity = TSALLIS_MASK_LOW;
    p->two_d = 0;
    p->shift = 4;
    p->topk = 0;
    p->flags = 0;
    return TSALLIS_OK;
}

const char* tsallis_status_string(int32_t status) {
    switch (status & 0xff) {
        case TSALLIS_OK: return "ok";
        case TSALLIS_ERR_INVALID_ARG: return "invalid argument";
        case TSALLIS_ERR_ALIGNMENT: return "pointer not 16-byte aligned";
        case TSALLIS_ERR_CUDA: return "CUDA runtime error";
        case TSALLIS_ERR_NO_VALID_THRESHOLD: return "no valid threshold (fewer than two non-empty levels)";
        case TSALLIS_ERR_TIMEOUT: return "device wait timed out";
        case TSALLIS_ERR_OOM: return "out of device memory";
        case TSALLIS_ERR_UNIMPLEMENTED: return "not implemented";
        default: return "unknown status";
    }
}

tsallis_status tsallis_create(tsallis_ctx** out, int device) {
    TSL_TRACE();
    if (!out) return TSALLIS_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return device < 0 ? TSALLIS_ERR_INVALID_ARG : TSALLIS_ERR_CUDA;
    }
    tsallis_ctx* c = new (std::nothrow) tsallis_ctx();
    if (!c) return TSALLIS_ERR_OOM;
    c->device = device;
    DeviceGuard g(device);
    int l2 = 0;
    if (!g.ok() || cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device) != cudaSuccess) {
        delete c;
        return TSALLIS_ERR_CUDA;
    }
    c->l2_bytes = l2;
    if (segment1d_prepare() != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return TSALLIS_ERR_CUDA;
    }
    if (segment1d_occupancy(c->copies, kMaxLevels, &c->max_blocks_per_sm) != cudaSuccess ||
        c->max_blocks_per_sm < 1) {
        delete c;
        return TSALLIS_ERR_CUDA;
    }
    c->blocks_per_sm = c->max_blocks_per_sm;
    if (slice_cluster_prepare() != cudaSuccess || slice_cluster_occupancy(&c->cluster_max) != cudaSuccess) {
        cudaGetLastError();
        c->cluster_max = 0;   // the tile kernel serves every shape
    }
    if (slice_spec_prepare() != cudaSuccess || slice_spec_occupancy(&c->spec_blocks_per_sm) != cudaSuccess ||
        c->spec_blocks_per_sm < 1) {
        cudaGetLastError();
        delete c;
        return TSALLIS_ERR_CUDA;
    }
    if (slice_pipe_prepare() != cudaSuccess || slice_pipe_occupancy(&c->pipe_blocks_per_sm) != cudaSuccess ||
        c->pipe_blocks_per_sm < 1) {
        cudaGetLastError();
        delete c;
        return TSALLIS_ERR_CUDA;
    }
    if (preproc_prepare() != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return TSALLIS_ERR_CUDA;
    }
    if (mlp_prepare() != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return TSALLIS_ERR_CUDA;
    }
    if (seg2d_prepare() != cudaSuccess || hist2d_occupancy(&c->hist2d_blocks_per_sm) != cudaSuccess ||
        c->hist2d_blocks_per_sm < 1) {
        cudaGetLastError();
        delete c;
        return TSALLIS_ERR_CUDA;
    }
    // double-float tables: the small reduction tables (host-built), then a
    // log2 table of counts up to 2^18 computed on the device from them
    std::vector<unsigned char> tab(df_tables_bytes());
    if (cudaMalloc(&c->log2_table, sizeof(float) * 2 * (size_t)(kLog2TableMax + 1)) != cudaSuccess ||
        cudaMalloc(&c->df_tables, tab.size()) != cudaSuccess) {
        cudaGetLastError();
        if (c->log2_table) cudaFree(c->log2_table);
        delete c;
        return TSALLIS_ERR_OOM;
    }
    df_tables_fill(tab.data(), c->log2_table, kLog2TableMax);
    if (cudaMemcpy(c->df_tables, tab.data(), tab.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        build_log2_table(c->log2_table, kLog2TableMax + 1, c->df_tables, 0) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(c->df_tables);
        cudaFree(c->log2_table);
        delete c;
        return TSALLIS_ERR_CUDA;
    }
    if (cudaMalloc(&c->check, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(c->check, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        tsallis_destroy(c);
        return TSALLIS_ERR_CUDA;
    }
    *out = c;
    return TSALLIS_OK;
}

void tsallis_destroy(tsallis_ctx* c) {
    if (!c) return;
    {
        DeviceGuard g(c->device);
        if (c->scratch) cudaFree(c->scratch);
        if (c->batch_buf) cudaFree(c->batch_buf);
        if (c->s2_buf) cudaFree(c->s2_buf);
        if (c->df_tables) cudaFree(c->df_tables);
        if (c->log2_table) cudaFree(c->log2_table);
        if (c->ptab) cudaFree(c->ptab);
        for (ProposerSlot& S : c->prop) {
            if (S.params) cudaFree(S.params);
            if (S.act) cudaFree(S.act);
        }
        if (c->prop_x) cudaFree(c->prop_x);
        if (c->pred_buf) cudaFree(c->pred_buf);
        if (c->check) cudaFree(c->check);
        if (c->hp_buf) cudaFree(c->hp_buf);
        if (c->spec_buf) cudaFree(c->spec_buf);
        if (c->pipe_buf) cudaFree(c->pipe_buf);
        if (c->hp_ready) {
            for (cudaStream_t& h : c->hp_stream) cudaStreamDestroy(h);
            for (cudaEvent_t& e : c->hp_ev) cudaEventDestroy(e);
        }
    }
    delete c;
}

tsallis_status tsallis_set_wait_timeout(tsallis_ctx* c, uint64_t ns) {
    if (!c || ns == 0) return TSALLIS_ERR_INVALID_ARG;
    c->timeout_ns = ns;
    return TSALLIS_OK;
}

tsallis_status tsallis_set_launch_shape(tsallis_ctx* c, int32_t tile_vox, int32_t blocks_per_sm) {
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    if (tile_vox < 4096 || tile_vox > (1 << 22) || (tile_vox & 7)) return TSALLIS_ERR_INVALID_ARG;
    if (blocks_per_sm < 0 || blocks_per_sm > c->max_blocks_per_sm) return TSALLIS_ERR_INVALID_ARG;
    c->tile_vox = tile_vox;
    c->blocks_per_sm = blocks_per_sm > 0 ? blocks_per_sm : c->max_blocks_per_sm;
    return TSALLIS_OK;
}

tsallis_status tsallis_set_slice_kernel(tsallis_ctx* c, int32_t kind) {
    if (!c || (kind != TSALLIS_SLICE_KERNEL_AUTO && kind != TSALLIS_SLICE_KERNEL_TILES &&
               kind != TSALLIS_SLICE_KERNEL_CLUSTER && kind != TSALLIS_SLICE_KERNEL_PREDICT &&
               kind != TSALLIS_SLICE_KERNEL_PIPELINE))
        return TSALLIS_ERR_INVALID_ARG;
    if (kind == TSALLIS_SLICE_KERNEL_CLUSTER && c->cluster_max < 1) return TSALLIS_ERR_UNIMPLEMENTED;
    c->slice_kernel = kind;
    return TSALLIS_OK;
}

tsallis_status tsallis_set_speculation(tsallis_ctx* c, int32_t on) {
    if (!c || (on != 0 && on != 1)) return TSALLIS_ERR_INVALID_ARG;
    c->speculate = on;
    return TSALLIS_OK;
}

tsallis_status tsallis_set_prediction(tsallis_ctx* c, int32_t row_stride, int32_t window) {
    if (!c || row_stride < 1 || row_stride > 4096 || window < 1 || window > kSpecMaxWin) return TSALLIS_ERR_INVALID_ARG;
    c->spec_stride = row_stride;
    c->spec_win = window;
    return TSALLIS_OK;
}

tsallis_status tsallis_test_withhold_predictions(tsallis_ctx* c, int32_t on) {
    if (!c || (on != 0 && on != 1)) return TSALLIS_ERR_INVALID_ARG;
    c->spec_test_flags = on ? kSpecDebugNoPrediction : 0u;
    return TSALLIS_OK;
}

tsallis_status tsallis_histogram(tsallis_ctx* c, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                                 const tsallis_params* p, int32_t* d_hist, cudaStream_t stream) {
    TSL_TRACE();
    tsallis_status st = check_params(p);
    if (st != TSALLIS_OK) return st;
    if ((st = check_shape(nx, ny, nz)) != TSALLIS_OK) return st;
    if (nz == 0) return TSALLIS_OK;
    if (!d_vol || !d_hist) return TSALLIS_ERR_INVALID_ARG;
    if (!aligned16(d_vol)) return TSALLIS_ERR_ALIGNMENT;
    const long long slice = nx * ny;
    const long long gvox = p->mode == TSALLIS_PER_SLICE ? slice : slice * nz;
    const long long ng = p->mode == TSALLIS_PER_SLICE ? nz : 1;
    if (gvox > (1ll << 31) - 1) return TSALLIS_ERR_INVALID_ARG;
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    if (p->two_d) return cuda_status(hist2d_enqueue(c, d_vol, nx, ny, nz, p, d_hist, ng, stream));
    if ((st = ensure_scratch(c, 0, 0)) != TSALLIS_OK) return st;
    if (cudaMemsetAsync(d_hist, 0, (size_t)ng * p->nbins * sizeof(int32_t), stream) != cudaSuccess)
        return TSALLIS_ERR_CUDA;
    SegArgs a;
    fill_common(a, p, c);
    a.vol = d_vol;
    a.group_vox = gvox;
    a.ngroups = (int)ng;
    a.ntiles = (int)((gvox + a.tile_vox - 1) / a.tile_vox);
    a.phases = kPhaseHist;
    if (ng * a.ntiles > 0xffffffffll) return TSALLIS_ERR_INVALID_ARG;
    a.ntotal = (unsigned)(ng * a.ntiles);
    ScratchView v = view(c);
    a.hdr = v.hdr;
    a.ghist = d_hist;
    return cuda_status(launch_segment1d(a, grid_for(c, a.ntotal), c->copies, stream));
}

tsallis_status tsallis_search(tsallis_ctx* c, const int32_t* d_hist, int64_t nh, const tsallis_params* p,
                              int32_t* d_t, float* d_phi, int32_t* d_status, float* d_curve, cudaStream_t stream) {
    TSL_TRACE();
    tsallis_status st = check_params(p);
    if (st != TSALLIS_OK) return st;
    if (nh < 0 || nh > (1ll << 31) - 1) return TSALLIS_ERR_INVALID_ARG;
    if (nh == 0) return TSALLIS_OK;
    if (!d_hist || !d_t || !d_phi || !d_status) return TSALLIS_ERR_INVALID_ARG;
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    if (p->two_d) {
        if ((st = check_window2d(c, p)) != TSALLIS_OK) return st;
        if (p->topk > 0 && d_curve) return TSALLIS_ERR_INVALID_ARG;   // the window evaluates only some pairs
        const long long K = nh < kSearch2dChunk ? nh : kSearch2dChunk;
        if ((st = ensure_s2(c, s2_search_bytes(p, K))) != TSALLIS_OK) return st;
        return cuda_status(search2d_enqueue(c, c->s2_buf, d_hist, nh, p, d_t, nullptr, d_phi, d_status, d_curve,
                                            stream));
    }
    if (p->topk > 0) {
        if (d_curve) return TSALLIS_ERR_INVALID_ARG;   // the window search evaluates only some levels
        return search_window(c, d_hist, nh, p, d_t, d_phi, d_status, stream);
    }
    return cuda_status(launch_search1d(d_hist, nh, p->nbins, p->q, d_t, d_phi, d_status, d_curve, c->df_tables,
                                       stream));
}

tsallis_status tsallis_binarize(tsallis_ctx* c, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                                const int32_t* d_t, const tsallis_params* p, uint8_t* d_mask, cudaStream_t stream) {
    TSL_TRACE();
    tsallis_status st = check_params(p);
    if (st != TSALLIS_OK) return st;
    if ((st = check_shape(nx, ny, nz)) != TSALLIS_OK) return st;
    if (nz == 0) return TSALLIS_OK;
    if (!d_vol || !d_mask || !d_t) return TSALLIS_ERR_INVALID_ARG;
    if (!aligned16(d_vol) || !aligned16(d_mask)) return TSALLIS_ERR_ALIGNMENT;
    const long long slice = nx * ny;
    const long long gvox = p->mode == TSALLIS_PER_SLICE ? slice : slice * nz;
    const long long ng = p->mode == TSALLIS_PER_SLICE ? nz : 1;
    if (gvox > (1ll << 31) - 1) return TSALLIS_ERR_INVALID_ARG;
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    if ((st = ensure_scratch(c, 0, 0)) != TSALLIS_OK) return st;
    SegArgs a;
    fill_common(a, p, c);
    if (p->two_d) {   // threshold t of each (t, s) pair, on the grey level
        a.bin_shift = p->shift;
        a.t_stride = 2;
    }
    a.vol = d_vol;
    a.mask = d_mask;
    a.group_vox = gvox;
    a.ngroups = (int)ng;
    a.ntiles = (int)((gvox + a.tile_vox - 1) / a.tile_vox);
    a.phases = kPhaseBin;
    if (ng * a.ntiles > 0xffffffffll) return TSALLIS_ERR_INVALID_ARG;
    a.ntotal = (unsigned)(ng * a.ntiles);
    a.t_in = d_t;
    ScratchView v = view(c);
    a.hdr = v.hdr;
    return cuda_status(launch_segment1d(a, grid_for(c, a.ntotal), c->copies, stream));
}

namespace {
// tsallis_segment with the kernel chosen as for a volume of nz_choice slices
// (the host-buffer entry point segments chunks of a volume and keeps the
// whole volume's choice, so its results equal the device path's bit for bit).
tsallis_status segment_impl(tsallis_ctx* c, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                            const tsallis_params* p, uint8_t* d_mask, int32_t* d_t, float* d_phi, int32_t* d_status,
                            cudaStream_t stream, long long nz_choice);
}  // namespace

tsallis_status tsallis_segment(tsallis_ctx* c, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                               const tsallis_params* p, uint8_t* d_mask, int32_t* d_t, float* d_phi,
                               int32_t* d_status, cudaStream_t stream) {
    TSL_TRACE();
    return segment_impl(c, d_vol, nx, ny, nz, p, d_mask, d_t, d_phi, d_status, stream, nz);
}

namespace {
tsallis_status segment_impl(tsallis_ctx* c, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                            const tsallis_params* p, uint8_t* d_mask, int32_t* d_t, float* d_phi, int32_t* d_status,
                            cudaStream_t stream, long long nz_choice) {
    tsallis_status st = check_params(p);
    if (st != TSALLIS_OK) return st;
    if ((st = check_shape(nx, ny, nz)) != TSALLIS_OK) return st;
    if (nz == 0) return TSALLIS_OK;
    if (!d_vol || !d_mask || !d_t || !d_phi || !d_status) return TSALLIS_ERR_INVALID_ARG;
    if (!aligned16(d_vol) || !aligned16(d_mask)) return TSALLIS_ERR_ALIGNMENT;
    const long long slice = nx * ny;
    const long long gvox = p->mode == TSALLIS_PER_SLICE ? slice : slice * nz;
    const long long ng = p->mode == TSALLIS_PER_SLICE ? nz : 1;
    if (gvox > (1ll << 31) - 1) return TSALLIS_ERR_INVALID_ARG;
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    if (p->two_d) return segment2d(c, d_vol, nx, ny, nz, p, ng, gvox, d_mask, d_t, d_phi, d_status, stream);
    if (p->topk > 0) {
        const tsallis_volume v{d_vol, d_mask, nx, ny, nz};
        return tsallis_segment_batch(c, &v, 1, p, d_t, d_phi, d_status, stream);
    }
    if (use_slice_pipe(c, p, slice, nz))
        return segment_pipe(c, d_vol, nx, ny, nz, p, d_mask, d_t, d_phi, d_status, stream);
    if (use_slice_spec(c, p, slice, nz))
        return segment_spec(c, d_vol, nx, ny, nz, p, d_mask, d_t, d_phi, d_status, stream);
    if (use_slice_cluster(c, p, slice, nz_choice)) {
        if ((st = ensure_scratch(c, 0, 0)) != TSALLIS_OK) return st;
        ClusterArgs a;
        std::memset(&a, 0, sizeof(a));
        a.vol = d_vol;
        a.mask = d_mask;
        a.slice_vox = slice;
        a.part_vox = ((slice + kClusterCtas - 1) / kClusterCtas + 7) / 8 * 8;
        a.nz = (int)nz;
        a.lo = p->lo;
        a.L = p->nbins;
        a.q = p->q;
        a.polarity = p->polarity;
        a.flags = p->flags;
        a.timeout_ns = c->timeout_ns;
        a.hdr = view(c).hdr;
        a.t_out = d_t;
        a.phi_out = d_phi;
        a.status = d_status;
        a.df_tables = c->df_tables;
        const int ncl = (int)(nz < c->cluster_max ? nz : c->cluster_max);
        return cuda_status(launch_slice_cluster(a, ncl, stream));
    }
    const long long ntiles_all = ng * ((gvox + c->tile_vox - 1) / c->tile_vox);
    if ((st = ensure_scratch(c, ng, ntiles_all, c->speculate ? exc_entries(ntiles_all, c->tile_vox) : 0)) !=
        TSALLIS_OK)
        return st;
    SegArgs a;
    fill_common(a, p, c);
    a.vol = d_vol;
    a.mask = d_mask;
    a.group_vox = gvox;
    a.ngroups = (int)ng;
    a.ntiles = (int)((gvox + a.tile_vox - 1) / a.tile_vox);
    a.phases = kPhaseHist | kPhaseSearch | kPhaseBin;
    if (ng * a.ntiles > 0xffffffffll) return TSALLIS_ERR_INVALID_ARG;
    a.ntotal = (unsigned)(ng * a.ntiles);
    ScratchView v = view(c);
    a.hdr = v.hdr;
    a.arrive = v.arrive;
    a.done_flag = v.done_flag;
    a.bdone = v.bdone;
    a.that = v.that;
    a.spec = c->speculate;
    a.exc = v.exc;
    a.exc_n = v.exc_n;
    a.exc_w = c->speculate ? kExcWindow : 0;
    if (p->mode == TSALLIS_PER_SLICE) {
        a.ptab = pow_table(c, gvox, p->q, stream);
        a.ptab_n = gvox;
    }
    a.bq = v.bq;
    a.ghist = v.ghist;
    a.t_out = d_t;
    a.phi_out = d_phi;
    a.status = d_status;
    return cuda_status(launch_segment1d(a, grid_for(c, a.ntotal), c->copies, stream));
}
}  // namespace

tsallis_status tsallis_probe_dfmath(tsallis_ctx* c, const uint32_t* d_h, int64_t n, uint32_t N, float q,
                                   double* d_pow, double* d_log2, cudaStream_t stream) {
    if (!c || n < 0 || N < 1 || !(q > 0.0f) || !(q <= 4.0f)) return TSALLIS_ERR_INVALID_ARG;
    if (n == 0) return TSALLIS_OK;
    if (!d_h || !d_pow || !d_log2) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    return cuda_status(launch_probe_dfmath(d_h, n, N, q, d_pow, d_log2, c->df_tables, stream));
}

tsallis_status tsallis_segment_batch(tsallis_ctx* c, const tsallis_volume* h_vols, int32_t nvol,
                                     const tsallis_params* p, int32_t* d_t, float* d_phi, int32_t* d_status,
                                     cudaStream_t stream) {
    TSL_TRACE();
    tsallis_status st = check_params(p);
    if (st != TSALLIS_OK) return st;
    if (!c || nvol < 0) return TSALLIS_ERR_INVALID_ARG;
    if (nvol == 0) return TSALLIS_OK;
    if (!h_vols || !d_t || !d_phi || !d_status) return TSALLIS_ERR_INVALID_ARG;
    ProposerSlot& S = c->prop[0];
    // validate every volume and lay out its groups and tiles
    std::vector<BatchVolDesc> vd((size_t)nvol);
    long long ng = 0, ntot = 0;
    for (int i = 0; i < nvol; ++i) {
        const tsallis_volume& v = h_vols[i];
        if ((st = check_shape(v.nx, v.ny, v.nz)) != TSALLIS_OK) return st;
        if (v.nz == 0) return TSALLIS_ERR_INVALID_ARG;
        if (!v.vol || !v.mask) return TSALLIS_ERR_INVALID_ARG;
        if (!aligned16(v.vol) || !aligned16(v.mask)) return TSALLIS_ERR_ALIGNMENT;
        const long long slice = v.nx * v.ny;
        const long long gvox = p->mode == TSALLIS_PER_SLICE ? slice : slice * v.nz;
        const long long gv = p->mode == TSALLIS_PER_SLICE ? v.nz : 1;
        if (gvox > (1ll << 31) - 1) return TSALLIS_ERR_INVALID_ARG;
        const long long nt = (gvox + c->tile_vox - 1) / c->tile_vox;
        vd[i] = BatchVolDesc{v.vol, v.mask, gvox, (int)gv, (int)nt, (int)ng, (int)ntot};
        ng += gv;
        ntot += gv * nt;
        // group and tile numbers must fit the work-queue entries (20 bits each)
        if (ng >= (1 << 20) - 1 || nt >= (1 << 20) - 1 || ntot > 0x7fffffffll) return TSALLIS_ERR_INVALID_ARG;
    }
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    if (p->two_d) {
        // the 2-D form runs volume by volume (its kernels take one volume)
        long long h = 0;
        for (int i = 0; i < nvol; ++i) {
            const tsallis_volume& v = h_vols[i];
            const long long gv = vd[i].ngroups;
            if ((st = segment2d(c, v.vol, v.nx, v.ny, v.nz, p, gv, vd[i].gvox, v.mask, d_t + 2 * h, d_phi + h,
                                d_status + h, stream)) != TSALLIS_OK)
                return st;
            h += gv;
        }
        return TSALLIS_OK;
    }
    const unsigned predict = p->flags & (TSALLIS_FLAG_PREDICT_PROPOSER | TSALLIS_FLAG_PREDICT_SUBSAMPLE);
    if (predict && (p->mode != TSALLIS_WHOLE_VOLUME || p->topk > 0 ||
                    ((predict & TSALLIS_FLAG_PREDICT_PROPOSER) && (!S.ready || p->nbins != kMlpOut))))
        return TSALLIS_ERR_INVALID_ARG;
    const bool spec = c->speculate || predict;
    // exception lists only for the speculation setting: with a prediction per
    // volume the first-pass mask is kept when it is exact as written (listing
    // the voxels near the prediction cost more than the second reads it saved)
    const bool lists = c->speculate && !predict;
    if ((st = ensure_scratch(c, ng, ntot, lists ? exc_entries(ntot, c->tile_vox) : 0)) != TSALLIS_OK) return st;
    // the group table, written on the device (capturable in a CUDA graph)
    const size_t table = (size_t)ng * sizeof(GroupDesc);
    if (!c->batch_buf || c->batch_bytes < table) {
        size_t cap = c->batch_bytes > 0 ? c->batch_bytes : 4096;
        while (cap < table) cap *= 2;
        if (c->batch_buf) {
            if (cudaDeviceSynchronize() != cudaSuccess) return TSALLIS_ERR_CUDA;
            cudaFree(c->batch_buf);
            c->batch_buf = nullptr;
            c->batch_bytes = 0;
        }
        if (cudaMalloc(&c->batch_buf, cap) != cudaSuccess) {
            cudaGetLastError();
            return TSALLIS_ERR_OOM;
        }
        c->batch_bytes = cap;
    }
    GroupDesc* groups = static_cast<GroupDesc*>(c->batch_buf);
    for (int i0 = 0; i0 < nvol; i0 += kExpandVols) {
        ExpandArgs ea;
        std::memset(&ea, 0, sizeof(ea));
        ea.nvol = nvol - i0 < kExpandVols ? nvol - i0 : kExpandVols;
        for (int k = 0; k < ea.nvol; ++k) ea.v[k] = vd[(size_t)(i0 + k)];
        const int gend = i0 + ea.nvol < nvol ? vd[(size_t)(i0 + ea.nvol)].group_off : (int)ng;
        ea.ngroups = gend - vd[(size_t)i0].group_off;
        ea.out = groups;
        if (launch_expand_groups(ea, stream) != cudaSuccess) return TSALLIS_ERR_CUDA;
    }
    if (p->topk > 0) {
        // window search: histograms, proposer + certified window search,
        // then Algorithm 1 (three launches; volumes are read twice as in
        // the one-launch path)
        if (!S.ready || p->nbins != kMlpOut) return TSALLIS_ERR_INVALID_ARG;
        ScratchView sv = view(c);
        const size_t hb = (size_t)ng * kMaxLevels * sizeof(int);
        SegArgs h;
        fill_common(h, p, c);
        h.groups = groups;
        h.ngroups = (int)ng;
        h.ntotal = (unsigned)ntot;
        h.phases = kPhaseHist;
        h.hdr = sv.hdr;
        h.ghist = sv.ghist;
        if (cudaMemsetAsync(sv.ghist, 0, hb, stream) != cudaSuccess ||
            launch_segment1d(h, grid_for(c, h.ntotal), c->copies, stream) != cudaSuccess)
            return TSALLIS_ERR_CUDA;
        if ((st = search_window(c, sv.ghist, ng, p, d_t, d_phi, d_status, stream)) != TSALLIS_OK) return st;
        SegArgs b = h;
        b.phases = kPhaseBin;
        b.t_in = d_t;
        b.t_stride = 1;
        if (cudaMemsetAsync(sv.ghist, 0, hb, stream) != cudaSuccess ||   // scratch left zeroed
            launch_segment1d(b, grid_for(c, b.ntotal), c->copies, stream) != cudaSuccess)
            return TSALLIS_ERR_CUDA;
        return TSALLIS_OK;
    }
    const int32_t* hints = nullptr;
    if (predict) {
        // predicted thresholds: the histogram of the middle sixteenth of each
        // volume's slices, read by the proposer (or searched exactly)
        const size_t tb = ((size_t)nvol * sizeof(GroupDesc) + 255) & ~size_t(255);
        const size_t hb = (size_t)nvol * kMaxLevels * sizeof(int32_t);
        const size_t need = tb + hb + 3 * (((size_t)nvol * 4 + 255) & ~size_t(255));
        if (!c->pred_buf || (size_t)c->pred_cap < need) {
            if (c->pred_buf) {
                if (cudaDeviceSynchronize() != cudaSuccess) return TSALLIS_ERR_CUDA;
                cudaFree(c->pred_buf);
                c->pred_buf = nullptr;
            }
            if (cudaMalloc(&c->pred_buf, need) != cudaSuccess) {
                cudaGetLastError();
                c->pred_cap = 0;
                return TSALLIS_ERR_OOM;
            }
            c->pred_cap = (int)need;
        }
        char* pb = static_cast<char*>(c->pred_buf);
        GroupDesc* sub = reinterpret_cast<GroupDesc*>(pb);
        int32_t* sh = reinterpret_cast<int32_t*>(pb + tb);
        const size_t vb = ((size_t)nvol * 4 + 255) & ~size_t(255);
        int32_t* ht = reinterpret_cast<int32_t*>(pb + tb + hb);
        float* hphi = reinterpret_cast<float*>(pb + tb + hb + vb);
        int32_t* hst = reinterpret_cast<int32_t*>(pb + tb + hb + 2 * vb);
        std::vector<BatchVolDesc> sd((size_t)nvol);
        long long stot = 0;
        for (int i = 0; i < nvol; ++i) {
            const tsallis_volume& v = h_vols[i];
            const long long slice = v.nx * v.ny;
            const long long ns = v.nz / 16 > 0 ? v.nz / 16 : 1, z0 = (v.nz - ns) / 2;
            const long long gv = ns * slice;
            const long long nt = (gv + c->tile_vox - 1) / c->tile_vox;
            sd[i] = BatchVolDesc{v.vol + z0 * slice, v.mask + z0 * slice, gv, 1, (int)nt, i, (int)stot};
            stot += nt;
        }
        for (int i0 = 0; i0 < nvol; i0 += kExpandVols) {
            ExpandArgs ea;
            std::memset(&ea, 0, sizeof(ea));
            ea.nvol = nvol - i0 < kExpandVols ? nvol - i0 : kExpandVols;
            for (int k = 0; k < ea.nvol; ++k) ea.v[k] = sd[(size_t)(i0 + k)];
            ea.ngroups = ea.nvol;
            ea.out = sub;
            if (launch_expand_groups(ea, stream) != cudaSuccess) return TSALLIS_ERR_CUDA;
        }
        SegArgs h;
        fill_common(h, p, c);
        h.groups = sub;
        h.ngroups = nvol;
        h.ntotal = (unsigned)stot;
        h.phases = kPhaseHist;
        h.hdr = view(c).hdr;
        h.ghist = sh;
        if (cudaMemsetAsync(sh, 0, hb, stream) != cudaSuccess ||
            launch_segment1d(h, grid_for(c, h.ntotal), c->copies, stream) != cudaSuccess)
            return TSALLIS_ERR_CUDA;
        if (predict & TSALLIS_FLAG_PREDICT_PROPOSER) {
            if ((st = ensure_mlp_act(c, 0, nvol)) != TSALLIS_OK || (st = ensure_prop(c, nvol)) != TSALLIS_OK) return st;
            if (propose(c, S, sh, false, nullptr, nvol, 1, ht, stream) != cudaSuccess) return TSALLIS_ERR_CUDA;
        } else if (launch_search1d(sh, nvol, p->nbins, p->q, ht, hphi, hst, nullptr, c->df_tables, stream) !=
                   cudaSuccess) {
            return TSALLIS_ERR_CUDA;
        }
        hints = ht;
    }
    SegArgs a;
    fill_common(a, p, c);
    a.groups = groups;
    a.ngroups = (int)ng;
    a.ntotal = (unsigned)ntot;
    a.phases = kPhaseHist | kPhaseSearch | kPhaseBin;
    a.flags = p->flags & TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL;
    ScratchView sv = view(c);
    a.hdr = sv.hdr;
    a.arrive = sv.arrive;
    a.done_flag = sv.done_flag;
    a.bdone = sv.bdone;
    a.that = sv.that;
    a.spec = spec;
    a.hint = hints;
    a.exc = sv.exc;
    a.exc_n = sv.exc_n;
    a.exc_w = lists ? kExcWindow : 0;
    if (p->mode == TSALLIS_PER_SLICE) {
        // slices of the first volume's size get the term table (others
        // compute their terms)
        a.ptab_n = vd[0].gvox;
        a.ptab = pow_table(c, a.ptab_n, p->q, stream);
    }
    a.bq = sv.bq;
    a.ghist = sv.ghist;
    a.t_out = d_t;
    a.phi_out = d_phi;
    a.status = d_status;
    return cuda_status(launch_segment1d(a, grid_for(c, a.ntotal), c->copies, stream));
}

tsallis_status tsallis_proposer_set(tsallis_ctx* c, const float* h_params, int64_t n) {
    TSL_TRACE();
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    ProposerSlot& S = c->prop[c->prop_sel];
    if (!h_params || n != kMlpParams) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    tsallis_status st = ensure_mlp_params(c, c->prop_sel);
    if (st != TSALLIS_OK) return st;
    const size_t f = (size_t)kMlpParams * sizeof(float);
    if (cudaMemcpy(S.mlp.p32, h_params, f, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(S.mlp.m, 0, f) != cudaSuccess || cudaMemset(S.mlp.v, 0, f) != cudaSuccess ||
        mlp_to_bf16(S.mlp.p32, S.mlp.p16, kMlpParams, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return TSALLIS_ERR_CUDA;
    S.step = 0;
    S.ready = true;
    return TSALLIS_OK;
}

tsallis_status tsallis_proposer_get(tsallis_ctx* c, float* h_params, int64_t n) {
    TSL_TRACE();
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    ProposerSlot& S = c->prop[c->prop_sel];
    if (!h_params || n != kMlpParams || !S.ready) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(h_params, S.mlp.p32, (size_t)kMlpParams * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TSALLIS_ERR_CUDA;
    return TSALLIS_OK;
}

namespace {
const char kPropMagic[8] = {'T', 'S', 'P', 'R', 'O', 'P', '0', '1'};
}

tsallis_status tsallis_proposer_load(tsallis_ctx* c, const char* path) {
    if (!c || !path) return TSALLIS_ERR_INVALID_ARG;
    FILE* f = std::fopen(path, "rb");
    if (!f) return TSALLIS_ERR_INVALID_ARG;
    char magic[8];
    int64_t n = 0;
    std::vector<float> buf;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kPropMagic, 8) == 0 &&
              std::fread(&n, sizeof(n), 1, f) == 1 && n == kMlpParams;
    if (ok) {
        buf.resize((size_t)n);
        ok = std::fread(buf.data(), sizeof(float), (size_t)n, f) == (size_t)n;
    }
    std::fclose(f);
    if (!ok) return TSALLIS_ERR_INVALID_ARG;
    return tsallis_proposer_set(c, buf.data(), n);
}

tsallis_status tsallis_proposer_save(tsallis_ctx* c, const char* path) {
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    ProposerSlot& S = c->prop[c->prop_sel];
    if (!path || !S.ready) return TSALLIS_ERR_INVALID_ARG;
    std::vector<float> buf((size_t)kMlpParams);
    tsallis_status st = tsallis_proposer_get(c, buf.data(), kMlpParams);
    if (st != TSALLIS_OK) return st;
    FILE* f = std::fopen(path, "wb");
    if (!f) return TSALLIS_ERR_INVALID_ARG;
    const int64_t n = kMlpParams;
    const bool ok = std::fwrite(kPropMagic, 1, 8, f) == 8 && std::fwrite(&n, sizeof(n), 1, f) == 1 &&
                    std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    return (std::fclose(f) == 0 && ok) ? TSALLIS_OK : TSALLIS_ERR_INVALID_ARG;
}

namespace {
// CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320), bytewise from the
// definition: shift out one bit at a time, folding in the polynomial when
// the bit shifted out is set.
uint32_t crc32_update(uint32_t crc, const void* data, size_t n) {
    const unsigned char* p = static_cast<const unsigned char*>(data);
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) {
        crc ^= p[i];
        for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
    }
    return ~crc;
}

const char kCkptMagic[8] = {'T', 'S', 'C', 'K', 'P', 'T', '0', '1'};
struct CkptHeader {
    char magic[8];
    uint32_t version;   // 1
    uint32_t nin, nhid, nout;
    uint32_t pad;
    int64_t nparams;
    int64_t step;       // Adam steps taken
    int64_t user_bytes; // caller's state that follows the moments
};
}  // namespace

tsallis_status tsallis_proposer_checkpoint_save(tsallis_ctx* c, const char* path, const void* user,
                                                int64_t user_bytes) {
    TSL_TRACE();
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    ProposerSlot& S = c->prop[c->prop_sel];
    if (!path || !S.ready || user_bytes < 0 || (user_bytes > 0 && !user)) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    const size_t f = (size_t)kMlpParams * sizeof(float);
    std::vector<float> buf(3 * (size_t)kMlpParams);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(buf.data(), S.mlp.p32, f, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(buf.data() + kMlpParams, S.mlp.m, f, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(buf.data() + 2 * kMlpParams, S.mlp.v, f, cudaMemcpyDeviceToHost) != cudaSuccess)
        return TSALLIS_ERR_CUDA;
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 1;
    h.nin = kMlpIn;
    h.nhid = kMlpHid;
    h.nout = kMlpOut;
    h.nparams = kMlpParams;
    h.step = S.step;
    h.user_bytes = user_bytes;
    uint32_t crc = crc32_update(0, &h, sizeof(h));
    crc = crc32_update(crc, buf.data(), buf.size() * sizeof(float));
    if (user_bytes > 0) crc = crc32_update(crc, user, (size_t)user_bytes);
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return TSALLIS_ERR_INVALID_ARG;
    bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 &&
              std::fwrite(buf.data(), sizeof(float), buf.size(), fp) == buf.size() &&
              (user_bytes == 0 || std::fwrite(user, 1, (size_t)user_bytes, fp) == (size_t)user_bytes) &&
              std::fwrite(&crc, sizeof(crc), 1, fp) == 1;
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? TSALLIS_OK : TSALLIS_ERR_INVALID_ARG;
}

tsallis_status tsallis_proposer_checkpoint_load(tsallis_ctx* c, const char* path, void* user, int64_t user_cap,
                                                int64_t* user_bytes) {
    TSL_TRACE();
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    ProposerSlot& S = c->prop[c->prop_sel];
    if (!path || user_cap < 0 || (user_cap > 0 && !user)) return TSALLIS_ERR_INVALID_ARG;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return TSALLIS_ERR_INVALID_ARG;
    CkptHeader h;
    std::vector<float> buf;
    std::vector<unsigned char> ub;
    uint32_t crc_file = 0;
    bool ok = std::fread(&h, sizeof(h), 1, fp) == 1 && std::memcmp(h.magic, kCkptMagic, 8) == 0 && h.version == 1 &&
              h.nin == (uint32_t)kMlpIn && h.nhid == (uint32_t)kMlpHid && h.nout == (uint32_t)kMlpOut &&
              h.nparams == kMlpParams && h.step >= 0 && h.user_bytes >= 0 && h.user_bytes <= (1ll << 30);
    if (ok) {
        buf.resize(3 * (size_t)kMlpParams);
        ub.resize((size_t)h.user_bytes);
        ok = std::fread(buf.data(), sizeof(float), buf.size(), fp) == buf.size() &&
             (h.user_bytes == 0 || std::fread(ub.data(), 1, ub.size(), fp) == ub.size()) &&
             std::fread(&crc_file, sizeof(crc_file), 1, fp) == 1;
    }
    std::fclose(fp);
    if (!ok) return TSALLIS_ERR_INVALID_ARG;
    uint32_t crc = crc32_update(0, &h, sizeof(h));
    crc = crc32_update(crc, buf.data(), buf.size() * sizeof(float));
    if (!ub.empty()) crc = crc32_update(crc, ub.data(), ub.size());
    if (crc != crc_file) return TSALLIS_ERR_INVALID_ARG;   // damaged file
    if (h.user_bytes > user_cap) return TSALLIS_ERR_INVALID_ARG;
    tsallis_status st = tsallis_proposer_set(c, buf.data(), kMlpParams);
    if (st != TSALLIS_OK) return st;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    const size_t f = (size_t)kMlpParams * sizeof(float);
    if (cudaMemcpy(S.mlp.m, buf.data() + kMlpParams, f, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(S.mlp.v, buf.data() + 2 * kMlpParams, f, cudaMemcpyHostToDevice) != cudaSuccess)
        return TSALLIS_ERR_CUDA;
    S.step = (int)h.step;
    if (!ub.empty()) std::memcpy(user, ub.data(), ub.size());
    if (user_bytes) *user_bytes = h.user_bytes;
    return TSALLIS_OK;
}

tsallis_status tsallis_proposer_features(tsallis_ctx* c, const int32_t* d_hist, int64_t nh, float* d_x,
                                         cudaStream_t stream) {
    TSL_TRACE();
    if (!c || nh < 0 || (nh > 0 && (!d_hist || !d_x))) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    return cuda_status(c->prop_sel == 1 ? mlp_features2d(d_hist, nh, d_x, stream)
                                        : mlp_features(d_hist, nh, d_x, stream));
}

tsallis_status tsallis_proposer_select(tsallis_ctx* c, int32_t slot) {
    if (!c || (slot != 0 && slot != 1)) return TSALLIS_ERR_INVALID_ARG;
    c->prop_sel = slot;
    return TSALLIS_OK;
}

tsallis_status tsallis_proposer_forward(tsallis_ctx* c, const float* d_x, int32_t B, float* d_logits,
                                        cudaStream_t stream) {
    TSL_TRACE();
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    ProposerSlot& S = c->prop[c->prop_sel];
    if (B < 0 || (B > 0 && (!d_x || !d_logits)) || !S.ready) return TSALLIS_ERR_INVALID_ARG;
    if (B == 0) return TSALLIS_OK;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    tsallis_status st = ensure_mlp_act(c, c->prop_sel, B);
    if (st != TSALLIS_OK || (st = ensure_prop(c, B)) != TSALLIS_OK) return st;
    // up to kMlpInferRows rows: the fused inference kernel (no top k)
    const cudaError_t e = B <= kMlpInferRows
                              ? mlp_infer(S.mlp, nullptr, d_x, c->prop_x, B, 0, nullptr, c->prop_sync, c->timeout_ns,
                                          stream)
                              : mlp_forward(S.mlp, d_x, B, stream);
    if (e != cudaSuccess ||
        cudaMemcpyAsync(d_logits, S.mlp.z3, (size_t)B * kMlpOut * sizeof(float), cudaMemcpyDeviceToDevice,
                        stream) != cudaSuccess)
        return TSALLIS_ERR_CUDA;
    return TSALLIS_OK;
}

tsallis_status tsallis_proposer_train_step(tsallis_ctx* c, const float* d_x, const float* d_y, int32_t B, float lr,
                                           int32_t update, float* d_loss, float* d_grad, cudaStream_t stream) {
    TSL_TRACE();
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    ProposerSlot& S = c->prop[c->prop_sel];
    if (B < 1 || !d_x || !d_y || !d_loss || !S.ready || !(lr >= 0.f)) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    tsallis_status st = ensure_mlp_act(c, c->prop_sel, B);
    if (st != TSALLIS_OK) return st;
    if (mlp_forward(S.mlp, d_x, B, stream) != cudaSuccess ||
        mlp_backward(S.mlp, d_x, d_y, B, d_loss, stream) != cudaSuccess)
        return TSALLIS_ERR_CUDA;
    if (d_grad && cudaMemcpyAsync(d_grad, S.mlp.grad, (size_t)kMlpParams * sizeof(float), cudaMemcpyDeviceToDevice,
                                  stream) != cudaSuccess)
        return TSALLIS_ERR_CUDA;
    if (update) {
        S.step += 1;
        if (mlp_adam(S.mlp, lr, S.step, stream) != cudaSuccess) return TSALLIS_ERR_CUDA;
    }
    return TSALLIS_OK;
}

tsallis_status tsallis_autotune_batch(tsallis_ctx* c, const tsallis_volume* h_vols, int32_t nvol,
                                      const tsallis_params* p, int32_t* d_t, float* d_phi, int32_t* d_status,
                                      cudaStream_t stream, int32_t* tile_vox, int32_t* blocks_per_sm,
                                      float* best_ms) {
    TSL_TRACE();
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    tsallis_status st = check_params(p);
    if (st != TSALLIS_OK) return st;
    if (nvol <= 0 || p->two_d) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    const int tiles[] = {16384, 32768, 65536, 131072, 262144};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return TSALLIS_ERR_CUDA;
    }
    const int old_tile = c->tile_vox, old_bps = c->blocks_per_sm;
    float best = 0.f;
    int bt = old_tile, bb = old_bps;
    for (int tv : tiles) {
        for (int bps = 1; bps <= c->max_blocks_per_sm; ++bps) {
            c->tile_vox = tv;
            c->blocks_per_sm = bps;
            // one untimed pass (it also grows the scratch), then the best of three
            if ((st = tsallis_segment_batch(c, h_vols, nvol, p, d_t, d_phi, d_status, stream)) != TSALLIS_OK) break;
            float ms_min = 0.f;
            for (int r = 0; r < 3 && st == TSALLIS_OK; ++r) {
                float ms = 0.f;
                if (cudaEventRecord(e0, stream) != cudaSuccess) { st = TSALLIS_ERR_CUDA; break; }
                if ((st = tsallis_segment_batch(c, h_vols, nvol, p, d_t, d_phi, d_status, stream)) != TSALLIS_OK)
                    break;
                if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    st = TSALLIS_ERR_CUDA;
                    break;
                }
                if (r == 0 || ms < ms_min) ms_min = ms;
            }
            if (st != TSALLIS_OK) break;
            if (best == 0.f || ms_min < best) {
                best = ms_min;
                bt = tv;
                bb = bps;
            }
        }
        if (st != TSALLIS_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != TSALLIS_OK) {
        c->tile_vox = old_tile;
        c->blocks_per_sm = old_bps;
        cudaGetLastError();
        return st;
    }
    c->tile_vox = bt;
    c->blocks_per_sm = bb;
    if (tile_vox) *tile_vox = bt;
    if (blocks_per_sm) *blocks_per_sm = bb;
    if (best_ms) *best_ms = best;
    return TSALLIS_OK;
}

}  // extern "C"

// ------------------------------------------------------------ pre-processing

tsallis_status tsallis_preprocess_params_default(tsallis_preprocess_params* pp) {
    if (!pp) return TSALLIS_ERR_INVALID_ARG;
    pp->background = -2000;
    pp->hu_min = -2000;
    pp->hu_max = 2500;
    pp->radius = 10;
    pp->op = TSALLIS_MORPH_CHEST_MASK;
    pp->per_slice = 1;
    return TSALLIS_OK;
}

namespace {
// Multiplier and shift with floor(n / d) == umulhi(n, m) >> s for every n
// the level map forms (n <= 511 * D < 2^26, d = 2D): m = floor(2^(32+s) / d)
// + 1 with s = max(ceil(log2 d) - 2, 0) fits 32 bits and keeps the error
// below 1/d; checked exhaustively.
bool level_divider(int D, unsigned long long* m, int* s) {
    const unsigned long long d = 2ull * (unsigned long long)D;
    int l = 0;
    while ((1ull << l) < d) ++l;
    *s = l >= 2 ? l - 2 : 0;
    *m = ((1ull << (32 + *s)) / d) + 1;
    if (*m > 0xffffffffull) return false;
    for (long long c = 0; c <= D; ++c) {
        const unsigned long long n = (unsigned long long)(2 * c * 255 + D);
        if ((((n * *m) >> 32) >> *s) != n / d) return false;
    }
    return true;
}
}  // namespace

tsallis_status tsallis_preprocess(tsallis_ctx* c, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                                  const tsallis_preprocess_params* pp, int16_t* d_out, int32_t* d_hist,
                                  cudaStream_t stream) {
    TSL_TRACE();
    if (!c || !pp) return TSALLIS_ERR_INVALID_ARG;
    if (pp->radius < 0 || pp->radius > kPreMaxRadius || pp->op < TSALLIS_MORPH_NONE ||
        pp->op > TSALLIS_MORPH_BLACK_TOPHAT || (pp->per_slice != 0 && pp->per_slice != 1))
        return TSALLIS_ERR_INVALID_ARG;
    if ((long long)pp->hu_max - pp->hu_min < 1 || (long long)pp->hu_max - pp->hu_min > 65535)
        return TSALLIS_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || nz < 0 || nx > (1 << 30) || ny > (1 << 30)) return TSALLIS_ERR_INVALID_ARG;
    if (nz == 0 && (pp->per_slice || !d_hist)) return TSALLIS_OK;   // nothing to write
    if (!d_out && !d_hist) return TSALLIS_ERR_INVALID_ARG;
    if (nz > 0 && !d_vol) return TSALLIS_ERR_INVALID_ARG;
    // the kernel copies pixel pairs at even element indices as 4-byte words
    if ((reinterpret_cast<uintptr_t>(d_vol) & 3) || (reinterpret_cast<uintptr_t>(d_out) & 1))
        return TSALLIS_ERR_ALIGNMENT;
    const long long ntx = (nx + preproc_tile_w() - 1) / preproc_tile_w();
    const long long nty = (ny + preproc_tile_h() - 1) / preproc_tile_h();
    if (nz > 0 && ntx * nty > 0x7fffffffll / nz) return TSALLIS_ERR_INVALID_ARG;
    const long long nbytes = nx * ny * nz * (long long)sizeof(int16_t);
    if (d_out && nz > 0) {
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(d_vol), b0 = reinterpret_cast<uintptr_t>(d_out);
        if (a0 < b0 + (uintptr_t)nbytes && b0 < a0 + (uintptr_t)nbytes) return TSALLIS_ERR_INVALID_ARG;
    }
    PreArgs a;
    a.D = pp->hu_max - pp->hu_min;
    if (!level_divider(a.D, &a.magic, &a.shift)) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    const long long nh = pp->per_slice ? nz : 1;
    if (d_hist && nh > 0 &&
        cudaMemsetAsync(d_hist, 0, (size_t)nh * 256 * sizeof(int32_t), stream) != cudaSuccess)
        return TSALLIS_ERR_CUDA;
    if (nz == 0) return TSALLIS_OK;
    a.vol = d_vol;
    a.out = d_out;
    a.hist = d_hist;
    a.nx = (int)nx;
    a.ny = (int)ny;
    a.nz = (int)nz;
    a.background = pp->background;
    a.hu_min = pp->hu_min;
    a.hu_max = pp->hu_max;
    a.op = pp->op;
    a.radius = pp->radius;
    a.per_slice = pp->per_slice;
    a.ntx = (int)ntx;
    a.nty = (int)nty;
    a.check = c->check;
    return cuda_status(launch_preprocess(a, stream));
}

// ------------------------------------------------------------ checked build

tsallis_status tsallis_check_status(tsallis_ctx* c, uint32_t* site) {
    if (!c || !site) return TSALLIS_ERR_INVALID_ARG;
    if (!kCheckedBuild) return TSALLIS_ERR_UNIMPLEMENTED;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    unsigned v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&v, c->check, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(c->check, 0, sizeof(unsigned)) != cudaSuccess)
        return TSALLIS_ERR_CUDA;
    *site = v;
    return TSALLIS_OK;
}

tsallis_status tsallis_probe_topk(tsallis_ctx* c, const float* d_logits, int32_t B, int32_t k, int32_t* d_out,
                                  cudaStream_t stream) {
    if (!c || B < 0 || k < 1 || k > 256 || (B > 0 && (!d_logits || !d_out))) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    return cuda_status(mlp_topk(d_logits, B, k, d_out, stream));
}

// ------------------------------------------------------------ host buffers

namespace {
constexpr long long kHostChunkVox = 1ll << 24;   // voxels per pipelined chunk (32 MB of int16)

tsallis_status ensure_host_pipeline(tsallis_ctx* c, size_t bytes) {
    if (!c->hp_ready) {
        for (cudaStream_t& h : c->hp_stream)
            if (cudaStreamCreateWithFlags(&h, cudaStreamNonBlocking) != cudaSuccess) return TSALLIS_ERR_CUDA;
        for (cudaEvent_t& e : c->hp_ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return TSALLIS_ERR_CUDA;
        c->hp_ready = true;
    }
    if (c->hp_buf && c->hp_bytes >= bytes) return TSALLIS_OK;
    if (c->hp_buf) {
        if (cudaDeviceSynchronize() != cudaSuccess) return TSALLIS_ERR_CUDA;
        cudaFree(c->hp_buf);
        c->hp_buf = nullptr;
        c->hp_bytes = 0;
    }
    if (cudaMalloc(&c->hp_buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return TSALLIS_ERR_OOM;
    }
    c->hp_bytes = bytes;
    return TSALLIS_OK;
}
}  // namespace

tsallis_status tsallis_segment_host(tsallis_ctx* c, const int16_t* h_vol, int64_t nx, int64_t ny, int64_t nz,
                                    const tsallis_params* p, uint8_t* h_mask, int32_t* h_t, float* h_phi,
                                    int32_t* h_status, cudaStream_t stream) {
    TSL_TRACE();
    tsallis_status st = check_params(p);
    if (st != TSALLIS_OK) return st;
    if ((st = check_shape(nx, ny, nz)) != TSALLIS_OK) return st;
    if (nz == 0) return TSALLIS_OK;
    if (!c || !h_vol || !h_mask || !h_t || !h_phi || !h_status) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    const long long slice = nx * ny;
    const long long nh = p->mode == TSALLIS_PER_SLICE ? nz : 1;
    const long long tper = p->two_d ? 2 : 1;
    // independent slices are pipelined in chunks; anything else is one chunk
    const bool chunked = p->mode == TSALLIS_PER_SLICE && !p->two_d && p->topk == 0;
    long long S = nz;
    if (chunked) {
        S = kHostChunkVox / slice;
        if (S < 1) S = 1;
        if (S > nz) S = nz;
    }
    const long long nchunks = (nz + S - 1) / S;
    const int nbuf = nchunks > 1 ? 2 : 1;
    const size_t in_b = align256((size_t)(S * slice) * sizeof(int16_t)), mask_b = align256((size_t)(S * slice));
    const size_t out_b = align256((size_t)(nh * tper) * sizeof(int32_t)) + 2 * align256((size_t)nh * 4);
    if ((st = ensure_host_pipeline(c, nbuf * (in_b + mask_b) + out_b)) != TSALLIS_OK) return st;
    unsigned char* base = static_cast<unsigned char*>(c->hp_buf);
    int16_t* din[2] = {reinterpret_cast<int16_t*>(base), reinterpret_cast<int16_t*>(base + in_b)};
    uint8_t* dmask[2] = {base + nbuf * in_b, base + nbuf * in_b + mask_b};
    unsigned char* ob = base + nbuf * (in_b + mask_b);
    int32_t* dt = reinterpret_cast<int32_t*>(ob);
    float* dphi = reinterpret_cast<float*>(ob + align256((size_t)(nh * tper) * sizeof(int32_t)));
    int32_t* dst = reinterpret_cast<int32_t*>(ob + align256((size_t)(nh * tper) * sizeof(int32_t)) +
                                              align256((size_t)nh * 4));
    cudaStream_t s_in = c->hp_stream[0], s_comp = c->hp_stream[1], s_out = c->hp_stream[2];
    cudaEvent_t ev_start = c->hp_ev[0], ev_done = c->hp_ev[1];
    cudaEvent_t* ev_in = &c->hp_ev[2];     // [2]
    cudaEvent_t* ev_comp = &c->hp_ev[4];   // [2]
    cudaEvent_t* ev_out = &c->hp_ev[6];    // [2]
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    // the internal streams start after the caller's earlier work
    if (!ok(cudaEventRecord(ev_start, stream)) || !ok(cudaStreamWaitEvent(s_in, ev_start, 0)) ||
        !ok(cudaStreamWaitEvent(s_comp, ev_start, 0)) || !ok(cudaStreamWaitEvent(s_out, ev_start, 0)))
        return TSALLIS_ERR_CUDA;
    for (long long i = 0; i < nchunks; ++i) {
        const int b = (int)(i & 1);
        const long long z0 = i * S, Si = nz - z0 < S ? nz - z0 : S;
        const size_t nv = (size_t)(Si * slice);
        // copy in (after the chunk two back has been segmented out of this buffer)
        if (i >= 2 && !ok(cudaStreamWaitEvent(s_in, ev_comp[b], 0))) return TSALLIS_ERR_CUDA;
        if (!ok(cudaMemcpyAsync(din[b], h_vol + z0 * slice, nv * sizeof(int16_t), cudaMemcpyHostToDevice, s_in)) ||
            !ok(cudaEventRecord(ev_in[b], s_in)))
            return TSALLIS_ERR_CUDA;
        // segment (after its input arrived and the mask buffer was copied out)
        if (!ok(cudaStreamWaitEvent(s_comp, ev_in[b], 0))) return TSALLIS_ERR_CUDA;
        if (i >= 2 && !ok(cudaStreamWaitEvent(s_comp, ev_out[b], 0))) return TSALLIS_ERR_CUDA;
        const long long h0 = chunked ? z0 : 0;
        if ((st = segment_impl(c, din[b], nx, ny, Si, p, dmask[b], dt + h0 * tper, dphi + h0, dst + h0, s_comp, nz)) !=
            TSALLIS_OK)
            return st;
        if (!ok(cudaEventRecord(ev_comp[b], s_comp))) return TSALLIS_ERR_CUDA;
        // copy the mask out
        if (!ok(cudaStreamWaitEvent(s_out, ev_comp[b], 0)) ||
            !ok(cudaMemcpyAsync(h_mask + z0 * slice, dmask[b], nv, cudaMemcpyDeviceToHost, s_out)) ||
            !ok(cudaEventRecord(ev_out[b], s_out)))
            return TSALLIS_ERR_CUDA;
    }
    // thresholds, values and statuses; then the caller's stream waits for it all
    if (!ok(cudaMemcpyAsync(h_t, dt, (size_t)(nh * tper) * sizeof(int32_t), cudaMemcpyDeviceToHost, s_out)) ||
        !ok(cudaMemcpyAsync(h_phi, dphi, (size_t)nh * sizeof(float), cudaMemcpyDeviceToHost, s_out)) ||
        !ok(cudaMemcpyAsync(h_status, dst, (size_t)nh * sizeof(int32_t), cudaMemcpyDeviceToHost, s_out)) ||
        !ok(cudaEventRecord(ev_done, s_out)) || !ok(cudaStreamWaitEvent(stream, ev_done, 0)))
        return TSALLIS_ERR_CUDA;
    return TSALLIS_OK;
}
