// C ABI of the thresholding path (declared in include/tsallis.h): argument
// checks, the context's scratch memory, and dispatch to the kernels.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/tsallis.h"
#include "kernels.h"

using namespace tsl;

struct tsallis_ctx {
    int device = 0;
    int sm_count = 0;
    long long l2_bytes = 0;
    void* scratch = nullptr;      // ScratchHeader, then per-group arrays
    size_t scratch_bytes = 0;
    long long cap_groups = 0;
    unsigned long long timeout_ns = 1000000000ull;
    // launch shape of the 1-D persistent kernel
    int copies = 1;
    int tile_vox = 32768;
    int blocks_per_sm = 0;
    // batch work list (device copy) and its host image
    void* batch_buf = nullptr;
    size_t batch_bytes = 0;
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
    if (!(p->q > 0.0f) || !std::isfinite(p->q)) return TSALLIS_ERR_INVALID_ARG;
    if (p->nbins < 2 || p->nbins > kMaxLevels) return TSALLIS_ERR_INVALID_ARG;
    if (p->lo < -65536 || p->lo > 65535) return TSALLIS_ERR_INVALID_ARG;
    if (p->mode != TSALLIS_PER_SLICE && p->mode != TSALLIS_WHOLE_VOLUME) return TSALLIS_ERR_INVALID_ARG;
    if (p->polarity != TSALLIS_MASK_LOW && p->polarity != TSALLIS_MASK_HIGH) return TSALLIS_ERR_INVALID_ARG;
    if (p->two_d != 0 && p->two_d != 1) return TSALLIS_ERR_INVALID_ARG;
    if (p->two_d) {
        if (p->shift < 0 || p->shift > 15) return TSALLIS_ERR_INVALID_ARG;
        int L2 = p->nbins >> p->shift;
        if (L2 < 2 || L2 > 256) return TSALLIS_ERR_INVALID_ARG;
    }
    if (p->topk < 0) return TSALLIS_ERR_INVALID_ARG;
    if (p->flags & ~TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL) return TSALLIS_ERR_INVALID_ARG;
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

// Grows the context's scratch so it holds at least ngroups groups. The
// layout depends only on the capacity (arrive[cap], ready[cap], tmo[cap], then
// ghist[cap][kMaxLevels]), so state left by one launch lines up with the next.
// New memory is zeroed; the kernels keep it zeroed between launches.
size_t scratch_layout(long long cap, size_t* ghist_off) {
    size_t off = sizeof(ScratchHeader) + (size_t)cap * 3 * sizeof(int);
    off = (off + 255) & ~size_t(255);
    if (ghist_off) *ghist_off = off;
    return off + (size_t)cap * kMaxLevels * sizeof(int);
}

tsallis_status ensure_scratch(tsallis_ctx* c, long long ngroups) {
    if (c->scratch && ngroups <= c->cap_groups) return TSALLIS_OK;
    long long cap = c->cap_groups > 0 ? c->cap_groups : 16;
    while (cap < ngroups) cap *= 2;
    if (c->scratch) {
        if (cudaDeviceSynchronize() != cudaSuccess) return TSALLIS_ERR_CUDA;
        cudaFree(c->scratch);
        c->scratch = nullptr;
        c->scratch_bytes = 0;
        c->cap_groups = 0;
    }
    const size_t bytes = scratch_layout(cap, nullptr);
    if (cudaMalloc(&c->scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        return TSALLIS_ERR_OOM;
    }
    if (cudaMemset(c->scratch, 0, bytes) != cudaSuccess) return TSALLIS_ERR_CUDA;
    c->scratch_bytes = bytes;
    c->cap_groups = cap;
    return TSALLIS_OK;
}

struct ScratchView {
    ScratchHeader* hdr;
    int* arrive;
    int* ready;
    int* tmo;
    int* ghist;
};

ScratchView view(tsallis_ctx* c) {
    char* b = (char*)c->scratch;
    size_t goff = 0;
    scratch_layout(c->cap_groups, &goff);
    ScratchView v;
    v.hdr = (ScratchHeader*)b;
    v.arrive = (int*)(b + sizeof(ScratchHeader));
    v.ready = v.arrive + c->cap_groups;
    v.tmo = v.ready + c->cap_groups;
    v.ghist = (int*)(b + goff);
    return v;
}

int grid_for(tsallis_ctx* c, unsigned nticket) {
    long long g = (long long)c->sm_count * (c->blocks_per_sm > 0 ? c->blocks_per_sm : 1);
    if ((long long)nticket < g) g = nticket;
    return (int)(g < 1 ? 1 : g);
}

void fill_common(SegArgs& a, const tsallis_params* p, tsallis_ctx* c) {
    std::memset(&a, 0, sizeof(a));
    a.lo = p->lo;
    a.L = p->nbins;
    a.q = p->q;
    a.polarity = p->polarity;
    a.bin_shift = 0;
    a.flags = p->flags;
    a.timeout_ns = c->timeout_ns;
    a.tile_vox = c->tile_vox;
}

tsallis_status cuda_status(cudaError_t e) { return e == cudaSuccess ? TSALLIS_OK : TSALLIS_ERR_CUDA; }

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
    if (segment1d_occupancy(c->copies, kMaxLevels, &c->blocks_per_sm) != cudaSuccess || c->blocks_per_sm < 1) {
        delete c;
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
    }
    delete c;
}

tsallis_status tsallis_set_wait_timeout(tsallis_ctx* c, uint64_t ns) {
    if (!c || ns == 0) return TSALLIS_ERR_INVALID_ARG;
    c->timeout_ns = ns;
    return TSALLIS_OK;
}

tsallis_status tsallis_histogram(tsallis_ctx* c, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                                 const tsallis_params* p, int32_t* d_hist, cudaStream_t stream) {
    tsallis_status st = check_params(p);
    if (st != TSALLIS_OK) return st;
    if ((st = check_shape(nx, ny, nz)) != TSALLIS_OK) return st;
    if (nz == 0) return TSALLIS_OK;
    if (!d_vol || !d_hist) return TSALLIS_ERR_INVALID_ARG;
    if (!aligned16(d_vol)) return TSALLIS_ERR_ALIGNMENT;
    if (p->two_d) return TSALLIS_ERR_UNIMPLEMENTED;
    const long long slice = nx * ny;
    const long long gvox = p->mode == TSALLIS_PER_SLICE ? slice : slice * nz;
    const long long ng = p->mode == TSALLIS_PER_SLICE ? nz : 1;
    if (gvox > (1ll << 31) - 1) return TSALLIS_ERR_INVALID_ARG;
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    if ((st = ensure_scratch(c, 0)) != TSALLIS_OK) return st;
    if (cudaMemsetAsync(d_hist, 0, (size_t)ng * p->nbins * sizeof(int32_t), stream) != cudaSuccess)
        return TSALLIS_ERR_CUDA;
    SegArgs a;
    fill_common(a, p, c);
    a.vol = d_vol;
    a.group_vox = gvox;
    a.ngroups = (int)ng;
    a.ntiles = (int)((gvox + a.tile_vox - 1) / a.tile_vox);
    a.phases = kPhaseHist;
    a.nticket = (unsigned)(ng * a.ntiles);
    ScratchView v = view(c);
    a.hdr = v.hdr;
    a.ghist = d_hist;
    return cuda_status(launch_segment1d(a, grid_for(c, a.nticket), c->copies, stream));
}

tsallis_status tsallis_search(tsallis_ctx* c, const int32_t* d_hist, int64_t nh, const tsallis_params* p,
                              int32_t* d_t, float* d_phi, int32_t* d_status, float* d_curve, cudaStream_t stream) {
    tsallis_status st = check_params(p);
    if (st != TSALLIS_OK) return st;
    if (nh < 0 || nh > (1ll << 31) - 1) return TSALLIS_ERR_INVALID_ARG;
    if (nh == 0) return TSALLIS_OK;
    if (!d_hist || !d_t || !d_phi || !d_status) return TSALLIS_ERR_INVALID_ARG;
    if (p->two_d) return TSALLIS_ERR_UNIMPLEMENTED;
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    return cuda_status(launch_search1d(d_hist, nh, p->nbins, p->q, d_t, d_phi, d_status, d_curve, stream));
}

tsallis_status tsallis_binarize(tsallis_ctx* c, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                                const int32_t* d_t, const tsallis_params* p, uint8_t* d_mask, cudaStream_t stream) {
    tsallis_status st = check_params(p);
    if (st != TSALLIS_OK) return st;
    if ((st = check_shape(nx, ny, nz)) != TSALLIS_OK) return st;
    if (nz == 0) return TSALLIS_OK;
    if (!d_vol || !d_mask || !d_t) return TSALLIS_ERR_INVALID_ARG;
    if (!aligned16(d_vol) || !aligned16(d_mask)) return TSALLIS_ERR_ALIGNMENT;
    if (p->two_d) return TSALLIS_ERR_UNIMPLEMENTED;
    const long long slice = nx * ny;
    const long long gvox = p->mode == TSALLIS_PER_SLICE ? slice : slice * nz;
    const long long ng = p->mode == TSALLIS_PER_SLICE ? nz : 1;
    if (gvox > (1ll << 31) - 1) return TSALLIS_ERR_INVALID_ARG;
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    if ((st = ensure_scratch(c, 0)) != TSALLIS_OK) return st;
    SegArgs a;
    fill_common(a, p, c);
    a.vol = d_vol;
    a.mask = d_mask;
    a.group_vox = gvox;
    a.ngroups = (int)ng;
    a.ntiles = (int)((gvox + a.tile_vox - 1) / a.tile_vox);
    a.phases = kPhaseBin;
    a.nticket = (unsigned)(ng * a.ntiles);
    a.t_in = d_t;
    ScratchView v = view(c);
    a.hdr = v.hdr;
    return cuda_status(launch_segment1d(a, grid_for(c, a.nticket), c->copies, stream));
}

tsallis_status tsallis_segment(tsallis_ctx* c, const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                               const tsallis_params* p, uint8_t* d_mask, int32_t* d_t, float* d_phi,
                               int32_t* d_status, cudaStream_t stream) {
    tsallis_status st = check_params(p);
    if (st != TSALLIS_OK) return st;
    if ((st = check_shape(nx, ny, nz)) != TSALLIS_OK) return st;
    if (nz == 0) return TSALLIS_OK;
    if (!d_vol || !d_mask || !d_t || !d_phi || !d_status) return TSALLIS_ERR_INVALID_ARG;
    if (!aligned16(d_vol) || !aligned16(d_mask)) return TSALLIS_ERR_ALIGNMENT;
    if (p->two_d) return TSALLIS_ERR_UNIMPLEMENTED;
    const long long slice = nx * ny;
    const long long gvox = p->mode == TSALLIS_PER_SLICE ? slice : slice * nz;
    const long long ng = p->mode == TSALLIS_PER_SLICE ? nz : 1;
    if (gvox > (1ll << 31) - 1) return TSALLIS_ERR_INVALID_ARG;
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok()) return TSALLIS_ERR_CUDA;
    if ((st = ensure_scratch(c, ng)) != TSALLIS_OK) return st;
    SegArgs a;
    fill_common(a, p, c);
    a.vol = d_vol;
    a.mask = d_mask;
    a.group_vox = gvox;
    a.ngroups = (int)ng;
    a.ntiles = (int)((gvox + a.tile_vox - 1) / a.tile_vox);
    a.phases = kPhaseHist | kPhaseSearch | kPhaseBin;
    const int grid0 = grid_for(c, 0xffffffffu);
    // binarise items trail histogram items by enough steps to cover the
    // items in flight, so their waits are normally already satisfied
    const int steps_in_flight = (grid0 + 2 * a.ntiles - 1) / (2 * a.ntiles);
    a.lag = ng == 1 ? 1 : steps_in_flight + 4;
    const long long nt = (ng + a.lag) * 2ll * a.ntiles;
    if (nt > 0xffffffffll) return TSALLIS_ERR_INVALID_ARG;
    a.nticket = (unsigned)nt;
    ScratchView v = view(c);
    a.hdr = v.hdr;
    a.arrive = v.arrive;
    a.ready = v.ready;
    a.tmo = v.tmo;
    a.ghist = v.ghist;
    a.t_out = d_t;
    a.phi_out = d_phi;
    a.status = d_status;
    return cuda_status(launch_segment1d(a, grid_for(c, a.nticket), c->copies, stream));
}

tsallis_status tsallis_segment_batch(tsallis_ctx* c, const tsallis_volume* h_vols, int32_t nvol,
                                     const tsallis_params* p, int32_t* d_t, float* d_phi, int32_t* d_status,
                                     cudaStream_t stream) {
    (void)h_vols; (void)nvol; (void)d_t; (void)d_phi; (void)d_status; (void)stream;
    if (!c) return TSALLIS_ERR_INVALID_ARG;
    tsallis_status st = check_params(p);
    if (st != TSALLIS_OK) return st;
    return TSALLIS_ERR_UNIMPLEMENTED;
}

}  // extern "C"
