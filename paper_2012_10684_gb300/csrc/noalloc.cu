// tsallis_segment_static: the fused 1-D segmentation for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc at all: code running under a memory
// manager that owns every device allocation (a pool handed out by a host
// framework, a real-time pipeline that pre-allocates everything at start-up
// and forbids allocation afterwards), or code that must not trigger the
// implicit synchronisation a cudaMalloc/cudaFree can cause. tsallis_segment
// needs a context, and creating one allocates scratch and tables. This entry
// point instead keeps all of its scratch in one file-scope __device__ array
// of fixed size, so it allocates nothing; the caller only passes its own
// input and output buffers.
//
// The array lives in every GPU that loads the library, for the life of the
// process. Its layout (sizes fixed at build time):
//   ScratchHeader | arrive, done_flag, bdone [kMaxGroups] | predicted
//   thresholds [kMaxGroups] | ghist
//   [kMaxGroups][4096] | binarise queue [kMaxTiles] | double-float tables |
//   two-entry log2 table.
// The kernel leaves every counter and histogram zeroed when it finishes
// (also after a timed-out wait), and queue entries carry the launch number,
// so the array needs clearing only once, at set-up.
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/tsallis.h"
#include "kernels.h"

namespace {

using namespace tsl;

constexpr long long kMaxGroups = 512;              // histograms per call
constexpr long long kMaxTiles = 16384;             // work tiles per call
constexpr int kStaticTileVox = 65536;              // voxels per tile
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffArrive = sizeof(ScratchHeader);
constexpr size_t kOffThat = kOffArrive + 3 * kMaxGroups * sizeof(int);
constexpr size_t kOffGhist = align256(kOffThat + kMaxGroups * sizeof(unsigned long long));
constexpr size_t kOffQueue = align256(kOffGhist + (size_t)kMaxGroups * kMaxLevels * sizeof(int));
constexpr size_t kOffTables = align256(kOffQueue + (size_t)kMaxTiles * sizeof(unsigned long long));
constexpr size_t kTablesBytes = 4096;              // room for the double-float tables
constexpr size_t kOffLog2 = align256(kOffTables + kTablesBytes);
constexpr size_t kStaticBytes = align256(kOffLog2 + 2 * 2 * sizeof(float));   // about 8.2 MB

// The scratch. In host code this name is only a stand-in for the device
// symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

struct DeviceState {
    bool ready = false;
    unsigned char* base = nullptr;   // device address of g_static_scratch
    int sm_count = 0;
    int blocks_per_sm = 0;
};

std::mutex g_mu;
DeviceState g_dev[kMaxDevices];

// Set-up for the current device: runs once per device, on its first call.
// Looks up the array's device address, clears it, writes the tables, and
// opts the kernel into its shared memory. Synchronous, no allocation.
tsallis_status setup(int dev, DeviceState& ds) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return TSALLIS_ERR_CUDA;
    }
    unsigned char* base = static_cast<unsigned char*>(p);
    if (df_tables_bytes() > kTablesBytes) return TSALLIS_ERR_CUDA;
    std::vector<unsigned char> tab(df_tables_bytes());
    const float log2_small[4] = {0.f, 0.f, 0.f, 0.f};   // log2(0) := 0, log2(1) = 0
    df_tables_fill(tab.data(), base + kOffLog2, 1);
    int sms = 0, bps = 0;
    if (cudaMemset(base, 0, kStaticBytes) != cudaSuccess ||
        cudaMemcpy(base + kOffTables, tab.data(), tab.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(base + kOffLog2, log2_small, sizeof(log2_small), cudaMemcpyHostToDevice) != cudaSuccess ||
        segment1d_prepare() != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        segment1d_occupancy(1, kMaxLevels, &bps) != cudaSuccess || bps < 1 ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return TSALLIS_ERR_CUDA;
    }
    ds.base = base;
    ds.sm_count = sms;
    ds.blocks_per_sm = bps;
    ds.ready = true;
    return TSALLIS_OK;
}

}  // namespace

extern "C" tsallis_status tsallis_segment_static(const int16_t* d_vol, int64_t nx, int64_t ny, int64_t nz,
                                                 const tsallis_params* p, uint8_t* d_mask, int32_t* d_t,
                                                 float* d_phi, int32_t* d_status, cudaStream_t stream) {
    // arguments, the same rules as tsallis_segment
    if (!p || !(p->q > 0.0f) || !(p->q <= 4.0f) || p->nbins < 2 || p->nbins > kMaxLevels ||
        p->lo < -32768 || p->lo > 32767 || (p->mode != TSALLIS_PER_SLICE && p->mode != TSALLIS_WHOLE_VOLUME) ||
        (p->polarity != TSALLIS_MASK_LOW && p->polarity != TSALLIS_MASK_HIGH) || p->two_d != 0 || p->topk != 0 ||
        (p->flags & ~TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL))
        return TSALLIS_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || nz < 0 || nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20)) return TSALLIS_ERR_INVALID_ARG;
    if (nz == 0) return TSALLIS_OK;
    if (!d_vol || !d_mask || !d_t || !d_phi || !d_status) return TSALLIS_ERR_INVALID_ARG;
    if (((uintptr_t)d_vol & 15u) || ((uintptr_t)d_mask & 15u)) return TSALLIS_ERR_ALIGNMENT;
    const long long slice = nx * ny;
    if (slice > (1ll << 31) - 1 || (p->mode == TSALLIS_WHOLE_VOLUME && slice * nz > (1ll << 31) - 1))
        return TSALLIS_ERR_INVALID_ARG;
    const long long gvox = p->mode == TSALLIS_PER_SLICE ? slice : slice * nz;
    const long long ng = p->mode == TSALLIS_PER_SLICE ? nz : 1;
    const long long ntiles = (gvox + kStaticTileVox - 1) / kStaticTileVox;
    // sizes beyond the fixed scratch
    if (ng > kMaxGroups || ng * ntiles > kMaxTiles) return TSALLIS_ERR_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return TSALLIS_ERR_CUDA;
    }
    DeviceState ds;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_dev[dev].ready) {
            const tsallis_status st = setup(dev, g_dev[dev]);
            if (st != TSALLIS_OK) return st;
        }
        ds = g_dev[dev];
    }

    SegArgs a;
    std::memset(&a, 0, sizeof(a));
    a.vol = d_vol;
    a.mask = d_mask;
    a.group_vox = gvox;
    a.ngroups = (int)ng;
    a.ntiles = (int)ntiles;
    a.tile_vox = kStaticTileVox;
    a.ntotal = (unsigned)(ng * ntiles);
    a.lo = p->lo;
    a.L = p->nbins;
    a.q = p->q;
    a.polarity = p->polarity;
    a.bin_shift = 0;
    a.t_stride = 1;
    a.phases = kPhaseHist | kPhaseSearch | kPhaseBin;
    a.flags = p->flags;
    a.timeout_ns = 1000000000ull;
    a.hdr = reinterpret_cast<ScratchHeader*>(ds.base);
    int* arrive = reinterpret_cast<int*>(ds.base + kOffArrive);
    a.arrive = arrive;
    a.done_flag = arrive + kMaxGroups;
    a.bdone = arrive + 2 * kMaxGroups;
    a.that = reinterpret_cast<unsigned long long*>(ds.base + kOffThat);
    a.spec = 1;
    a.exc_w = 0;   // no exception lists here: a first-pass mask counts only when exact as written
    a.ghist = reinterpret_cast<int*>(ds.base + kOffGhist);
    a.bq = reinterpret_cast<unsigned long long*>(ds.base + kOffQueue);
    a.t_out = d_t;
    a.phi_out = d_phi;
    a.status = d_status;
    a.df_tables = ds.base + kOffTables;
    long long grid = (long long)ds.sm_count * ds.blocks_per_sm;
    if (grid > (long long)a.ntotal) grid = a.ntotal;
    if (grid < 1) grid = 1;
    return launch_segment1d(a, (int)grid, 1, stream) == cudaSuccess ? TSALLIS_OK : TSALLIS_ERR_CUDA;
}
