// Per-slice 1-D thresholding that reads each voxel from HBM once: Algorithm 1
// is applied in the histogram pass with a predicted threshold, and the
// voxels whose side can still change are listed and rewritten once the
// exact threshold of section II-C ("Tsallis entropy", 1-D reading) is known.
//
// One cooperative launch (every block resident at once) in four phases
// separated by grid barriers:
//   1. predictions: block b takes slices b, b + G, ...; the histogram of
//      every s-th row of the slice and a plain FP32 search of it give a
//      predicted threshold t^ (its accuracy only affects speed, never the
//      result);
//   2. streaming: block b takes the b-th of G equal contiguous ranges of the
//      volume's voxels. Every voxel is counted into the block's histogram,
//      written to the mask with Algorithm 1 at its slice's t^, and, when its
//      level lies in the window (t^ - w, t^ + w], listed (position and
//      level) by its warp. At each slice boundary of the range the block
//      histogram is added to the slice's in global memory;
//   3. searches: block b takes slices b, b + G, ...: the exhaustive search
//      of the slice's histogram (search1d_fast) gives t. A voxel's mask bit
//      differs between t^ and t exactly when its level lies in
//      (min(t^, t), max(t^, t)]. So: t = t^, the mask is exact; |t - t^| <= w,
//      the listed voxels in that range are rewritten; otherwise (no
//      prediction, a list that overflowed, t far from t^, or no valid
//      threshold) the slice is queued for a second pass;
//   4. second passes of the queued slices, in pieces taken from a counter.
// The phases never wait on one another inside a phase, so the streaming
// phase runs at the rate of its voxel loop, and the small per-slice jobs
// (predictions, searches) run while the memory system is quiet.
//
// The grid barriers are bounded in time; one that runs out sets the
// launch's error flag, and every slice of that launch then reports
// TSALLIS_ERR_TIMEOUT (the next launch is unaffected).
#include <cmath>
#include <cstdint>

#include "common.cuh"
#include "dfmath.cuh"
#include "search1d.cuh"
#include "checked.cuh"
#include "firstpass.cuh"
#include "kernels.h"
#include "../../include/tsallis.h"

namespace tsl {

namespace {

using fp::kThreads;
using fp::kWarps;
using fp::kWarpBuf;
using fp::Sync;
using fp::prmt;
using fp::block_sync;
using fp::ld_stream;
using fp::Tile;
using fp::WarpList;
using fp::list_spill;
using fp::run_part;
using fp::PredSmem;
using fp::predict1d;
constexpr unsigned long long kPredReady = 1ull << 62;   // pred[z]: kPredReady | (t^ + 1)
constexpr int kFlagRebin = 1;                 // sflag[z]: the slice needs a second pass
// dynamic shared memory: the block histogram, the warps' list buffers, the
// search's terms; during a search its (level, count) list lies over the
// histogram and the list buffers
constexpr int kHistBytes = kMaxBins * 4;
constexpr int kOffList = kHistBytes;
constexpr int kOffTerms = kOffList + kWarps * kWarpBuf * 4;
constexpr int kSmemBytes = kOffTerms + kMaxBins * 8;
static_assert(kOffTerms >= kMaxBins * 8, "histogram and lists hold the search's (level, count) list");

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_add(int* p, int v) {
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long policy_evict_first() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// Grid barrier k (1, 2, ...): every block adds one to the counter; the
// barrier is passed once it reaches k blocks per block of the grid. The wait
// is bounded; once the launch's error flag is set no block waits any more.
__device__ void grid_sync(const SpecArgs& a, unsigned k, bool skip_arrival) {
    block_sync();
    if (threadIdx.x == 0) {
        __threadfence();
        if (!skip_arrival) atomicAdd(&a.hdr->gcount, 1u);
        const unsigned target = k * gridDim.x;
        const unsigned long long t0 = globaltimer_ns();
        while (ld_acquire_u32(&a.hdr->gcount) < target) {
            if (*(volatile int*)&a.hdr->err) break;
            if (globaltimer_ns() - t0 > a.timeout_ns) {
                atomicExch(&a.hdr->err, 1);
                break;
            }
            __nanosleep(128);
        }
        __threadfence();
    }
    block_sync();
}

// Start of block b's range of the volume's voxels (a multiple of 8).
__device__ __forceinline__ long long range_start(const SpecArgs& a, long long b) {
    return (b * a.nvox / (long long)gridDim.x) & ~7ll;
}

// Algorithm 1 at t over n voxels (a multiple of 8); t < 0 writes zeros.
__device__ void bin_pass(const int16_t* __restrict__ src, uint8_t* __restrict__ dst, int n, int t, int lo, int L,
                         bool le, unsigned long long pol) {
    const int T = (t >= L - 1) ? 32767 : (lo + t > 32767 ? 32767 : lo + t);
    const unsigned T2 = ((unsigned)T & 0xffffu) * 0x10001u;
    const uint4* v = reinterpret_cast<const uint4*>(src);
    uint2* d = reinterpret_cast<uint2*>(dst);
    for (int i = threadIdx.x; i < (n >> 3); i += kThreads) {
        uint2 m = make_uint2(0u, 0u);
        if (t >= 0) {
            const uint4 r = ld_stream(v + i, pol);
            unsigned c0, c1, c2, c3;
            if (le) {
                c0 = __vcmples2(r.x, T2); c1 = __vcmples2(r.y, T2); c2 = __vcmples2(r.z, T2); c3 = __vcmples2(r.w, T2);
            } else {
                c0 = __vcmpgts2(r.x, T2); c1 = __vcmpgts2(r.y, T2); c2 = __vcmpgts2(r.z, T2); c3 = __vcmpgts2(r.w, T2);
            }
            m = make_uint2(__byte_perm(c0, c1, 0x6420) & 0x01010101u, __byte_perm(c2, c3, 0x6420) & 0x01010101u);
        }
        st_stream(d + i, m);
    }
}

// ------------------------------------------------------------ corrections

// Rewrites the listed voxels of slice z whose level lies in [b0, b1] with
// Algorithm 1 at t (the side of every such voxel changes between t^ and t).
// The lists of the slice are those of the blocks bl .. bh whose ranges meet
// it (sixteen per block, one per warp). Warp w takes the lists w, w + 16,
// ..., 32 at a time: a warp scan of their counts lays their entries end to
// end, and each lane gathers up to 8 entries at once (a binary search over
// the lanes' offsets finds an entry's list).
__device__ void rewrite_listed(const SpecArgs& a, int z, long long bl, long long bh, int t, int b0, int b1,
                               int wbase, bool le, uint8_t* smask) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long S = a.slice_vox;
    const int nl = (int)(bh - bl + 1) * kWarps;
    for (int kb = warp; kb < nl; kb += kWarps * 32) {
        const int kl = kb + kWarps * lane;   // this lane's list
        int ne = 0;
        long long src = 0;
        if (kl < nl && range_start(a, bl + kl / kWarps) < range_start(a, bl + kl / kWarps + 1)) {   // ranges that hold voxels
            const long long b = bl + kl / kWarps;
            const int seg = (int)(z - range_start(a, b) / S);
            const long long li = (b * a.nseg + seg) * kWarps + (kl % kWarps);
            ne = __ldcg(&a.tcnt[li]);
            src = (b * kWarps + (kl % kWarps)) * (long long)a.wcap + __ldcg(&a.toff[li]);
        }
        int inc = ne;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += o;
        }
        const int exc = inc - ne, tot = __shfl_sync(0xffffffffu, inc, 31);
        for (int e0 = 0; e0 < tot; e0 += 32 * 8) {
            unsigned x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * 32 + lane;
                int lo = 0;   // the last lane whose offset is at most e
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (__shfl_sync(0xffffffffu, exc, lo + step) <= e) lo += step;
                const long long sl = __shfl_sync(0xffffffffu, src, lo);
                const int ex = __shfl_sync(0xffffffffu, exc, lo);
                x[u] = e < tot ? __ldcg(a.exc + sl + (e - ex)) : 0xffffffffu;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (x[u] == 0xffffffffu) continue;
                const int lev = (int)(x[u] & 0xffu) + wbase;
                const unsigned pos = x[u] >> 8;
                if (lev >= b0 && lev <= b1 && in_range(pos, S, a.check, kSiteSpecPatch))
                    smask[pos] = (uint8_t)(((lev <= t) == le) ? 1 : 0);
            }
        }
    }
}

struct KSmem {
    PredSmem psm;
    SearchSmem ssm;
    DfTables df;
    int last;
};

}  // namespace

__global__ void __launch_bounds__(kThreads, 2) k_slice_spec(const SpecArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    int* hist = reinterpret_cast<int*>(smem);
    char* shb = reinterpret_cast<char*>(smem);
    unsigned* lists = reinterpret_cast<unsigned*>(smem + kOffList);
    float2* sT = reinterpret_cast<float2*>(smem + kOffTerms);
    int2* sIC = reinterpret_cast<int2*>(smem);   // over the histogram and lists, during a search
    __shared__ KSmem ks;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int epoch = *(volatile int*)&a.hdr->epoch;
    const long long S = a.slice_vox;
    const long long G = gridDim.x, b = blockIdx.x;
    const bool le = a.polarity == 0;
    const unsigned long long pol = policy_evict_first();
    const int C0 = -4 * a.lo, top = 4 * (a.L - 1);

    for (int i = tid; i < kMaxBins; i += kThreads) hist[i] = 0;
    df_stage(&ks.df, static_cast<const DfTables*>(a.df_tables), tid, kThreads);
    block_sync();

    // ======================== 1. predictions
    for (long long z = b; z < a.nz; z += G) {
        const int16_t* svol = a.vol + z * S;
        const int s_ = a.sub_stride;
        const int nrows = a.ny >= s_ ? a.ny / s_ : 1;
        const int y0 = a.ny >= s_ ? s_ / 2 : a.ny / 2;
        const long long nsub = (long long)nrows * a.nx;
        if ((a.nx & 7) == 0) {
            const int wpr = a.nx >> 3;
            const long long nw = nsub / 8;
            for (long long i0 = 0; i0 < nw; i0 += 4 * kThreads) {
                uint4 r[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const long long i = i0 + u * kThreads + tid;
                    r[u] = make_uint4(0u, 0u, 0u, 0u);
                    if (i < nw) {
                        const int row = (int)(i / wpr), c = (int)(i % wpr);
                        r[u] = __ldg(reinterpret_cast<const uint4*>(svol + (long long)(y0 + row * s_) * a.nx) + c);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (i0 + u * kThreads + tid >= nw) continue;
                    const unsigned w4[4] = {r[u].x, r[u].y, r[u].z, r[u].w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int va = (int)prmt(w4[j], 0u, 0x9910u), vb = ((int)w4[j]) >> 16;
                        atomicAdd(reinterpret_cast<int*>(shb + min(max(va * 4 + C0, 0), top)), 1);
                        atomicAdd(reinterpret_cast<int*>(shb + min(max(vb * 4 + C0, 0), top)), 1);
                    }
                }
            }
        } else {
            for (long long i = tid; i < nsub; i += kThreads) {
                const int row = (int)(i / a.nx), c = (int)(i % a.nx);
                const int va = svol[(long long)(y0 + row * s_) * a.nx + c];
                atomicAdd(reinterpret_cast<int*>(shb + min(max(va * 4 + C0, 0), top)), 1);
            }
        }
        block_sync();
        int th = predict1d(hist, a.L, a.q, reinterpret_cast<int2*>(lists), ks.psm);
        if (a.flags & kSpecDebugNoPrediction) th = -1;   // test hook: no predictions
        for (int i = tid; i < kMaxBins; i += kThreads) hist[i] = 0;
        if (tid == 0) a.pred[z] = kPredReady | (unsigned)(th + 1);
        block_sync();   // the histogram is zeroed before it counts again
    }
    grid_sync(a, 1, false);

    // ======================== 2. streaming: this block's range of voxels
    {
        const long long r0 = range_start(a, b), r1 = range_start(a, b + 1);
        WarpList wl;
        wl.buf = lists + warp * kWarpBuf;
        wl.glob = a.exc + (b * kWarps + warp) * (long long)a.wcap;
        wl.n = 0;
        wl.g = 0;
        wl.cap = a.wcap;
        int seg = 0;
        for (long long p = r0; p < r1; ++seg) {
            const long long z = p / S, e = (r1 < (z + 1) * S) ? r1 : (z + 1) * S;
            const unsigned long long pv = *(volatile unsigned long long*)&a.pred[z];
            const int th = (pv & kPredReady) ? (int)(pv & 0xffffffffu) - 1 : -1;
            Tile x;
            x.C0 = C0;
            x.top = top;
            x.bin = th >= 0;
            x.MT2 = (unsigned)(0x8000 - 4 * (th + 1)) * 0x10001u;
            x.POL = le ? 0x01010101u : 0u;
            {
                const int wlo = th - a.win + 1, whi = th + a.win > a.L - 1 ? a.L - 1 : th + a.win;
                x.WA2 = (unsigned)(0x8000 - 4 * (wlo > 0 ? wlo : 0)) * 0x10001u;
                x.WB2 = (unsigned)(0x8000 - 4 * (whi + 1)) * 0x10001u;
                x.wbase = wlo;
            }
            wl.over = false;
            const int gstart = wl.g;
            run_part<false>(x, a.vol + p, a.mask + p, (int)(e - p), (unsigned)(p - z * S), shb, wl, pol);
            if (x.bin) list_spill(wl);
            // the warp's list of this part of slice z: where it starts and how
            // long it is (-1: incomplete; the slice then gets a second pass)
            if (lane == 0) {
                const long long li = (b * a.nseg + seg) * kWarps + warp;
                a.toff[li] = gstart;
                a.tcnt[li] = (!x.bin || wl.over) ? -1 : wl.g - gstart;
                if (!x.bin || wl.over) atomicOr(&a.sflag[z], kFlagRebin);
            }
            block_sync();   // the block histogram is complete
            int* gh = a.ghist + z * kMaxBins;
            for (int i = tid; i < a.L; i += kThreads) {
                const int c = hist[i];
                if (c) {
                    red_add(&gh[i], c);
                    hist[i] = 0;
                }
            }
            block_sync();   // zeroed before the next part counts
            p = e;
        }
    }
    grid_sync(a, 2, (a.flags & TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL) && b == 0);   // test hook: block 0 never arrives

    // ======================== 3. searches and corrections
    const bool failed = *(volatile int*)&a.hdr->err != 0;
    for (long long z = b; z < a.nz; z += G) {
        int* gh = a.ghist + z * kMaxBins;
        const SearchResult r =
            (a.ptab != nullptr && S == a.ptab_n)
                ? search1d_fast<Sync>(gh, a.L, a.q, a.ptab, S, ks.ssm, sIC, sT, &ks.df)
                : search1d_block<Sync>(gh, a.L, a.q, nullptr, ks.ssm, sT, sIC, &ks.df);
        // the slice's histogram is left zeroed; the block histogram (the
        // search's scratch) is zeroed again
        for (int i = tid * 4; i < kMaxBins; i += kThreads * 4) *reinterpret_cast<int4*>(gh + i) = make_int4(0, 0, 0, 0);
        for (int i = tid * 4; i < kMaxBins; i += kThreads * 4) *reinterpret_cast<int4*>(hist + i) = make_int4(0, 0, 0, 0);
        const unsigned long long pv = *(volatile unsigned long long*)&a.pred[z];
        const int th = (pv & kPredReady) ? (int)(pv & 0xffffffffu) - 1 : -1;
        // the blocks whose ranges meet the slice
        long long bl = (z * S * G) / a.nvox, bh = ((z + 1) * S * G) / a.nvox;
        while (bl > 0 && range_start(a, bl) > z * S) --bl;
        while (bl + 1 < G && range_start(a, bl + 1) <= z * S) ++bl;
        if (bh >= G) bh = G - 1;
        while (bh > bl && range_start(a, bh) >= (z + 1) * S) --bh;
        while (bh + 1 < G && range_start(a, bh + 1) < (z + 1) * S) ++bh;
        const bool listed = th >= 0 && !(*(volatile int*)&a.sflag[z] & kFlagRebin);
        const int t = r.t, dt = t - th;
        int fix;   // 0 exact, 1 rewrite listed voxels, 2 second pass
        if (t >= 0 && th >= 0 && dt == 0) fix = 0;
        else if (t >= 0 && listed && dt >= -a.win && dt <= a.win) fix = 1;
        else fix = 2;
        if (fix == 1)
            rewrite_listed(a, (int)z, bl, bh, t, (th < t ? th : t) + 1, th < t ? t : th, th - a.win + 1, le,
                           a.mask + z * S);
        if (tid == 0) {
            a.t_out[z] = failed ? -1 : t;
            a.phi_out[z] = failed ? 0.f : r.phi;
            a.status[z] = failed ? TSALLIS_ERR_TIMEOUT : (r.status | (fix < 2 ? TSALLIS_STATUS_FIRST_PASS_EXACT : 0));
            a.sflag[z] = 0;
            a.pred[z] = 0ull;
            if (fix == 2 && !failed) {
                // the slice's pieces join the second-pass queue
                const int np = (int)((S + a.piece_vox - 1) / a.piece_vox);
                const unsigned base = atomicAdd(&a.hdr->b_tail, (unsigned)np);
                for (int k = 0; k < np; ++k)
                    if (in_range(base + k, (long long)a.nz * a.npiece, a.check, kSiteSpecQueue))
                        a.rbq[base + k] = ((unsigned)z << 12) | (unsigned)k;
            }
        }
        block_sync();   // the scratch is free before the next search
    }
    grid_sync(a, 3, false);

    // ======================== 4. second passes
    {
        const unsigned nq = *(volatile unsigned*)&a.hdr->b_tail;
        for (;;) {
            if (tid == 0) ks.last = (int)atomicAdd(&a.hdr->b_next, 1u);
            block_sync();
            const unsigned k = (unsigned)ks.last;
            block_sync();
            if (k >= nq) break;
            const unsigned e = __ldcg(&a.rbq[k]);
            const long long z = e >> 12, off = (long long)(e & 0xfffu) * a.piece_vox;
            const int n = (int)(S - off < a.piece_vox ? S - off : a.piece_vox);
            bin_pass(a.vol + z * S + off, a.mask + z * S + off, n, __ldcg(&a.t_out[z]), a.lo, a.L, le, pol);
        }
    }

    // exit: the last block restores the counters for the next launch
    block_sync();
    if (tid == 0) {
        __threadfence();
        ks.last = atomicAdd(&a.hdr->done, 1u) == gridDim.x - 1;
    }
    block_sync();
    if (ks.last && tid == 0) {
        __threadfence();
        a.hdr->gcount = 0;
        a.hdr->b_next = 0;
        a.hdr->b_tail = 0;
        a.hdr->done = 0;
        a.hdr->err = 0;
        a.hdr->epoch = epoch + 1;
        __threadfence();
    }
}

int slice_spec_smem_bytes() { return kSmemBytes; }

cudaError_t slice_spec_prepare() {
    return cudaFuncSetAttribute(k_slice_spec, cudaFuncAttributeMaxDynamicSharedMemorySize, slice_spec_smem_bytes());
}

cudaError_t slice_spec_occupancy(int* blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_slice_spec, kThreads,
                                                         slice_spec_smem_bytes());
}

cudaError_t launch_slice_spec(const SpecArgs& a, int grid, cudaStream_t s) {
    // cooperative: every block is resident at once (the grid barriers rely on it)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = slice_spec_smem_bytes();
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_slice_spec, a);
}

}  // namespace tsl
