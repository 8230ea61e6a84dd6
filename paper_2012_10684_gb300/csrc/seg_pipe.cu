// Per-slice 1-D thresholding in one persistent pass that reads each voxel
// from HBM once in the usual case: the histogram of section II-C, the
// exhaustive search of the Tsallis objective and Algorithm 1.
//
// The volume's slices are cut into chunks (at most 8 per slice, taken in
// slice order from one global counter, claimed one chunk ahead). Every block
// repeats, choosing in this order:
//   * search a slice whose last chunk it counted (all 512 threads; the
//     threshold is published for the slice and as the launch's latest);
//   * finish the oldest chunk it counted, once that chunk's slice has its
//     threshold t (see below);
//   * count the next chunk: each voxel goes into the block's shared-memory
//     histogram and, when the chunk has a predicted threshold t^, is
//     written to the mask with Algorithm 1 at t^; a warp lists the 16-byte
//     groups (8 voxels) that hold a voxel whose level lies in the window
//     (t^ - w, t^ + w].
//     t^ is the latest published threshold of the launch; before any is
//     published, the plain FP32 search of a 1/16 sample of the chunk's own
//     voxels. The block histogram is then added to the slice's in global
//     memory and the block arrives on the slice's counter;
//   * otherwise wait, bounded, for the threshold of its oldest chunk.
// A voxel's mask differs between t^ and t exactly when its level lies in
// (min(t^, t), max(t^, t)]. So a chunk is finished: when t = t^, with
// nothing to do; when |t - t^| <= w and its lists are complete, by
// binarising the listed groups again; otherwise (no prediction, a list that
// overflowed, t far from t^, or no valid threshold) by binarising it again.
//
// A block keeps at most kRing chunks it has counted but not finished, with
// their predictions and list lengths, and claims no new chunk while it holds
// kRing - 2; the oldest of them then lies in a slice all of whose chunks were
// claimed earlier (a slice has at most 8 chunks), and a claimed chunk is
// always counted before its block waits, so every wait ends. Each wait is
// also bounded in time: one that runs out sets the launch's error flag, every
// block stops, and every slice of the call reports TSALLIS_ERR_TIMEOUT (the
// last block restores the scratch state for the next launch).
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

using fp::kThreads;   // 512
using fp::kWarps;     // 16
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

constexpr int kRing = kPipeRing;              // counted chunks awaiting their threshold
constexpr int kMaxChunksPerSlice = 8;
static_assert(kRing - 2 > kMaxChunksPerSlice, "a full ring spans more than one slice");
constexpr int kSampleStride = 16;             // prediction sample: one 16-byte word in 16
// dynamic shared memory: the block histogram, the warps' list buffers, the
// search's terms; during a search its (level, count) list lies over the
// histogram and the list buffers, and during a prediction the sample's
// (level, count) list over the list buffers
constexpr int kOffList = kMaxBins * 4;
constexpr int kOffTerms = kOffList + kWarps * kWarpBuf * 4;
constexpr int kSmemBytes = kOffTerms + kMaxBins * 8;
static_assert(kOffTerms >= kMaxBins * 8, "histogram and lists hold the search's (level, count) list");

__device__ __forceinline__ void red_add(int* p, int v) {
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
    return *(const volatile unsigned long long*)p;
}
__device__ __forceinline__ unsigned long long policy(bool last) {
    unsigned long long p;
    if (last)
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    else
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Algorithm 1 at t over n voxels (a multiple of 8): mask = (level <= t) for
// polarity low, (level > t) for high; t < 0 (no valid threshold) writes 0.
__device__ void binarise_chunk(const Tile& x, const int16_t* __restrict__ src, uint8_t* __restrict__ dst, int n,
                               int t, unsigned long long pol) {
    const uint4* v = reinterpret_cast<const uint4*>(src);
    uint2* d = reinterpret_cast<uint2*>(dst);
    const int nv = n >> 3, tid = threadIdx.x;
    if (t < 0) {
        for (int i = tid; i < nv; i += kThreads) st_stream(d + i, make_uint2(0u, 0u));
        return;
    }
    // bit 15 of o + MT2 (16-bit lanes, o <= 0x3ffc): o >= 4 (t + 1), i.e. level > t
    const unsigned MT2 = (unsigned)(0x8000 - 4 * (t + 1)) * 0x10001u;
    auto mask8 = [&](uint4 r) {
        const unsigned w[4] = {r.x, r.y, r.z, r.w};
        unsigned m[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int a = (int)prmt(w[j], 0u, 0x9910u), b = ((int)w[j]) >> 16;
            const int oa = min(max(a * 4 + x.C0, 0), x.top), ob = min(max(b * 4 + x.C0, 0), x.top);
            m[j] = prmt((unsigned)oa, (unsigned)ob, 0x5410u) + MT2;
        }
        // selector nibbles 9, b, d, f: the sign bytes of the four 16-bit lanes
        return make_uint2((prmt(m[0], m[1], 0xFDB9u) & 0x01010101u) ^ x.POL,
                          (prmt(m[2], m[3], 0xFDB9u) & 0x01010101u) ^ x.POL);
    };
    constexpr int U = 4;
    int i0 = 0;
    for (; i0 + U * kThreads <= nv; i0 += U * kThreads) {
        uint4 r[U];
#pragma unroll
        for (int u = 0; u < U; ++u) r[u] = ld_stream(v + i0 + u * kThreads + tid, pol);
#pragma unroll
        for (int u = 0; u < U; ++u) st_stream(d + i0 + u * kThreads + tid, mask8(r[u]));
    }
    for (int i = i0 + tid; i < nv; i += kThreads) st_stream(d + i, mask8(ld_stream(v + i, pol)));
}

// The histogram of one 16-byte word in kSampleStride of n voxels.
__device__ void sample_chunk(const Tile& x, const int16_t* __restrict__ src, int n, char* shb) {
    const uint4* v = reinterpret_cast<const uint4*>(src);
    const int nw = (n >> 3) / kSampleStride;
    for (int i = threadIdx.x; i < nw; i += kThreads) {
        const uint4 r = __ldg(v + (long long)i * kSampleStride);
        const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int a = (int)prmt(w[j], 0u, 0x9910u), b = ((int)w[j]) >> 16;
            atomicAdd(reinterpret_cast<int*>(shb + min(max(a * 4 + x.C0, 0), x.top)), 1);
            atomicAdd(reinterpret_cast<int*>(shb + min(max(b * 4 + x.C0, 0), x.top)), 1);
        }
    }
}

enum Kind : int { kCount = 0, kFinish = 1, kSearch = 2, kWait = 3, kExit = 4 };

// What finishing a chunk takes once its slice's threshold t is known.
enum Finish : int { kDone = 0, kPatch = 1, kRebin = 2 };

struct RingEntry {
    int chunk;
    int pred;              // t^ (-1: none)
    int cnt[kWarps];       // list lengths (-1: overflowed)
};

struct PipeSmem {
    SearchSmem ssm;
    PredSmem psm;
    DfTables df;
    // thread 0's state
    unsigned long long tag;       // readiness tag of this launch
    unsigned long long wait_t0;   // start of the current wait (0: not waiting)
    RingEntry ring[kRing];        // counted chunks awaiting their threshold
    int rhead, rcount;
    int exhausted;                // every chunk has been claimed
    int kind[2], arg[2], arg2[2], arg3[2];   // the decision (alternate slots)
};

// The slice's search, kept out of line: it needs more registers than the
// chunk loops, and runs about once per block.
__device__ __noinline__ SearchResult slice_search(const PipeArgs& a, const int* gh, PipeSmem& ks, int2* sIC,
                                                  float2* sT) {
    const long long S = a.slice_vox;
    return (a.ptab != nullptr && S == a.ptab_n)
               ? search1d_fast<Sync>(gh, a.L, a.q, a.ptab, S, ks.ssm, sIC, sT, &ks.df)
               : search1d_block<Sync>(gh, a.L, a.q, nullptr, ks.ssm, sT, sIC, &ks.df);
}

// Binarises again, with Algorithm 1 at t, the listed 16-byte groups of a
// chunk (those holding a voxel within the window of t^): every voxel whose
// side changes between t^ and t is in one of them. Warp w takes its own
// list.
__device__ void patch_chunk(const PipeArgs& a, const RingEntry& e, int slot, int t, const int16_t* __restrict__ csrc,
                            uint8_t* __restrict__ cmask, int n, const Tile& x) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned* list = a.exc + (((long long)blockIdx.x * kRing + slot) * kWarps + warp) * a.wcap;
    const int cnt = e.cnt[warp];
    const uint4* v = reinterpret_cast<const uint4*>(csrc);
    uint2* d = reinterpret_cast<uint2*>(cmask);
    const unsigned MT2 = (unsigned)(0x8000 - 4 * (t + 1)) * 0x10001u;
    for (int i = lane; i < cnt; i += 32) {
        const unsigned g = __ldcg(list + i);
        if (!in_range(g, n >> 3, a.check, kSitePipePatch)) continue;
        const uint4 r = __ldcs(v + g);
        const unsigned w[4] = {r.x, r.y, r.z, r.w};
        unsigned m[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = (int)prmt(w[j], 0u, 0x9910u), q = ((int)w[j]) >> 16;
            const int op = min(max(p * 4 + x.C0, 0), x.top), oq = min(max(q * 4 + x.C0, 0), x.top);
            m[j] = prmt((unsigned)op, (unsigned)oq, 0x5410u) + MT2;
        }
        st_stream(d + g, make_uint2((prmt(m[0], m[1], 0xFDB9u) & 0x01010101u) ^ x.POL,
                                    (prmt(m[2], m[3], 0xFDB9u) & 0x01010101u) ^ x.POL));
    }
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 2) k_slice_pipe(const PipeArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    int* hist = reinterpret_cast<int*>(smem);
    char* shb = reinterpret_cast<char*>(smem);
    unsigned* lists = reinterpret_cast<unsigned*>(smem + kOffList);
    int2* sIC = reinterpret_cast<int2*>(smem);
    float2* sT = reinterpret_cast<float2*>(smem + kOffTerms);
    __shared__ PipeSmem ks;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nc = a.chunks_per_slice;
    const bool le = a.polarity == 0;

    for (int i = tid; i < kMaxBins; i += kThreads) hist[i] = 0;
    df_stage(&ks.df, static_cast<const DfTables*>(a.df_tables), tid, kThreads);
    if (tid == 0) {
        ks.tag = ld_volatile_u64(&a.hdr->serial) + 1;   // this launch's readiness tag
        ks.wait_t0 = 0;
        ks.rhead = 0;
        ks.rcount = 0;
        ks.exhausted = 0;
    }
    // thread 0's results in flight, used at the next decision: a claimed
    // chunk, the counter value of its last arrival, the oldest counted
    // chunk's readiness word, the launch's latest threshold, its error flag
    int claim = -1;
    int arr_z = -1, arr_old = 0;
    unsigned long long pf_ready = 0, pf_latest = 0;
    int pf_err = 0;
    block_sync();

    for (int it = 0;; ++it) {
        const int slot = it & 1;
        if (tid == 0) {
            const int NC = a.nz * nc;
            int kind = kWait, arg = 0, arg2 = 0, arg3 = 0;
            int rhead = ks.rhead, rcount = ks.rcount;
            if (pf_err) {
                kind = kExit;
            } else if (arr_z >= 0 && arr_old == nc - 1) {
                kind = kSearch;   // this block counted the slice's last chunk
                arg = arr_z;
                arr_z = -1;
                __threadfence();   // the other blocks' adds to the slice's histogram are seen after the barrier
            } else {
                arr_z = -1;
                if (rcount > 0 && (pf_ready >> 13) == ks.tag) {
                    // the oldest counted chunk's slice has its threshold
                    const RingEntry& e = ks.ring[rhead];
                    const int t = (int)(pf_ready & 0x1fffu) - 1;
                    int f = kRebin;
                    if (t >= 0 && e.pred == t) {
                        f = kDone;
                    } else if (t >= 0 && e.pred >= 0 && t - e.pred <= a.win && e.pred - t <= a.win) {
                        f = kPatch;
                        for (int w = 0; w < kWarps; ++w)
                            if (e.cnt[w] < 0) f = kRebin;
                    }
                    kind = kFinish;
                    arg = rhead;   // the ring slot (reused only after a later decision)
                    arg2 = t;
                    arg3 = f;
                    rhead = (rhead + 1) % kRing;
                    --rcount;
                } else {
                    if (claim < 0 && !ks.exhausted && rcount < kRing - 2)
                        claim = (int)min(atomicAdd(&a.hdr->h_next, 1u), (unsigned)NC);
                    if (claim >= NC) {   // fresh or prefetched: past the last chunk
                        ks.exhausted = 1;
                        claim = -1;
                    }
                    if (claim >= 0) {
                        kind = kCount;
                        arg = claim;
                        arg2 = (rhead + rcount) % kRing;   // its ring slot
                        // the prediction: the launch's latest threshold, if any (-2: none yet)
                        arg3 = (pf_latest >> 13) == ks.tag ? (int)(pf_latest & 0x1fffu) - 1 : -2;
                        ks.ring[arg2].chunk = claim;
                        ++rcount;
                        claim = -1;
                        // claim the next chunk now; its number arrives while this one is counted
                        if (!ks.exhausted && rcount < kRing - 2)
                            claim = (int)min(atomicAdd(&a.hdr->h_next, 1u), (unsigned)NC);
                    } else if (rcount == 0) {
                        kind = ks.exhausted ? kExit : kWait;
                    }
                }
            }
            if (kind == kWait) {
                // nothing to do until the oldest chunk's threshold arrives
                const unsigned long long now = globaltimer_ns();
                if (ks.wait_t0 == 0) ks.wait_t0 = now;
                if (now - ks.wait_t0 > a.timeout_ns) {
                    atomicExch(&a.hdr->err, 1);
                    kind = kExit;
                } else {
                    __nanosleep(256);
                }
            } else {
                ks.wait_t0 = 0;
            }
            // read now, used at the next decision
            pf_err = *(volatile int*)&a.hdr->err;
            pf_latest = ld_volatile_u64(&a.hdr->pipe_latest);
            if (rcount > 0) pf_ready = ld_volatile_u64(&a.ready[ks.ring[rhead].chunk / nc]);
            ks.rhead = rhead;
            ks.rcount = rcount;
            ks.kind[slot] = kind;
            ks.arg[slot] = arg;
            ks.arg2[slot] = arg2;
            ks.arg3[slot] = arg3;
        }
        block_sync();
        const int kind = ks.kind[slot], arg = ks.arg[slot];
        if (kind == kExit) break;
        if (kind == kWait) continue;

        if (kind == kCount || kind == kFinish) {
            const int rs = kind == kCount ? ks.arg2[slot] : arg;   // ring slot
            const int chunk = ks.ring[rs].chunk;
            const int z = chunk / nc, c = chunk - z * nc;
            const long long off = (long long)z * a.slice_vox + (long long)c * a.chunk_vox;
            const long long rest = a.slice_vox - (long long)c * a.chunk_vox;
            const int n = (int)(rest < a.chunk_vox ? rest : a.chunk_vox);
            const bool ok = in_range(z, a.nz, a.check, kSitePipeChunk);
            if (kind == kFinish) {
                const int t = ks.arg2[slot], f = ks.arg3[slot];
                if (ok && f == kRebin)
                    binarise_chunk(fp::make_tile(a.lo, a.L, t, a.win, le), a.vol + off, a.mask + off, n, t,
                                   policy(false));
                else if (ok && f == kPatch)
                    patch_chunk(a, ks.ring[rs], rs, t, a.vol + off, a.mask + off, n,
                                fp::make_tile(a.lo, a.L, t, a.win, le));
                continue;
            }
            // ---- count (and, with a prediction, binarise and list) the chunk
            int th = ks.arg3[slot];
            if (th == -2) {
                // no threshold published yet: predict from a sample of the chunk
                if (ok) sample_chunk(fp::make_tile(a.lo, a.L, -1, a.win, le), a.vol + off, n, shb);
                block_sync();
                th = predict1d(hist, a.L, a.q, reinterpret_cast<int2*>(lists), ks.psm);
                for (int i = tid; i < kMaxBins; i += kThreads) hist[i] = 0;
                block_sync();   // zeroed before the chunk is counted
            }
            if (a.flags & kPipeDebugNoPrediction) th = -1;   // test hook: every chunk is binarised again
            const Tile x = fp::make_tile(a.lo, a.L, th, a.win, le);
            WarpList wl;
            wl.buf = lists + warp * kWarpBuf;
            wl.glob = a.exc + (((long long)blockIdx.x * kRing + rs) * kWarps + warp) * a.wcap;
            wl.n = 0;
            wl.g = 0;
            wl.cap = a.wcap;
            wl.over = false;
            if (ok) run_part<true>(x, a.vol + off, a.mask + off, n, 0u, shb, wl, policy(true));
            if (x.bin) list_spill(wl);
            if (lane == 0) ks.ring[rs].cnt[warp] = wl.over ? -1 : wl.g;
            if (tid == 0) ks.ring[rs].pred = th;
            block_sync();   // the block histogram is complete
            int* gh = a.ghist + (long long)z * kMaxBins;
            for (int i = tid; i < a.L; i += kThreads) {
                const int v = hist[i];
                if (v) {
                    red_add(&gh[i], v);
                    hist[i] = 0;
                }
            }
            block_sync();   // every add of the chunk is issued
            if (tid == 0) {
                if ((a.flags & TSALLIS_FLAG_DEBUG_SKIP_ARRIVAL) && chunk == 0) {
                    // test hook: the first chunk never arrives
                } else {
                    __threadfence();
                    arr_old = atomicAdd(&a.parts[z], 1);   // looked at in the next decision
                    arr_z = z;
                }
            }
        } else {   // kSearch: every chunk of slice arg has arrived
            const int z = arg;
            int* gh = a.ghist + (long long)z * kMaxBins;
            const SearchResult r = slice_search(a, gh, ks, sIC, sT);
            // the slice's histogram is left zeroed, and the block histogram (the search's scratch)
            for (int i = tid * 4; i < kMaxBins; i += kThreads * 4) *reinterpret_cast<int4*>(gh + i) = make_int4(0, 0, 0, 0);
            for (int i = tid * 4; i < kMaxBins; i += kThreads * 4) *reinterpret_cast<int4*>(hist + i) = make_int4(0, 0, 0, 0);
            if (tid == 0) {
                a.t_out[z] = r.t;
                a.phi_out[z] = r.phi;
                a.status[z] = r.status;
                a.parts[z] = 0;
                // the readiness word carries t itself: nothing else needs ordering before it
                const unsigned long long w = (ks.tag << 13) | (unsigned long long)(r.t + 1);
                *(volatile unsigned long long*)&a.ready[z] = w;
                if (r.t >= 0) *(volatile unsigned long long*)&a.hdr->pipe_latest = w;   // the next predictions
            }
            block_sync();   // the scratch is free before the block counts again
        }
    }

    // exit: the last block restores the scratch state for the next launch
    __shared__ int last;
    if (tid == 0) {
        __threadfence();
        last = atomicAdd(&a.hdr->done, 1u) == gridDim.x - 1;
    }
    block_sync();
    if (!last) return;
    __threadfence();
    const bool failed = *(volatile int*)&a.hdr->err != 0;
    if (failed) {
        // slices that never completed keep partial histograms and counters
        for (long long i = tid; i < (long long)a.nz * kMaxBins; i += kThreads) a.ghist[i] = 0;
        for (int z = tid; z < a.nz; z += kThreads) {
            a.parts[z] = 0;
            a.t_out[z] = -1;
            a.phi_out[z] = 0.f;
            a.status[z] = TSALLIS_ERR_TIMEOUT;
        }
    }
    block_sync();
    if (tid == 0) {
        __threadfence();
        a.hdr->h_next = 0;
        a.hdr->done = 0;
        a.hdr->err = 0;
        a.hdr->serial = ks.tag;
        __threadfence();
    }
}

int slice_pipe_smem_bytes() { return kSmemBytes; }

cudaError_t slice_pipe_prepare() {
    return cudaFuncSetAttribute(k_slice_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, slice_pipe_smem_bytes());
}

cudaError_t slice_pipe_occupancy(int* blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_slice_pipe, kThreads,
                                                         slice_pipe_smem_bytes());
}

int pipe_chunks_per_slice(long long slice_vox, long long* chunk_vox) {
    // chunks of at least 131072 voxels (fewer, longer chunks measured
    // faster than 32768 or 65536 on 512x512 slices), at most
    // kMaxChunksPerSlice per slice
    long long c = (slice_vox + kMaxChunksPerSlice - 1) / kMaxChunksPerSlice;
    c = (c + 7) / 8 * 8;
    if (c < 131072) c = 131072;
    if (c > slice_vox) c = slice_vox;
    *chunk_vox = c;
    return (int)((slice_vox + c - 1) / c);
}

cudaError_t launch_slice_pipe(const PipeArgs& a, int grid, cudaStream_t s) {
    // cooperative: every block is resident at once (the waits rely on it)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = slice_pipe_smem_bytes();
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_slice_pipe, a);
}

}  // namespace tsl
