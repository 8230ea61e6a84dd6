// 1-D thresholding path: histogram, search and binarise fused in one
// persistent kernel (two 512-thread blocks per SM).
//
// Work is split into tiles of a group's voxels (a group is one slice, or
// the whole volume, or one volume of a batch). Each block repeatedly takes
// one tile:
//   * a binarise tile of the oldest group whose threshold is published, if
//     it still has untaken tiles (per-group counters, a head pointer that
//     only moves forward), so a slice is re-read while it is still in L2;
//   * otherwise the next histogram tile (one global counter);
//   * otherwise (every histogram tile is taken) it waits, bounded, for the
//     oldest unfinished group's threshold.
// A histogram tile counts its voxels into a shared-memory histogram and adds
// it to the group's histogram in global memory. The block that adds the last
// tile of a group runs the exhaustive search of section II-C on it (all 512
// threads) and publishes the threshold. A binarise tile applies Algorithm 1.
//
// Histogram tiles never wait, and a block waits for a threshold only after
// every histogram tile has been taken by running blocks, so waits end.
// Every wait is bounded in time; a wait that runs out is reported per group.
#include <cmath>

#include "common.cuh"
#include "dfmath.cuh"
#include "search1d.cuh"
#include "checked.cuh"
#include "kernels.h"

namespace tsl {

constexpr int kSegThreads = kSearchThreads;  // 512
constexpr int kSegMinBlocks = 2;
constexpr int kExcSmem = kMaxBins * 2;   // a tile's exceptions held in shared memory (in the search's sT and sIC)

__device__ __forceinline__ long long lmin(long long a, long long b) { return a < b ? a : b; }

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long policy_evict_last() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long policy_evict_first() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// 16-byte read-only load that skips L1, with an L2 eviction policy.
__device__ __forceinline__ uint4 ld_v4_policy(const void* p, unsigned long long pol) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p), "l"(pol));
    return r;
}

// ------------------------------------------------------------ tiles

// Histogram of 8 voxels: clamp both 16-bit halves of each word to
// [lo, hi] with packed min/max, then one shared-memory atomic per voxel at
// shb[v] (shb = sh - lo, so shb[v] is level v - lo).
__device__ __forceinline__ void hist8(uint4 r, unsigned LO2, unsigned HI2, int* shb) {
    const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const unsigned c = __vmins2(__vmaxs2(w[j], LO2), HI2);
        atomicAdd(shb + (int)(short)(c & 0xffffu), 1);
        atomicAdd(shb + (((int)c) >> 16), 1);
    }
}

__device__ __forceinline__ int clamp_level(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Algorithm 1 on 8 voxels with packed 16x2 compares: byte = 1 where
// v <= T (le) or v > T (!le).
__device__ __forceinline__ uint2 mask8(uint4 r, unsigned T2, bool le) {
    unsigned m0, m1, m2, m3;
    if (le) {
        m0 = __vcmples2(r.x, T2); m1 = __vcmples2(r.y, T2); m2 = __vcmples2(r.z, T2); m3 = __vcmples2(r.w, T2);
    } else {
        m0 = __vcmpgts2(r.x, T2); m1 = __vcmpgts2(r.y, T2); m2 = __vcmpgts2(r.z, T2); m3 = __vcmpgts2(r.w, T2);
    }
    // bytes 0 and 2 of each compare word hold one voxel each
    return make_uint2(__byte_perm(m0, m1, 0x6420) & 0x01010101u, __byte_perm(m2, m3, 0x6420) & 0x01010101u);
}

// Level <= t in Algorithm 1 terms: level = clamp(v - lo, 0, L-1) >> shift,
// so for 0 <= t < top level it is v <= lo + ((t + 1) << shift) - 1; at or
// above the top level every voxel qualifies. Clamped to the int16 range
// (v <= 32767 always holds).
__device__ __forceinline__ int bin_threshold(int t, int lo, int L, int shift) {
    const int T = (t >= ((L - 1) >> shift)) ? 32767 : lo + ((t + 1) << shift) - 1;
    return T > 32767 ? 32767 : T;
}

// First-pass exceptions: voxels whose (clamped) value lies in [wlo, whi],
// the window of levels around the predicted threshold, are appended to a
// shared-memory list as (position in group << 16) | (level - wbase).
struct ExcCtx {
    unsigned long long* list;   // shared memory
    int* n;             // shared counter
    int cap;
    unsigned wlo2, whi2;   // window bounds as packed 16x2 values
    int wlo, whi;
    int lo;             // value of level 0
    int wbase;          // level stored as 0
    long long pos0;     // position in the group of src[0]
};

__device__ __forceinline__ void exc_append1(const ExcCtx& e, long long pos, int c) {
    if (c >= e.wlo && c <= e.whi) {
        const int k = atomicAdd(e.n, 1);
        if (k < e.cap) e.list[k] = ((unsigned long long)pos << 16) | (unsigned)(c - e.lo - e.wbase);
    }
}

// The exceptions among 8 clamped voxels (4 packed words) at group position
// pos. The lanes of a warp reserve their entries with one shared atomic
// (each lane's offset is the sum of the counts of the lower active lanes,
// built from ballots of the count's bits).
__device__ __forceinline__ void exc_append8(const ExcCtx& e, const unsigned (&cl)[4], long long pos) {
    unsigned bits = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const unsigned m = __vcmpges2(cl[j], e.wlo2) & __vcmples2(cl[j], e.whi2);
        bits |= ((m & 1u) | ((m >> 15) & 2u)) << (2 * j);
    }
    const unsigned act = __activemask();
    if (__any_sync(act, bits != 0) == 0) return;
    const unsigned cnt = __popc(bits);
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt = (1u << lane) - 1u;
    unsigned off = 0, tot = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const unsigned bal = __ballot_sync(act, (cnt >> b) & 1u);
        off += (unsigned)__popc(bal & lt) << b;
        tot += (unsigned)__popc(bal) << b;
    }
    const int leader = __ffs(act) - 1;
    int base = 0;
    if ((int)lane == leader) base = atomicAdd(e.n, (int)tot);
    int k = __shfl_sync(act, base, leader) + (int)off;
    while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1;
        const unsigned w = cl[b >> 1];
        const int c = (b & 1) ? ((int)w >> 16) : (int)(short)(w & 0xffffu);
        if (k < e.cap) e.list[k] = ((unsigned long long)(pos + b) << 16) | (unsigned)(c - e.lo - e.wbase);
        ++k;
    }
}

// Histogram of 8 voxels that also returns the clamped words (for the
// exception test).
__device__ __forceinline__ void hist8c(uint4 r, unsigned LO2, unsigned HI2, int* shb, unsigned (&cl)[4]) {
    const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const unsigned c = __vmins2(__vmaxs2(w[j], LO2), HI2);
        cl[j] = c;
        atomicAdd(shb + (int)(short)(c & 0xffffu), 1);
        atomicAdd(shb + (((int)c) >> 16), 1);
    }
}

// n voxels at src into the block histogram. kBin: Algorithm 1 is applied in
// the same pass with a predicted threshold (mask8 below), writing dst; kExc:
// the voxels near that threshold are also listed (ExcCtx).
template <bool kBin, bool kExc>
__device__ void hist_tile(const int16_t* __restrict__ src, long long n, int lo, int hi, int* shb,
                          unsigned long long pol, uint8_t* __restrict__ dst, unsigned T2, bool le, int T,
                          const ExcCtx& ex) {
    const int tid = threadIdx.x;
    const unsigned LO2 = ((unsigned)lo & 0xffffu) * 0x10001u;
    const unsigned HI2 = ((unsigned)hi & 0xffffu) * 0x10001u;
    const int head = (int)lmin(n, ((16 - ((uintptr_t)src & 15)) & 15) >> 1);
    if (tid < head) {
        const int x = src[tid];
        const int c = clamp_level(x, lo, hi);
        atomicAdd(shb + c, 1);
        if (kBin) dst[tid] = (uint8_t)(((x <= T) == le) ? 1 : 0);
        if (kExc) exc_append1(ex, ex.pos0 + tid, c);
    }
    const uint4* v = reinterpret_cast<const uint4*>(src + head);
    uint8_t* d = dst + head;
    const long long nv = (n - head) >> 3;
    const long long p0 = ex.pos0 + head;
    long long i = tid;
    unsigned cl[4];
    for (; i + 3 * kSegThreads < nv; i += 4 * kSegThreads) {
        const uint4 r0 = ld_v4_policy(v + i, pol);
        const uint4 r1 = ld_v4_policy(v + i + kSegThreads, pol);
        const uint4 r2 = ld_v4_policy(v + i + 2 * kSegThreads, pol);
        const uint4 r3 = ld_v4_policy(v + i + 3 * kSegThreads, pol);
        if (kBin) {
            st_stream(d + i * 8, mask8(r0, T2, le));
            st_stream(d + (i + kSegThreads) * 8, mask8(r1, T2, le));
            st_stream(d + (i + 2 * kSegThreads) * 8, mask8(r2, T2, le));
            st_stream(d + (i + 3 * kSegThreads) * 8, mask8(r3, T2, le));
        }
        hist8c(r0, LO2, HI2, shb, cl);
        if (kExc) exc_append8(ex, cl, p0 + i * 8);
        hist8c(r1, LO2, HI2, shb, cl);
        if (kExc) exc_append8(ex, cl, p0 + (i + kSegThreads) * 8);
        hist8c(r2, LO2, HI2, shb, cl);
        if (kExc) exc_append8(ex, cl, p0 + (i + 2 * kSegThreads) * 8);
        hist8c(r3, LO2, HI2, shb, cl);
        if (kExc) exc_append8(ex, cl, p0 + (i + 3 * kSegThreads) * 8);
    }
    for (; i < nv; i += kSegThreads) {
        const uint4 r = ld_v4_policy(v + i, pol);
        if (kBin) st_stream(d + i * 8, mask8(r, T2, le));
        hist8c(r, LO2, HI2, shb, cl);
        if (kExc) exc_append8(ex, cl, p0 + i * 8);
    }
    const long long t0 = head + (nv << 3);
    if (t0 + tid < n) {
        const int x = src[t0 + tid];
        const int c = clamp_level(x, lo, hi);
        atomicAdd(shb + c, 1);
        if (kBin) dst[t0 + tid] = (uint8_t)(((x <= T) == le) ? 1 : 0);
        if (kExc) exc_append1(ex, ex.pos0 + t0 + tid, c);
    }
}

// Algorithm 1 over n voxels. t < 0 (no valid threshold) writes zeros.
__device__ void bin_tile(const int16_t* __restrict__ src, uint8_t* __restrict__ dst, long long n, int t, int lo,
                         int L, int shift, int polarity, unsigned long long pol) {
    const int tid = threadIdx.x;
    const int T = bin_threshold(t, lo, L, shift);
    const unsigned T2 = ((unsigned)T & 0xffffu) * 0x10001u;
    const bool le = polarity == 0;
    const bool none = t < 0;
    auto one = [&](int x) -> uint8_t { return none ? 0 : (uint8_t)(((x <= T) == le) ? 1 : 0); };
    const int head = (int)lmin(n, ((16 - ((uintptr_t)src & 15)) & 15) >> 1);
    if (tid < head) dst[tid] = one(src[tid]);
    const uint4* v = reinterpret_cast<const uint4*>(src + head);
    uint8_t* d = dst + head;
    const long long nv = (n - head) >> 3;
    long long i = tid;
    for (; i + 3 * kSegThreads < nv; i += 4 * kSegThreads) {
        const uint4 r0 = ld_v4_policy(v + i, pol);
        const uint4 r1 = ld_v4_policy(v + i + kSegThreads, pol);
        const uint4 r2 = ld_v4_policy(v + i + 2 * kSegThreads, pol);
        const uint4 r3 = ld_v4_policy(v + i + 3 * kSegThreads, pol);
        st_stream(d + i * 8, none ? make_uint2(0u, 0u) : mask8(r0, T2, le));
        st_stream(d + (i + kSegThreads) * 8, none ? make_uint2(0u, 0u) : mask8(r1, T2, le));
        st_stream(d + (i + 2 * kSegThreads) * 8, none ? make_uint2(0u, 0u) : mask8(r2, T2, le));
        st_stream(d + (i + 3 * kSegThreads) * 8, none ? make_uint2(0u, 0u) : mask8(r3, T2, le));
    }
    for (; i < nv; i += kSegThreads) st_stream(d + i * 8, none ? make_uint2(0u, 0u) : mask8(ld_v4_policy(v + i, pol), T2, le));
    const long long t0 = head + (nv << 3);
    if (t0 + tid < n) dst[t0 + tid] = one(src[t0 + tid]);
}

// ------------------------------------------------------------ scheduling

struct Work {
    int kind;   // 0 none, 1 histogram, 2 binarise
    int group;
    int tile;
    int t;      // binarise: threshold (-2: its wait ran out, skip); histogram:
                // predicted threshold to binarise with in the same pass (-1: none)
};

__device__ __forceinline__ int group_tiles(const SegArgs& a, int g) {
    return a.groups != nullptr ? a.groups[g].ntiles : a.ntiles;
}

// Histogram work item k -> (group, tile). Batches: binary search over the
// groups' first-tile offsets.
__device__ __forceinline__ void locate(const SegArgs& a, unsigned k, int& g, int& tile) {
    if (a.groups == nullptr) {
        g = (int)(k / (unsigned)a.ntiles);
        tile = (int)(k % (unsigned)a.ntiles);
        return;
    }
    int lo = 0, hi = a.ngroups - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((unsigned)a.groups[mid].tile_off <= k) lo = mid; else hi = mid - 1;
    }
    g = lo;
    tile = (int)(k - (unsigned)a.groups[lo].tile_off);
}

// Binarise queue entries: bits 40..63 the launch tag (1 + epoch mod
// 0xffffff: never 0), bits 20..39 the group, bits 0..19 the tile. An entry
// is valid for this launch once its tag matches. The block that takes an
// entry clears it, and after a launch whose waits ran out the last block
// clears the whole queue, so no entry outlives its launch and a tag can
// never be matched by an entry of an earlier launch, however often the tag
// wraps.
__device__ __forceinline__ unsigned bq_tag(int epoch) { return (unsigned)epoch % 0xffffffu + 1u; }
__device__ __forceinline__ unsigned long long bq_pack(int epoch, int g, int tile) {
    return ((unsigned long long)bq_tag(epoch) << 40) | ((unsigned long long)g << 20) | (unsigned)tile;
}
__device__ __forceinline__ bool bq_valid(unsigned long long e, int epoch) {
    return (unsigned)(e >> 40) == bq_tag(epoch);
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Predicted threshold of group g for this launch: the first histogram tile
// of the group to be scheduled fixes it (compare-and-swap on the group's
// slot) to the threshold found most recently in this launch, or to -1 (no
// prediction, the first pass only counts) when none is found yet. Values
// carry the launch tag, so nothing from an earlier launch is used.
__device__ __forceinline__ int group_hint(const SegArgs& a, int epoch, int g) {
    const unsigned long long tag = (unsigned long long)(unsigned)(epoch + 1) << 32;
    const unsigned long long hmask = 0xffffffff00000000ull;
    const unsigned long long cur = *(volatile unsigned long long*)&a.hdr->latest;
    const int t = (cur & hmask) == tag ? (int)(cur & 0xffffffffu) - 1 : -1;
    unsigned long long old = *(volatile unsigned long long*)&a.that[g];
    if ((old & hmask) != tag) {
        const unsigned long long prev = atomicCAS(&a.that[g], old, tag | (unsigned)(t + 1));
        if (prev == old) return t;
        old = prev;
    }
    return (old & hmask) == tag ? (int)(old & 0xffffffffu) - 1 : -1;
}

constexpr int kNoopTile = 0xfffff;   // queue entry of a group whose first-pass mask is exact
constexpr int kPatchItem = 0x80000;  // queue entry: rewrite a share of the group's listed voxels

// A group's region of the exception pool: 1/32 of the voxels its tiles span,
// at the offset of its first tile (so regions never overlap).
__device__ __forceinline__ long long exc_off_of(const SegArgs& a, int g) {
    const long long t0 = a.groups != nullptr ? a.groups[g].tile_off : (long long)g * a.ntiles;
    return (t0 * a.tile_vox) >> 5;
}
__device__ __forceinline__ long long exc_cap_of(const SegArgs& a, int g) {
    return ((long long)group_tiles(a, g) * a.tile_vox) >> 5;
}

// Per-block scheduler state (lane 0 of the scheduler warp).
struct SchedState {
    long long pend;   // claimed binarise queue position not yet published (-1: none)
    bool b_turn;      // alternate histogram and binarise items when both exist
};

// The next work item of this block (run by the scheduler lane).
//
// Histogram tiles come from one counter. When the block that completes a
// group has published its threshold, it appends the group's binarise tiles
// to a flat queue (one atomicAdd reserves the positions). Schedulers claim
// queue positions with a single atomicAdd each; a claim made before the
// position is published is kept pending while the scheduler keeps handing
// out histogram tiles, so claims never block histogram progress. When both
// kinds are available, a block alternates between them, which keeps each
// slice's re-read close behind its first read (so it hits L2). Once every
// histogram tile is taken, the scheduler waits (bounded) for its pending
// position.
__device__ Work next_work(const SegArgs& a, int epoch, SchedState& st) {
    Work w{0, 0, 0, 0};
    ScratchHeader* h = a.hdr;
    if (a.phases == kPhaseHist) {
        const unsigned k = atomicAdd(&h->h_next, 1u);
        if (k < a.ntotal) { w.kind = 1; locate(a, k, w.group, w.tile); w.t = -1; }
        return w;
    }
    if (a.phases == kPhaseBin) {
        const unsigned k = atomicAdd(&h->b_next, 1u);
        if (k < a.ntotal) {
            int tile;
            locate(a, k, w.group, tile);
            w.kind = 2;
            w.tile = group_tiles(a, w.group) - 1 - tile;
            w.t = a.t_in[(long long)w.group * a.t_stride];
        }
        return w;
    }
    for (;;) {
        if (st.pend >= 0) {
            const unsigned long long e = ld_acquire_u64(&a.bq[st.pend]);
            if (bq_valid(e, epoch)) {
                a.bq[st.pend] = 0ull;   // taken: no later launch can see it
                const int g = (int)((e >> 20) & 0xfffff), tile = (int)(e & 0xfffff);
                if (tile == kNoopTile) {   // nothing to re-binarise
                    st.pend = -1;
                    continue;
                }
                if (g >= a.ngroups || (tile & (kPatchItem - 1)) >= group_tiles(a, g)) {
                    // not an entry this launch wrote: give it up, the call reports TIMEOUT
                    atomicExch(&h->err, 1);
                    st.pend = -1;
                    continue;
                }
                w.kind = 2;
                w.group = g;
                w.tile = tile;
                w.t = __ldcg(&a.t_out[w.group]);
                st.pend = -1;
                st.b_turn = false;
                return w;
            }
        } else if (st.b_turn && *(volatile unsigned*)&h->b_next < *(volatile unsigned*)&h->b_tail) {
            const unsigned k = atomicAdd(&h->b_next, 1u);
            if (k < a.ntotal) { st.pend = k; continue; }
        }
        if (*(volatile unsigned*)&h->h_next < a.ntotal) {
            const unsigned k = atomicAdd(&h->h_next, 1u);
            if (k < a.ntotal) {
                w.kind = 1;
                locate(a, k, w.group, w.tile);
                w.t = -1;   // the prediction is fixed when the tile starts (workers)
                st.b_turn = true;
                return w;
            }
        }
        // every histogram tile is taken
        if (st.pend < 0) {
            const unsigned k = atomicAdd(&h->b_next, 1u);
            if (k >= a.ntotal) return w;   // every binarise tile is claimed: done
            st.pend = k;
        }
        // wait (bounded) for the pending position to be published
        const unsigned long long t0 = globaltimer_ns();
        unsigned ns = 64;
        while (!bq_valid(ld_acquire_u64(&a.bq[st.pend]), epoch)) {
            if (globaltimer_ns() - t0 > a.timeout_ns) {
                // its group never completed in time: give the position up;
                // the group reports TIMEOUT
                atomicExch(&h->err, 1);
                st.pend = -1;
                break;
            }
            __nanosleep(ns);
            if (ns < 2048) ns <<= 1;
        }
    }
}

// ------------------------------------------------------------ the kernel

constexpr int kBlockThreads = kSegThreads + 32;        // 544
constexpr int kBarHandoff = 1;                         // scheduler + workers
constexpr int kBarWork = 2;                            // workers only

__device__ __forceinline__ void work_sync() {
    asm volatile("bar.sync %0, %1;" ::"n"(kBarWork), "n"(kSegThreads) : "memory");
}
__device__ __forceinline__ void handoff_sync() {
    asm volatile("bar.sync %0, %1;" ::"n"(kBarHandoff), "n"(kBlockThreads) : "memory");
}
using WorkSync = NamedSync<kBarWork, 0>;

// Dynamic shared memory: the block histogram sh[kMaxBins], then the
// search's scratch: double-float terms sT[kMaxBins] and the compacted
// (level, count) list sIC[kMaxBins].
__global__ void __launch_bounds__(kBlockThreads, kSegMinBlocks) k_segment1d(const SegArgs a) {
    extern __shared__ int4 smem_raw[];
    int* sh = reinterpret_cast<int*>(smem_raw);
    float2* sT = reinterpret_cast<float2*>(reinterpret_cast<char*>(smem_raw) + kMaxBins * sizeof(int));
    int2* sIC = reinterpret_cast<int2*>(sT + kMaxBins);
    __shared__ SearchSmem ssm;
    __shared__ Work s_work[2];
    __shared__ int s_last;
    __shared__ int s_any;
    __shared__ int s_exc_n, s_exc_cnt, s_exc_base, s_hint;
    // a tile's exceptions (the search's scratch, sT and sIC, is free then)
    unsigned long long* sexc = reinterpret_cast<unsigned long long*>(sT);
    const int tid = threadIdx.x;
    const int epoch = *(volatile int*)&a.hdr->epoch;

    __shared__ DfTables sdf;
    for (int i = tid; i < kMaxBins; i += kBlockThreads) sh[i] = 0;
    df_stage(&sdf, static_cast<const DfTables*>(a.df_tables), tid, kBlockThreads);
    if (tid == 0) s_exc_n = 0;
    __syncthreads();

    if (tid >= kSegThreads) {
        // ================= scheduler warp: prepares item i + 1 while the
        // workers process item i (double-buffered hand-off)
        SchedState st{-1, false};
        for (int i = 0;; ++i) {
            if (tid == kSegThreads) s_work[i & 1] = next_work(a, epoch, st);
            handoff_sync();
            if (s_work[i & 1].kind == 0) break;
        }
    } else {
        // ================= workers
        const DfTables* dft = &sdf;
        const int hi = a.lo + a.L - 1 > 32767 ? 32767 : a.lo + a.L - 1;
        int* shb = sh - a.lo;   // shb[v] is level v - lo
        const unsigned long long pol_keep = policy_evict_last();
        const unsigned long long pol_drop = policy_evict_first();
        for (int i = 0;; ++i) {
            handoff_sync();
            Work w = s_work[i & 1];
            if (w.kind == 0) break;
            // checked build: an item outside the groups or its group's tiles
            // is skipped by every worker (w is the same for the whole block)
            if (kCheckedBuild && (!in_range(w.group, a.ngroups, a.check, kSiteSegGroup) ||
                                  (!(w.kind == 2 && (w.tile & kPatchItem)) &&
                                   !in_range(w.tile, group_tiles(a, w.group), a.check, kSiteSegTile))))
                continue;
            const int16_t* gvol;
            uint8_t* gmask;
            long long gn;
            if (a.groups != nullptr) {
                const GroupDesc gd = a.groups[w.group];
                gvol = gd.vol; gmask = gd.mask; gn = gd.nvox;
            } else {
                gvol = a.vol + (long long)w.group * a.group_vox;
                gmask = a.mask + (long long)w.group * a.group_vox;
                gn = a.group_vox;
            }
            const long long off = (long long)w.tile * a.tile_vox;
            const long long n = lmin((long long)a.tile_vox, gn - off);
            if (w.kind == 1 && a.spec) {
                // the group's predicted threshold: given per group, or fixed by
                // its first tile to start
                if (tid == 0) {
                    if (a.hint != nullptr) {
                        const int hh = a.hint[w.group];
                        *(volatile unsigned long long*)&a.that[w.group] =
                            ((unsigned long long)(unsigned)(epoch + 1) << 32) | (unsigned)(hh + 1);
                        s_hint = hh;
                    } else {
                        s_hint = group_hint(a, epoch, w.group);
                    }
                }
                work_sync();
                w.t = s_hint;
            }
            if (w.kind == 1) {
                ExcCtx ex;
                ex.pos0 = off;
                const bool with_exc = w.t >= 0 && a.exc_w > 0;
                if (w.t >= 0) {
                    const int T = bin_threshold(w.t, a.lo, a.L, 0);
                    const unsigned T2 = ((unsigned)T & 0xffffu) * 0x10001u;
                    if (with_exc) {
                        ex.list = sexc;
                        ex.n = &s_exc_n;
                        ex.cap = kExcSmem;
                        ex.lo = a.lo;
                        ex.wbase = w.t - a.exc_w + 1;
                        const int wl = a.lo + ex.wbase, wh = a.lo + w.t + a.exc_w;   // window as values
                        ex.wlo = wl < a.lo ? a.lo : wl;
                        ex.whi = wh > hi ? hi : wh;
                        ex.wlo2 = ((unsigned)ex.wlo & 0xffffu) * 0x10001u;
                        ex.whi2 = ((unsigned)ex.whi & 0xffffu) * 0x10001u;
                        hist_tile<true, true>(gvol + off, n, a.lo, hi, shb, pol_keep, gmask + off, T2,
                                              a.polarity == 0, T, ex);
                    } else {
                        hist_tile<true, false>(gvol + off, n, a.lo, hi, shb, pol_keep, gmask + off, T2,
                                               a.polarity == 0, T, ex);
                    }
                } else {
                    hist_tile<false, false>(gvol + off, n, a.lo, hi, shb, pol_keep, nullptr, 0u, true, 0, ex);
                }
                work_sync();
                if (with_exc) {
                    // this tile's exceptions into the group's list
                    if (tid == 0) {
                        const int ne = s_exc_n;
                        s_exc_n = 0;
                        s_exc_cnt = ne;
                        // a tile list that overflowed shared memory marks the group
                        // as overflowed (bit 30: the count then exceeds any region)
                        s_exc_base = ne > kExcSmem ? atomicOr(&a.exc_n[w.group], 0x40000000)
                                                   : atomicAdd(&a.exc_n[w.group], ne);
                    }
                    work_sync();
                    const int ne = s_exc_cnt, eb = s_exc_base;
                    const long long cap = exc_cap_of(a, w.group);
                    unsigned long long* gl = a.exc + exc_off_of(a, w.group);
                    if (ne <= kExcSmem)
                        for (int k = tid; k < ne && eb + k < cap; k += kSegThreads) gl[eb + k] = sexc[k];
                }
                // add the block histogram to the group's, leave sh zeroed
                int* gh = a.ghist + (long long)w.group * a.L;
                for (int b = tid; b < a.L; b += kSegThreads) {
                    const int c = sh[b];
                    sh[b] = 0;
                    if (c) atomicAdd(&gh[b], c);
                }
                if (a.phases & kPhaseSearch) {
                    __threadfence();
                    work_sync();
                    if (tid == 0) {
                        int last = 0;
                        if ((a.flags & 1u) && w.group == 0 && w.tile == 0) atomicExch(&a.hdr->err, 1);
                        else last = atomicAdd(&a.arrive[w.group], 1) == group_tiles(a, w.group) - 1;
                        s_last = last;
                    }
                    work_sync();
                    if (s_last) {
                        // this block completed the group: search it and publish
                        __threadfence();
                        SearchResult r =
                            (a.ptab != nullptr && gn == a.ptab_n && a.curve == nullptr)
                                ? search1d_fast<WorkSync>(gh, a.L, a.q, a.ptab, a.ptab_n, ssm, sIC, sT, dft)
                                : search1d_block<WorkSync>(
                                      gh, a.L, a.q, a.curve ? a.curve + (long long)w.group * (a.L - 1) : nullptr,
                                      ssm, sT, sIC, dft);
                        // the first pass binarised with a predicted threshold t^:
                        // its mask is exact when no voxel has a level between
                        // t^ and t (no voxel changes side)
                        bool exact = false, patch = false;
                        if (a.spec) {
                            const unsigned long long hv = *(volatile unsigned long long*)&a.that[w.group];
                            const int th = (hv >> 32) == (unsigned long long)(unsigned)(epoch + 1)
                                               ? (int)(hv & 0xffffffffu) - 1 : -1;
                            if (th >= 0 && r.t >= 0) {
                                const int b0 = (th < r.t ? th : r.t) + 1, b1 = th < r.t ? r.t : th;
                                int any = 0;
                                for (int b = b0 + tid; b <= b1; b += kSegThreads) any |= __ldcg(gh + b);
                                if (tid == 0) s_any = 0;
                                work_sync();
                                if (any) s_any = 1;
                                work_sync();
                                exact = s_any == 0;
                                const long long ne = a.exc_w > 0 ? *(volatile int*)&a.exc_n[w.group] : 0;
                                const int dt = r.t - th;
                                // every voxel that changes side has a level in
                                // (b0 - 1, b1]; inside the window it is listed, and
                                // the group's work items rewrite the listed voxels
                                patch = !exact && a.exc_w > 0 && dt >= -a.exc_w && dt <= a.exc_w &&
                                        ne <= exc_cap_of(a, w.group);
                                exact = exact || patch;
                            }
                        }
                        for (int b = tid; b < a.L; b += kSegThreads) gh[b] = 0;   // scratch left zeroed
                        const int nt = group_tiles(a, w.group);
                        if (tid == 0) {
                            a.t_out[w.group] = r.t;
                            a.phi_out[w.group] = r.phi;
                            a.status[w.group] = r.status | (exact ? TSALLIS_STATUS_FIRST_PASS_EXACT : 0);
                            a.arrive[w.group] = 0;
                            a.done_flag[w.group] = epoch + 1;
                            if (exact && !patch) atomicAdd(&a.bdone[w.group], nt);
                            if (r.t >= 0)
                                *(volatile unsigned long long*)&a.hdr->latest =
                                    ((unsigned long long)(unsigned)(epoch + 1) << 32) | (unsigned)(r.t + 1);
                            __threadfence();
                            s_last = (int)atomicAdd(&a.hdr->b_tail, (unsigned)nt);
                        }
                        work_sync();
                        // the group's binarise tiles enter the queue, most
                        // recently read tile first (no-op entries when the
                        // first-pass mask is exact: the queue length stays
                        // the number of tiles, which is how blocks know when
                        // all work is done)
                        const int base = s_last;
                        for (int j = tid; j < nt; j += kSegThreads)
                            if (in_range(base + j, a.ntotal, a.check, kSiteSegQueue))
                            st_release_u64(&a.bq[base + j],
                                           bq_pack(epoch, w.group,
                                                   patch ? (kPatchItem | j) : exact ? kNoopTile : nt - 1 - j));
                    }
                }
            } else if (w.t != -2 && (w.tile & kPatchItem)) {
                // rewrite a share of the group's listed voxels with Algorithm 1 at t
                const int k = w.tile & (kPatchItem - 1);
                const int nt = group_tiles(a, w.group);
                const long long ne = *(volatile int*)&a.exc_n[w.group];
                const long long per = (ne + nt - 1) / nt;
                const long long e0 = (long long)k * per, e1 = lmin(ne, e0 + per);
                const unsigned long long hv = *(volatile unsigned long long*)&a.that[w.group];
                const int th = (int)(hv & 0xffffffffu) - 1;
                const int wbase = th - a.exc_w + 1;
                const int b0 = (th < w.t ? th : w.t) + 1, b1 = th < w.t ? w.t : th;
                const bool le = a.polarity == 0;
                const unsigned long long* gl = a.exc + exc_off_of(a, w.group);
                for (long long e = e0 + tid; e < e1; e += kSegThreads) {
                    const unsigned long long x = __ldcg(gl + e);
                    const int lev = (int)(x & 0xffffu) + wbase;
                    if (lev >= b0 && lev <= b1) gmask[x >> 16] = ((lev <= w.t) == le) ? 1 : 0;
                }
                if (tid == 0) atomicAdd(&a.bdone[w.group], 1);
            } else if (w.t != -2) {
                bin_tile(gvol + off, gmask + off, n, w.t, a.lo, a.L, a.bin_shift, a.polarity, pol_drop);
                if (tid == 0 && (a.phases & kPhaseSearch)) atomicAdd(&a.bdone[w.group], 1);
            }
            work_sync();
        }
    }

    // exit: the last block restores the scratch for the next launch
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned d = atomicAdd(&a.hdr->done, 1u);
        s_last = (d == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        const bool err = *(volatile int*)&a.hdr->err != 0;
        if (a.phases & kPhaseSearch) {
            for (int g = tid; g < a.ngroups; g += kBlockThreads) {
                if (err && (*(volatile int*)&a.done_flag[g] != epoch + 1 ||
                            *(volatile int*)&a.bdone[g] != group_tiles(a, g))) {
                    // never searched (a skipped arrival) or not fully binarised in time
                    a.t_out[g] = -1;
                    a.phi_out[g] = 0.f;
                    a.status[g] = 5; /* TSALLIS_ERR_TIMEOUT */
                }
                a.bdone[g] = 0;
                if (a.exc_w > 0) a.exc_n[g] = 0;
                if (err) a.arrive[g] = 0;
            }
            if (err) {
                // clear every group's histogram
                const long long tot = (long long)a.ngroups * a.L;
                for (long long i = tid; i < tot; i += kBlockThreads) a.ghist[i] = 0;
            }
        }
        // positions given up on a timed-out wait may be published late:
        // clear the queue so that nothing of this launch outlives it
        if (err && a.bq)
            for (unsigned i = tid; i < a.ntotal; i += kBlockThreads) a.bq[i] = 0ull;
        __syncthreads();
        if (tid == 0) {
            a.hdr->h_next = 0;
            a.hdr->b_next = 0;
            a.hdr->b_tail = 0;
            a.hdr->done = 0;
            a.hdr->err = 0;
            a.hdr->epoch = epoch + 1;
            __threadfence();
        }
    }
}

__global__ void __launch_bounds__(kSearchThreads) k_search1d(const int32_t* __restrict__ hist, long long nh, int L,
                                                             float q, int32_t* __restrict__ t_out,
                                                             float* __restrict__ phi_out,
                                                             int32_t* __restrict__ status, float* __restrict__ curve,
                                                             const DfTables* __restrict__ dft) {
    __shared__ SearchSmem sm;
    __shared__ DfTables sdf;
    extern __shared__ int4 smem_search[];
    float2* sT = reinterpret_cast<float2*>(smem_search);
    int2* sIC = reinterpret_cast<int2*>(sT + kMaxBins);
    df_stage(&sdf, dft, threadIdx.x, blockDim.x);
    __syncthreads();
    for (long long g = blockIdx.x; g < nh; g += gridDim.x) {
        SearchResult r = search1d_block<BlockSync>(hist + g * L, L, q, curve ? curve + g * (L - 1) : nullptr, sm,
                                                   sT, sIC, &sdf);
        if (threadIdx.x == 0) {
            t_out[g] = r.t;
            phi_out[g] = r.phi;
            status[g] = r.status;
        }
        __syncthreads();
    }
}

// The window search, one block per histogram (search1d_window).
__global__ void __launch_bounds__(kSearchThreads) k_search1d_window(const int32_t* __restrict__ hist, long long nh,
                                                                    int L, float q, const int32_t* __restrict__ cand,
                                                                    int k, int32_t* __restrict__ t_out,
                                                                    float* __restrict__ phi_out,
                                                                    int32_t* __restrict__ status,
                                                                    const DfTables* __restrict__ dft) {
    __shared__ SearchSmem sm;
    __shared__ WindowSmem ws;
    __shared__ DfTables sdf;
    extern __shared__ int4 smem_window[];
    float2* sW = reinterpret_cast<float2*>(smem_window);
    float2* sQ = sW + kMaxBins;
    df_stage(&sdf, dft, threadIdx.x, blockDim.x);
    __syncthreads();
    for (long long g = blockIdx.x; g < nh; g += gridDim.x) {
        SearchResult r = search1d_window<BlockSync>(hist + g * L, L, q, cand + g * k, k, sm, ws, sW, sQ, &sdf);
        if (threadIdx.x == 0) {
            t_out[g] = r.t;
            phi_out[g] = r.phi;
            status[g] = r.status;
        }
        __syncthreads();
    }
}

cudaError_t launch_search1d_window(const int32_t* hist, long long nh, int L, float q, const int32_t* cand, int k,
                                   int32_t* t, float* phi, int32_t* status, const void* tables, cudaStream_t s) {
    if (nh <= 0) return cudaSuccess;
    const int grid = (int)(nh < 65535 ? nh : 65535);
    k_search1d_window<<<grid, kSearchThreads, 2 * kMaxBins * (int)sizeof(float2), s>>>(
        hist, nh, L, q, cand, k, t, phi, status, static_cast<const DfTables*>(tables));
    return cudaGetLastError();
}

// Test hook: the double-float power and log2 used by the search, for
// checking their accuracy against an independent double-precision result.
__global__ void k_probe_dfmath(const unsigned* __restrict__ h, long long n, unsigned N, float q,
                               double* __restrict__ pw, double* __restrict__ lg, const DfTables* __restrict__ T) {
    const F2 LN = df_log2_u32(N, T);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned x = h[i];
        pw[i] = (x >= 1u && x <= N) ? df_to_double(df_pow_ratio<true>(x, LN, q, T)) * 0x1p-64 : 0.0;
        lg[i] = x >= 1u ? df_to_double(df_log2_u32(x, T)) : 0.0;
    }
}

// log2(h) as float pairs for 0 <= h <= n - 1 (h = 0 gives 0).
__global__ void k_build_log2_table(float2* __restrict__ lt, int n, const DfTables* __restrict__ T) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const F2 v = i >= 1 ? df_log2_u32((unsigned)i, T) : F2{0.f, 0.f};
        lt[i] = make_float2(v.hi, v.lo);
    }
}

// Terms of the table search: tab[n] = 2^64 (n / n_max)^q (q = 1: n log2 n)
// as float pairs, the same values the search computes otherwise.
__global__ void k_build_pow_table(float2* __restrict__ tab, long long n_max, float q, const DfTables* __restrict__ T) {
    const F2 LN = df_log2_count<false>((unsigned)n_max, T);
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n <= n_max;
         n += (long long)gridDim.x * blockDim.x) {
        F2 v{0.f, 0.f};
        if (n > 0) v = q == 1.0f ? df_hlog2h<false>((unsigned)n, T) : df_pow_ratio<false>((unsigned)n, LN, q, T);
        tab[n] = make_float2(v.hi, v.lo);
    }
}

cudaError_t build_pow_table(float2* tab, long long n_max, float q, const void* tables, cudaStream_t s) {
    const long long blocks = (n_max + 256) / 256;
    k_build_pow_table<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(tab, n_max, q,
                                                                          static_cast<const DfTables*>(tables));
    return cudaGetLastError();
}

cudaError_t build_log2_table(void* lt, int n, const void* tables, cudaStream_t s) {
    k_build_log2_table<<<(n + 255) / 256, 256, 0, s>>>(static_cast<float2*>(lt), n,
                                                       static_cast<const DfTables*>(tables));
    return cudaGetLastError();
}

cudaError_t launch_probe_dfmath(const unsigned* h, long long n, unsigned N, float q, double* pw, double* lg,
                                const void* tables, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_probe_dfmath<<<256, 256, 0, s>>>(h, n, N, q, pw, lg, static_cast<const DfTables*>(tables));
    return cudaGetLastError();
}

// Group table of a batch: one thread per group, volume found by binary
// search over the volumes' first groups.
__global__ void k_expand_groups(const ExpandArgs a) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.ngroups) return;
    const int gg = a.v[0].group_off + g;
    int lo = 0, hi = a.nvol - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.v[mid].group_off <= gg) lo = mid; else hi = mid - 1;
    }
    const BatchVolDesc& v = a.v[lo];
    const int k = gg - v.group_off;
    GroupDesc d;
    d.vol = v.vol + (long long)k * v.gvox;
    d.mask = v.mask + (long long)k * v.gvox;
    d.nvox = v.gvox;
    d.ntiles = v.ntiles;
    d.tile_off = v.tile_off + k * v.ntiles;
    a.out[gg] = d;
}

cudaError_t launch_expand_groups(const ExpandArgs& a, cudaStream_t s) {
    if (a.ngroups <= 0) return cudaSuccess;
    k_expand_groups<<<(a.ngroups + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

int segment1d_threads() { return kBlockThreads; }
int segment1d_smem_bytes(int L, int copies) {
    (void)L;
    (void)copies;
    return kMaxBins * (int)(sizeof(int) + sizeof(float2) + sizeof(int2));
}

size_t df_tables_bytes() { return sizeof(DfTables); }

// Host-side construction of the double-float tables (double precision libm,
// split into float pairs).
void df_tables_fill(void* host, const void* log2_table, int log2_table_max) {
    DfTables* t = static_cast<DfTables*>(host);
    t->lt = static_cast<const float2*>(log2_table);
    t->lt_max = log2_table_max;
    for (int j = 0; j < 128; ++j) {
        const double c = 1.0 + (j + 0.5) / 128.0;
        const float inv = (float)(1.0 / c);
        const double lt = -std::log2((double)inv);
        const float hi = (float)lt;
        t->lg[j] = make_float4(inv, hi, (float)(lt - (double)hi), 0.f);
    }
    for (int j = 0; j < 65; ++j) {
        const double v = std::exp2((j - 32) / 64.0);
        const float hi = (float)v;
        t->ex[j] = make_float2(hi, (float)(v - (double)hi));
    }
}

// Opts every kernel variant into the shared memory it uses (above the
// default 48 KB). Per device: call with that device current.
cudaError_t segment1d_prepare() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_segment1d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  segment1d_smem_bytes(kMaxBins, 1))) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_search1d_window, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  2 * kMaxBins * (int)sizeof(float2))) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_search1d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kMaxBins * (int)(sizeof(float2) + sizeof(int2)));
}

cudaError_t segment1d_occupancy(int copies, int L, int* blocks_per_sm) {
    (void)L;
    if (copies != 1) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_segment1d, kBlockThreads,
                                                         segment1d_smem_bytes(kMaxBins, 1));
}

cudaError_t launch_segment1d(const SegArgs& a, int grid, int copies, cudaStream_t s) {
    if (copies != 1) return cudaErrorInvalidValue;
    k_segment1d<<<grid, kBlockThreads, segment1d_smem_bytes(kMaxBins, 1), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_search1d(const int32_t* hist, long long nh, int L, float q, int32_t* t, float* phi,
                            int32_t* status, float* curve, const void* tables, cudaStream_t s) {
    if (nh <= 0) return cudaSuccess;
    const int grid = (int)(nh < 65535 ? nh : 65535);
    const int smem = kMaxBins * (int)(sizeof(float2) + sizeof(int2));
    k_search1d<<<grid, kSearchThreads, smem, s>>>(hist, nh, L, q, t, phi, status, curve,
                                                  static_cast<const DfTables*>(tables));
    return cudaGetLastError();
}

}  // namespace tsl
