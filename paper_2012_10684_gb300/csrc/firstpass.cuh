// First-pass pieces shared by the per-slice kernels that binarise while they
// count (seg_spec.cu, seg_pipe.cu): the voxel loop that counts a voxel into
// the block histogram, writes its mask at a predicted threshold t^
// (Algorithm 1) and lists it when its level lies in the window
// (t^ - w, t^ + w]; and the plain FP32 search that predicts t^ from a
// histogram. Blocks of 512 threads (16 warps) synchronised on named barrier
// 1.
#pragma once
#include <cstdint>

#include "common.cuh"
#include "search1d.cuh"
#include "kernels.h"

namespace tsl {
namespace fp {
namespace {   // internal to each kernel's translation unit

constexpr int kThreads = kSearchThreads;      // 512: 16 warps
constexpr int kWarps = kThreads / 32;
constexpr int kWarpBuf = 2 * kSpecWarpList;   // a warp's list buffer in shared memory (entries)
using Sync = NamedSync<1, 0>;

__device__ __forceinline__ unsigned prmt(unsigned a, unsigned b, unsigned s) {
    unsigned d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(s));
    return d;
}
__device__ __forceinline__ void block_sync() { Sync::sync(); }
__device__ __forceinline__ uint4 ld_stream(const void* p, unsigned long long pol) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p), "l"(pol));
    return r;
}

// ------------------------------------------------------------ voxel loop
//
// A voxel's histogram slot is the byte offset o = 4 level, level =
// clamp(v - lo, 0, L - 1). Two offsets are packed as 16-bit lanes (all
// below 0x8000), and the comparisons of Algorithm 1 and of the list window
// become one add per pair: with C = 0x8000 - o_T, bit 15 of (o + C) is set
// exactly when o >= o_T.

struct Tile {
    int C0;             // -4 lo
    int top;            // 4 (L - 1)
    unsigned MT2;       // mask: 0x8000 - 4 (t^ + 1), both lanes
    unsigned POL;       // 0x01010101 (mask = level <= t^) or 0
    unsigned WA2, WB2;  // window: 0x8000 - 4 (lower bound), 0x8000 - 4 (upper bound + 1)
    int wbase;          // level stored as 0 in a list entry (t^ - w + 1)
    bool bin;           // a prediction exists
};

// The loop constants for threshold prediction th (-1: none; the voxels are
// only counted) and window win, levels clamp(v - lo, 0, L - 1).
__device__ __forceinline__ Tile make_tile(int lo, int L, int th, int win, bool le) {
    Tile x;
    x.C0 = -4 * lo;
    x.top = 4 * (L - 1);
    x.bin = th >= 0;
    x.MT2 = (unsigned)(0x8000 - 4 * (th + 1)) * 0x10001u;
    x.POL = le ? 0x01010101u : 0u;
    const int wlo = th - win + 1, whi = th + win > L - 1 ? L - 1 : th + win;
    x.WA2 = (unsigned)(0x8000 - 4 * (wlo > 0 ? wlo : 0)) * 0x10001u;
    x.WB2 = (unsigned)(0x8000 - 4 * (whi + 1)) * 0x10001u;
    x.wbase = wlo;
    return x;
}

// A warp's list: entries gather in its shared-memory buffer and are copied
// to its region of global memory (wcap entries) whenever half the buffer is
// used. All counts are the same in every lane of the warp.
struct WarpList {
    unsigned* buf;      // shared memory, kWarpBuf entries
    unsigned* glob;     // the warp's region in global memory
    int n;              // entries in buf
    int g;              // entries copied to glob
    int cap;            // wcap
    bool over;          // the region overflowed while listing the current slice
};

__device__ __forceinline__ void list_spill(WarpList& wl) {
    const int lane = threadIdx.x & 31;
    if (wl.g + wl.n > wl.cap) {
        wl.over = true;
    } else {
        for (int e = lane; e < wl.n; e += 32) wl.glob[wl.g + e] = wl.buf[e];
        wl.g += wl.n;
    }
    wl.n = 0;
    __syncwarp();   // the buffer is read before it is written again
}

// The listed voxels among 8 (packed offsets o2[4]; inw: their window bits,
// bit 15 / 31 of each word, zero for lanes past the end).
__device__ __forceinline__ void list8(const Tile& x, const unsigned (&o2)[4], unsigned inw, unsigned pos,
                                      WarpList& wl) {
    const unsigned lane = threadIdx.x & 31u;
    if (__ballot_sync(0xffffffffu, inw != 0) == 0u) return;
    unsigned bits = 0;
    // bit 2j: low half of word j, bit 2j+1: its high half
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const unsigned m = (o2[j] + x.WA2) & ~(o2[j] + x.WB2);
        bits |= (((m >> 15) & 1u) | ((m >> 30) & 2u)) << (2 * j);
    }
    if (inw == 0) bits = 0;
    const unsigned cnt = __popc(bits);
    unsigned off = 0, tot = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const unsigned bb = __ballot_sync(0xffffffffu, (cnt >> b) & 1u);
        off += (unsigned)__popc(bb & ((1u << lane) - 1u)) << b;
        tot += (unsigned)__popc(bb) << b;
    }
    int k = wl.n + (int)off;   // below kWarpBuf: at most 256 entries join a buffer holding under 256
    wl.n += (int)tot;
    while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1;
        const unsigned o = (b & 1) ? (o2[b >> 1] >> 16) : (o2[b >> 1] & 0xffffu);
        wl.buf[k++] = ((pos + (unsigned)b) << 8) | (unsigned)((int)(o >> 2) - x.wbase);
    }
    if (wl.n >= kSpecWarpList) list_spill(wl);
}

// The listed 16-byte groups (8 voxels) of a warp: lanes whose group has a
// voxel in the window (any != 0) append the group's index.
__device__ __forceinline__ void list_group(bool any, unsigned g, WarpList& wl) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned bal = __ballot_sync(0xffffffffu, any);
    if (bal == 0u) return;
    if (any) wl.buf[wl.n + __popc(bal & ((1u << lane) - 1u))] = g;
    wl.n += __popc(bal);   // below kWarpBuf: at most 32 join a buffer holding under 256
    if (wl.n >= kSpecWarpList) list_spill(wl);
}

// 8 voxels: histogram, first-pass mask, window bits.
__device__ __forceinline__ void vox8(const Tile& x, uint4 r, char* shb, uint2& m, unsigned (&o2)[4],
                                     unsigned& inw) {
    const unsigned w[4] = {r.x, r.y, r.z, r.w};
    inw = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int a = (int)prmt(w[j], 0u, 0x9910u), b = ((int)w[j]) >> 16;   // the two int16 values
        const int oa = min(max(a * 4 + x.C0, 0), x.top), ob = min(max(b * 4 + x.C0, 0), x.top);
        atomicAdd(reinterpret_cast<int*>(shb + oa), 1);
        atomicAdd(reinterpret_cast<int*>(shb + ob), 1);
        o2[j] = prmt((unsigned)oa, (unsigned)ob, 0x5410u);
        inw |= (o2[j] + x.WA2) & ~(o2[j] + x.WB2);
    }
    // bit 15 of each lane of o + MT2: level >= t^ + 1; prmt replicates it
    // over a byte (selector nibbles 9, b, d, f: the signs of bytes 1, 3, 5, 7)
    const unsigned m0 = o2[0] + x.MT2, m1 = o2[1] + x.MT2, m2 = o2[2] + x.MT2, m3 = o2[3] + x.MT2;
    m.x = (prmt(m0, m1, 0xFDB9u) & 0x01010101u) ^ x.POL;
    m.y = (prmt(m2, m3, 0xFDB9u) & 0x01010101u) ^ x.POL;
    inw &= 0x80008000u;
}

// n voxels (a multiple of 8) of one slice at slice position p0: counted,
// and with a prediction binarised and listed (kGroups: the 16-byte groups
// with a voxel in the window, by index from src; else the voxels, by slice
// position and level).
template <bool kGroups>
__device__ void run_part(const Tile& x, const int16_t* __restrict__ src, uint8_t* __restrict__ dst, int n,
                         unsigned p0, char* shb, WarpList& wl, unsigned long long pol) {
    const int tid = threadIdx.x;
    const uint4* v = reinterpret_cast<const uint4*>(src);
    uint2* d = reinterpret_cast<uint2*>(dst);
    const int nv = n >> 3;
    constexpr int U = 4;
    int i0 = 0;
    for (; i0 + U * kThreads <= nv; i0 += U * kThreads) {
        uint4 r[U];
#pragma unroll
        for (int u = 0; u < U; ++u) r[u] = ld_stream(v + i0 + u * kThreads + tid, pol);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * kThreads + tid;
            uint2 m;
            unsigned o2[4], inw;
            vox8(x, r[u], shb, m, o2, inw);
            if (x.bin) {
                st_stream(d + i, m);
                if (kGroups) list_group(inw != 0, (unsigned)i, wl);
                else list8(x, o2, inw, p0 + (unsigned)i * 8u, wl);
            }
        }
    }
    for (; i0 < nv; i0 += kThreads) {
        const int i = i0 + tid;
        const bool in = i < nv;
        uint2 m;
        unsigned o2[4] = {0u, 0u, 0u, 0u}, inw = 0;
        if (in) vox8(x, ld_stream(v + i, pol), shb, m, o2, inw);
        if (x.bin) {
            if (in) st_stream(d + i, m);
            if (kGroups) list_group(in && inw != 0, (unsigned)i, wl);
            else list8(x, o2, in ? inw : 0u, p0 + (unsigned)i * 8u, wl);
        }
    }
}

// ------------------------------------------------------------ prediction

struct PredSmem {
    int wn[kWarps];     // non-empty levels per warp
    int wc[kWarps];
    float wp[kWarps], ws[kWarps];
    float bv[kWarps];
    int bi[kWarps];
};

// Plain FP32 exhaustive search over levels [0, L) of the block histogram,
// on the compacted list of its non-empty levels (sL: kMaxBins (level,
// count) pairs in shared memory). Terms h^q (h log2 h at q = 1),
// unnormalised:
//   phi(t) = (1 - (Q_1 / N_1^q)(Q_2 / N_2^q)) / (q - 1),
//   q = 1: (log2 N_1 - Q_1 / N_1) + (log2 N_2 - Q_2 / N_2),
// at every non-empty level with a non-empty class 2. Returns -1 when fewer
// than two levels are non-empty. Four barriers.
__device__ int predict1d(const int* __restrict__ hist, int L, float q, int2* __restrict__ sL, PredSmem& ps) {
    constexpr int R = kMaxBins / kThreads;   // 8
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int base = tid * R;
    const bool shannon = q == 1.0f;
    int c[R];
    int nz = 0;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        c[k] = base + k < L ? hist[base + k] : 0;
        nz += c[k] > 0;
    }
    int nzi = nz;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, nzi, d);
        if (lane >= d) nzi += o;
    }
    if (lane == 31) ps.wn[warp] = nzi;
    block_sync();
    int M = 0, pos = nzi - nz;
    for (int w = 0; w < kWarps; ++w) {
        const int v = ps.wn[w];
        if (w < warp) pos += v;
        M += v;
    }
#pragma unroll
    for (int k = 0; k < R; ++k)
        if (c[k] > 0) sL[pos++] = make_int2(base + k, c[k]);
    block_sync();
    // this thread's entries (a contiguous run), terms, run sums
    const int per = (M + kThreads - 1) / kThreads;
    const int j0 = min(tid * per, M), j1 = min(j0 + per, M);
    int cs = 0;
    float wsum = 0.f;
    for (int j = j0; j < j1; ++j) {
        const float f = (float)sL[j].y;
        cs += sL[j].y;
        wsum += shannon ? f * __log2f(f) : exp2f(q * __log2f(f));
    }
    int ci = cs;
    float pi = wsum, si = wsum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int oc = __shfl_up_sync(0xffffffffu, ci, d);
        const float op = __shfl_up_sync(0xffffffffu, pi, d);
        const float os = __shfl_down_sync(0xffffffffu, si, d);
        if (lane >= d) { ci += oc; pi += op; }
        if (lane + d < 32) si += os;
    }
    if (lane == 31) { ps.wc[warp] = ci; ps.wp[warp] = pi; }
    if (lane == 0) ps.ws[warp] = si;
    block_sync();
    int na = ci - cs, ntot = 0;
    float qa = pi - wsum, qb = si;
    for (int k = 0; k < kWarps; ++k) {
        ntot += ps.wc[k];
        if (k < warp) { na += ps.wc[k]; qa += ps.wp[k]; }
        if (k > warp) qb += ps.ws[k];
    }
    float best = -INFINITY;
    int bi = -1;
    for (int j = j0; j < j1; ++j) {
        const int2 e = sL[j];
        const float f0 = (float)e.y;
        const float w = shannon ? f0 * __log2f(f0) : exp2f(q * __log2f(f0));
        na += e.y;
        qa += w;
        qb -= w;
        const int nb = ntot - na;
        if (nb > 0) {
            const float fa = (float)na, fb = (float)nb, qbp = fmaxf(qb, 0.f);
            float f;
            if (shannon) {
                f = (__log2f(fa) - __fdividef(qa, fa)) + (__log2f(fb) - __fdividef(qbp, fb));
            } else {
                const float ab = __fdividef(qa, exp2f(q * __log2f(fa))) * __fdividef(qbp, exp2f(q * __log2f(fb)));
                f = __fdividef(1.0f - ab, q - 1.0f);
            }
            if (f > best) { best = f; bi = e.x; }
        }
    }
    warp_argmax(best, bi);
    if (lane == 0) { ps.bv[warp] = best; ps.bi[warp] = bi; }
    block_sync();
    float v = -INFINITY;
    int t = -1;
    for (int k = 0; k < kWarps; ++k) argmax_merge(v, t, ps.bv[k], ps.bi[k]);
    return M < 2 ? -1 : t;
}

}  // namespace
}  // namespace fp
}  // namespace tsl
