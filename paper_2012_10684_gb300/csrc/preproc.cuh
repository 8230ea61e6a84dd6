// Pre-processing (section II-B) and morphology (section II-C "Morphology")
// of CT slices, fused into one pass over the volume:
//
//   1. each voxel's CT number becomes an 8-bit level: 0 at or below the
//      detector background, otherwise [hu_min, hu_max] mapped linearly onto
//      0..255 and rounded to nearest, halves up;
//   2. flat grey erosion and/or dilation of each slice by the digital disk of
//      radius R (offsets dx^2 + dy^2 <= R^2; offsets outside the slice are
//      left out of the window), as one or two passes in shared memory;
//   3. the chest-mask subtraction (level - opening), the other subtraction
//      (closing - level), or a plain erosion/dilation/opening/closing/copy;
//   4. the 256-level histogram of the result, per slice or for the volume,
//      for the Tsallis threshold search that follows.
//
// One block per 128 x 64 output tile of one slice. The tile and a halo of R
// rows (and R pixels, rounded up to a word) per pass are staged in shared
// memory as fp16 pairs: levels 0..255 are exact in fp16, and __hmin2/__hmax2
// take the minimum of two pixels per instruction. A pass computes, for each
// column word (two pixels) and a run of K output rows, the chord extremes
// H_w (the extreme over the horizontal segment of half-width w) of every
// input row the run's disks touch, built incrementally w = 0..R in
// registers, and folds H_{w(dy)} into the K accumulators, where
// w(dy) = floor(sqrt(R^2 - dy^2)) is the disk's half-width on row dy. The
// radius is a template parameter so that every shift and index is resolved
// at compile time.
#pragma once
#include <cuda_fp16.h>

#include "checked.cuh"
#include "kernels.h"
#include "preproc_args.h"

namespace tsl {
namespace pre {

constexpr int kTW = 128;            // output tile width, pixels
constexpr int kTWw = kTW / 2;       // ... in words of two pixels
constexpr int kTH = 64;             // output tile height, rows
constexpr int kThreads = 320;
constexpr int kChunks = 4;          // runs of rows per column word in a pass
constexpr int kWarps = kThreads / 32;

enum { kOpCopy = 0, kOpErode = 1, kOpDilate = 2, kOpOpen = 3, kOpClose = 4, kOpChest = 5, kOpBlackTop = 6 };

__host__ __device__ constexpr int isqrt_floor(int n) {
    int r = 0;
    while ((r + 1) * (r + 1) <= n) ++r;
    return r;
}
__host__ __device__ constexpr int pad_words(int R) { return (R + 1) / 2; }
__host__ __device__ constexpr int run0(int R) { return (kTH + 2 * R + kChunks - 1) / kChunks; }

// Shared-memory geometry of a tile for radius R and np passes.
struct Geom {
    int np, stride, rows;
};
__host__ __device__ inline Geom geom(int R, int np) {
    Geom g;
    g.np = np;
    g.stride = kTWw + 2 * np * pad_words(R);
    g.rows = np == 2 ? kChunks * run0(R) + 2 * R : kTH + np * 2 * R;
    return g;
}

__device__ __forceinline__ __half2 as_h2(uint32_t u) { return *reinterpret_cast<__half2*>(&u); }
__device__ __forceinline__ uint32_t as_u32(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }

template <bool kMax>
__device__ __forceinline__ __half2 ext2(__half2 a, __half2 b) { return kMax ? __hmax2(a, b) : __hmin2(a, b); }
template <bool kMax>
__device__ __forceinline__ __half2 neutral2() {
    return kMax ? __floats2half2_rn(0.f, 0.f) : __floats2half2_rn(255.f, 255.f);
}

// The two pixels starting at pixel p of a window of words w[]: a word when p
// is even, the upper half of one word and the lower half of the next when p
// is odd. p is a compile-time constant in every use.
template <int NW>
__device__ __forceinline__ __half2 pair_at(const uint32_t (&w)[NW], int p) {
    return (p & 1) ? as_h2(__byte_perm(w[p >> 1], w[(p >> 1) + 1], 0x5432)) : as_h2(w[p >> 1]);
}

// Disk extreme (min, or max when kMax) for column word cw and output rows
// y0 .. y0+K-1 of src (words, row stride `stride`). Reads rows y0-R ..
// y0+K-1+R and words cw-P .. cw+P.
template <int R, int K, bool kMax>
__device__ __forceinline__ void disk_run(const uint32_t* src, int stride, int y0, int cw, __half2 (&acc)[K]) {
    constexpr int P = pad_words(R);
    constexpr int NW = 2 * P + 1;
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = neutral2<kMax>();
#pragma unroll
    for (int i = 0; i < K + 2 * R; ++i) {
        const uint32_t* row = src + (y0 - R + i) * stride + (cw - P);
        uint32_t w[NW];
#pragma unroll
        for (int j = 0; j < NW; ++j) w[j] = row[j];
        __half2 h[R + 1];
        h[0] = as_h2(w[P]);
#pragma unroll
        for (int d = 1; d <= R; ++d)
            h[d] = ext2<kMax>(h[d - 1], ext2<kMax>(pair_at(w, 2 * P - d), pair_at(w, 2 * P + d)));
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int dy = i - R - k;      // input row relative to output row y0 + k
            if (dy >= -R && dy <= R) acc[k] = ext2<kMax>(acc[k], h[isqrt_floor(R * R - dy * dy)]);
        }
    }
}

__device__ __forceinline__ int level_of(int v, const PreArgs& a) {
    if (v <= a.background) return 0;
    const int c = min(max(v, a.hu_min), a.hu_max) - a.hu_min;
    return (int)(__umulhi((unsigned)(2 * c * 255 + a.D), (unsigned)a.magic) >> a.shift);
}

struct Tile {
    int z, x0, y0;          // image pixel of shared word column 0 / row 0
    int* whist;             // [kWarps][256]
    int rows, stride;       // shared tile geometry (words), for the checked build
    long long total;        // voxels of the volume, for the checked build
};

// Stores pass-0 results into the intermediate image, with pixels outside
// the slice set to the next pass's neutral value.
template <bool kNextMax>
__device__ __forceinline__ void store_mid(uint32_t* mid, int stride, int y, int cw, __half2 v, const Tile& t,
                                          const PreArgs& a) {
    const int gy = t.y0 + y, gx = t.x0 + 2 * cw;
    const bool row_in = gy >= 0 && gy < a.ny;
    const __half n = kNextMax ? __float2half(0.f) : __float2half(255.f);
    __half lo = __low2half(v), hi = __high2half(v);
    if (!row_in || gx < 0 || gx >= a.nx) lo = n;
    if (!row_in || gx + 1 < 0 || gx + 1 >= a.nx) hi = n;
    if (in_range((long long)y * stride + cw, (long long)t.rows * t.stride, a.check, kSitePreMid))
        mid[y * stride + cw] = as_u32(__halves2half2(lo, hi));
}

// Writes the result for one word (two pixels) of the output tile: the op's
// value from the morphology result res and the level g, the int16 output
// (one 4-byte store when both pixels are in and aligned) and the histogram.
__device__ __forceinline__ void emit(const PreArgs& a, const Tile& t, int y, int cw, __half2 res, uint32_t g,
                                     int& zeros) {
    const int gy = t.y0 + y, gx = t.x0 + 2 * cw;
    if (gy < 0 || gy >= a.ny || gx >= a.nx) return;
    const float2 rf = __half22float2(res), gf = __half22float2(as_h2(g));
    float f0, f1;
    switch (a.op) {
        case kOpChest: f0 = gf.x - rf.x; f1 = gf.y - rf.y; break;
        case kOpBlackTop: f0 = rf.x - gf.x; f1 = rf.y - gf.y; break;
        case kOpCopy: f0 = gf.x; f1 = gf.y; break;
        default: f0 = rf.x; f1 = rf.y; break;
    }
    const int v0 = (int)f0, v1 = (int)f1;      // exact: integers 0..255
    const bool two = gx + 1 < a.nx;
    if (a.out && in_range(((long long)t.z * a.ny + gy) * a.nx + gx + (two ? 1 : 0), t.total, a.check, kSitePreOut)) {
        int16_t* o = a.out + ((long long)t.z * a.ny + gy) * a.nx + gx;
        if (two && ((uintptr_t)o & 3u) == 0) {
            *reinterpret_cast<uint32_t*>(o) = (uint32_t)(v0 & 0xffff) | ((uint32_t)v1 << 16);
        } else {
            o[0] = (int16_t)v0;
            if (two) o[1] = (int16_t)v1;
        }
    }
    if (a.hist) {
        // v is in 0..255 (an opening never exceeds the image, a closing
        // never falls below it); the clamp only guards the index
        int* wh = t.whist + (threadIdx.x >> 5) * 256;
        if (v0 == 0) ++zeros;
        else if (in_range(v0, 256, a.check, kSitePreHist)) atomicAdd(&wh[min(max(v0, 0), 255)], 1);
        if (two) {
            if (v1 == 0) ++zeros;
            else if (in_range(v1, 256, a.check, kSitePreHist)) atomicAdd(&wh[min(max(v1, 0), 255)], 1);
        }
    }
}

// Checked build: the rows and words a disk run reads lie inside the tile.
template <int R, int K>
__device__ __forceinline__ bool window_ok(int y0, int cw, const Tile& t, const PreArgs& a) {
    constexpr int P = pad_words(R);
    return in_range(y0 - R, t.rows, a.check, kSitePreWindow) && in_range(y0 + K - 1 + R, t.rows, a.check, kSitePreWindow) &&
           in_range(cw - P, t.stride, a.check, kSitePreWindow) && in_range(cw + P, t.stride, a.check, kSitePreWindow);
}

template <int R, int K, bool kMax>
__device__ __forceinline__ void final_pass(const uint32_t* src, const uint32_t* in, int stride, int row0, int cw0,
                                           const PreArgs& a, const Tile& t, int& zeros) {
    // output rows row0 .. row0 + kTH - 1, words cw0 .. cw0 + kTWw - 1
    for (int it = threadIdx.x; it < kTWw * kChunks; it += kThreads) {
        const int cw = cw0 + it % kTWw;
        const int y0 = row0 + (it / kTWw) * K;
        if (kCheckedBuild && !window_ok<R, K>(y0, cw, t, a)) continue;
        __half2 acc[K];
        disk_run<R, K, kMax>(src, stride, y0, cw, acc);
#pragma unroll
        for (int k = 0; k < K; ++k) emit(a, t, y0 + k, cw, acc[k], in[(y0 + k) * stride + cw], zeros);
    }
}

template <int R, bool kMax>
__device__ __forceinline__ void first_of_two(const uint32_t* in, uint32_t* mid, int stride, const PreArgs& a,
                                             const Tile& t) {
    constexpr int P = pad_words(R);
    constexpr int K = run0(R);
    constexpr int ncw = kTWw + 2 * P;
    for (int it = threadIdx.x; it < ncw * kChunks; it += kThreads) {
        const int cw = P + it % ncw;
        const int y0 = R + (it / ncw) * K;
        if (kCheckedBuild && !window_ok<R, K>(y0, cw, t, a)) continue;
        __half2 acc[K];
        disk_run<R, K, kMax>(in, stride, y0, cw, acc);
#pragma unroll
        for (int k = 0; k < K; ++k) store_mid<!kMax>(mid, stride, y0 + k, cw, acc[k], t, a);
    }
}

template <int R>
__global__ void __launch_bounds__(kThreads) k_preprocess(PreArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int np = (a.op == kOpCopy) ? 0 : (a.op == kOpErode || a.op == kOpDilate) ? 1 : 2;
    const Geom gm = geom(R, np);
    int* whist = reinterpret_cast<int*>(smem);
    uint32_t* in = reinterpret_cast<uint32_t*>(smem + kWarps * 256 * sizeof(int));
    uint32_t* mid = in + gm.rows * gm.stride;

    const long long tile = blockIdx.x;
    const int tx = (int)(tile % a.ntx);
    const int ty = (int)((tile / a.ntx) % a.nty);
    Tile t;
    t.z = (int)(tile / ((long long)a.ntx * a.nty));
    t.x0 = tx * kTW - np * 2 * pad_words(R);
    t.y0 = ty * kTH - np * R;
    t.whist = whist;
    t.rows = gm.rows;
    t.stride = gm.stride;
    t.total = (long long)a.nz * a.ny * a.nx;

    if (a.hist)
        for (int i = threadIdx.x; i < kWarps * 256; i += kThreads) whist[i] = 0;
    // first pass erodes for erosion, opening and the chest mask
    const bool first_max = a.op == kOpDilate || a.op == kOpClose || a.op == kOpBlackTop;
    const __half fill = first_max ? __float2half(0.f) : __float2half(255.f);
    // Staging: whole in-image pixel pairs at 4-byte-aligned addresses are
    // copied raw with cp.async (all of a thread's copies in flight at once)
    // and turned into levels in place once they have landed; edge pairs and
    // pixels outside the slice are written directly.
    const long long slice0 = (long long)t.z * a.ny * a.nx;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int y = warp; y < gm.rows; y += kWarps) {
        const int gy = t.y0 + y;
        const bool row_in = gy >= 0 && gy < a.ny;
        const long long rowe = slice0 + (long long)gy * a.nx;     // element index of (gy, 0)
        for (int cw = lane; cw < gm.stride; cw += 32) {
            const int gx = t.x0 + 2 * cw;
            const long long e = rowe + gx;                        // element index of the pair
            uint32_t* dst = &in[y * gm.stride + cw];
            if (kCheckedBuild && row_in && gx >= 0 && gx < a.nx &&
                !in_range(e + (gx + 1 < a.nx ? 1 : 0), t.total, a.check, kSitePreVol)) {
                *dst = 0u;
                continue;
            }
            if (row_in && gx >= 0 && gx + 1 < a.nx && ((e & 1) == 0)) {
                const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(a.vol + e) : "memory");
            } else {
                __half lo = fill, hi = fill;
                if (row_in && gx >= 0 && gx < a.nx) lo = __int2half_rn(level_of(a.vol[e], a));
                if (row_in && gx + 1 >= 0 && gx + 1 < a.nx) hi = __int2half_rn(level_of(a.vol[e + 1], a));
                *dst = as_u32(__halves2half2(lo, hi));
            }
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    for (int y = warp; y < gm.rows; y += kWarps) {
        const int gy = t.y0 + y;
        if (gy < 0 || gy >= a.ny) continue;
        const long long rowe = slice0 + (long long)gy * a.nx;
        for (int cw = lane; cw < gm.stride; cw += 32) {
            const int gx = t.x0 + 2 * cw;
            if (gx >= 0 && gx + 1 < a.nx && (((rowe + gx) & 1) == 0)) {
                uint32_t* dst = &in[y * gm.stride + cw];
                const uint32_t raw = *dst;
                *dst = as_u32(__halves2half2(__int2half_rn(level_of((int16_t)(raw & 0xffffu), a)),
                                             __int2half_rn(level_of((int16_t)(raw >> 16), a))));
            }
        }
    }
    __syncthreads();

    int zeros = 0;
    constexpr int P = pad_words(R);
    if (np == 0) {
        for (int it = threadIdx.x; it < kTWw * kTH; it += kThreads) {
            const int y = it / kTWw, cw = it - y * kTWw;
            emit(a, t, y, cw, as_h2(in[y * gm.stride + cw]), in[y * gm.stride + cw], zeros);
        }
    } else if (np == 1) {
        if (first_max) final_pass<R, kTH / kChunks, true>(in, in, gm.stride, R, P, a, t, zeros);
        else final_pass<R, kTH / kChunks, false>(in, in, gm.stride, R, P, a, t, zeros);
    } else {
        if (first_max) first_of_two<R, true>(in, mid, gm.stride, a, t);
        else first_of_two<R, false>(in, mid, gm.stride, a, t);
        __syncthreads();
        if (first_max) final_pass<R, kTH / kChunks, false>(mid, in, gm.stride, 2 * R, 2 * P, a, t, zeros);
        else final_pass<R, kTH / kChunks, true>(mid, in, gm.stride, 2 * R, 2 * P, a, t, zeros);
    }
    if (!a.hist) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zeros += __shfl_xor_sync(0xffffffffu, zeros, o);
    if ((threadIdx.x & 31) == 0 && zeros) atomicAdd(&whist[(threadIdx.x >> 5) * 256], zeros);
    __syncthreads();
    int* gh = a.hist + (a.per_slice ? (long long)t.z * 256 : 0);
    for (int b = threadIdx.x; b < 256; b += kThreads) {
        int s = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += whist[w * 256 + b];
        if (s) atomicAdd(&gh[b], s);
    }
}

template <int R>
size_t smem_bytes(int np) {
    const Geom g = geom(R, np);
    return kWarps * 256 * sizeof(int) + (size_t)(np == 2 ? 2 : 1) * g.rows * g.stride * sizeof(uint32_t);
}

template <int R>
cudaError_t prepare_r() {
    return cudaFuncSetAttribute(k_preprocess<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<R>(2));
}

template <int R>
cudaError_t launch_r(const PreArgs& a, cudaStream_t s) {
    const int np = (a.op == kOpCopy) ? 0 : (a.op == kOpErode || a.op == kOpDilate) ? 1 : 2;
    const long long nblocks = (long long)a.ntx * a.nty * a.nz;
    k_preprocess<R><<<(unsigned)nblocks, kThreads, smem_bytes<R>(np), s>>>(a);
    return cudaGetLastError();
}

// Explicit instantiations of the per-radius entry points live in
// preproc_r*.cu, a few radii per file so that they compile in parallel.
#define TSL_PREPROC_INSTANTIATE(R)                                          \
    template cudaError_t prepare_r<R>();                                    \
    template cudaError_t launch_r<R>(const PreArgs&, cudaStream_t);

}  // namespace pre
}  // namespace tsl
