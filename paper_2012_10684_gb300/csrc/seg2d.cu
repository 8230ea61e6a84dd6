// 2-D form of the thresholding path (section II-C, "Tsallis entropy").
//
// The grey level of a voxel is f = b >> shift, b = clamp(v - lo, 0, L-1),
// giving L2 = L >> shift <= 256 grey levels; its mean level is
// g = floor(sum of f over the 3x3 in-slice window / 9), or over the 3x3x3
// window / 27 in whole-volume mode, indices clamped at the borders. h(f, g)
// is the 2-D histogram. For a pair (t, s), quadrant 1 is {f <= t, g <= s}
// and quadrant 2 is {f > t, g > s}; the other two quadrants are ignored.
// With Q_k the sum of h^q over quadrant k and N_k its count,
//     phi(t, s) = (1 - a b) / (q - 1),  a = Q_1 / N_1^q,  b = Q_2 / N_2^q
// (the pseudo-additive objective; Shannon limit at q = 1 as in 1-D). The
// maximiser's t is the threshold of Algorithm 1, applied to f.
//
// Kernels:
//   k_hist2d    the histogram. Each thread owns four adjacent columns and
//               sweeps down a run of rows, keeping the 3-row window of
//               horizontal 3-sums (over 1 or 3 slices) in registers as
//               packed 16-bit lanes; neighbours across threads come by warp
//               shuffles. Counts with |g - f| <= kBand (nearly all: the mean
//               tracks the grey level away from edges) go to a band-shaped
//               shared-memory histogram, the rest straight to global memory.
//   k_s2_rows   per row f: the terms w = 2^64 (h / 2^31)^q as double-float
//               pairs (h log2 h at q = 1) and the row prefix and suffix sums
//               of terms and counts;
//   k_s2_cols   per column: prefix over rows of the row prefixes (sums over
//               [0..t] x [0..s]) and suffix over rows of the row suffixes
//               (sums over [t..] x [s..]); quadrant-2 sums are accumulated
//               from their own corner, never as a total minus quadrant 1;
//   k_s2_eval   phi(t, s) in double-float with its error bound for every
//               pair, and per row t the row's running top (its best pair,
//               and the largest value + bound among the others);
//   k_s2_final  the maximum over the rows' tops; when another pair's bound
//               reaches it, the pairs inside the bounds are re-evaluated in
//               FP64 from the double-float sums, the FP64 maximiser wins, and
//               among pairs with its partition (the same quadrant counts) and
//               the same value the smallest (t, s) is returned.
#include <cmath>

#include "checked.cuh"
#include "common.cuh"
#include "dfmath.cuh"
#include "kernels.h"
#include "top.cuh"
#include "../../include/tsallis.h"

namespace tsl {

namespace {

constexpr int kBand = 32;                  // half-width of the shared-memory band
constexpr int kBandW = 2 * kBand + 1;
// Row stride of the band in shared memory: cell (f, d) at f * kBandStride + d
// lies in bank (4 f + g) mod 32 (g = f + d - kBand; 68 = 4 mod 32), so the
// cells of a small neighbourhood of (f, g) fall in distinct banks. With the
// stride kBandW (64 = 0 mod 32) the bank was g mod 32 alone: every voxel of
// one mean level g collided in one bank whatever its grey level.
constexpr int kBandStride = 69;
static_assert(kBandStride >= kBandW && (kBandStride - 1) % 32 == 4, "band stride");
constexpr int kH2Threads = 512;
constexpr int kH2RowsPerGroup = 16;        // rows one thread group sweeps per tile
constexpr int kS2Threads = 256;            // >= L2
constexpr float kFixedLog2N = 31.0f;       // terms scaled as (h / 2^31)^q: no total needed

// ------------------------------------------------------------ histogram

struct Hist2dArgs {
    const int16_t* vol;
    int nx, ny, nz;
    int lo, hi;            // hi = min(lo + L - 1, 32767)
    int shift, L2;
    int per_slice;         // 1: histogram z of slice z; 0: one histogram
    int qw;                // column quads per thread group (multiple of 32, <= 128)
    int nxb, nyc;          // x blocks and y chunks per slice
    long long ntiles;
    int* ghist;            // [nh][L2][L2], zeroed by the caller
};

// Grey levels of two packed int16 voxels, in 16-bit lanes.
__device__ __forceinline__ unsigned grey2(unsigned w, unsigned LO2, unsigned HI2, int shift, unsigned M2) {
    return (__vsub2(__vmins2(__vmaxs2(w, LO2), HI2), LO2) >> shift) & M2;
}
__device__ __forceinline__ unsigned grey1(int v, int lo, int hi, int shift) {
    v = v < lo ? lo : (v > hi ? hi : v);
    return (unsigned)(v - lo) >> shift;
}

// Grey levels of columns x0 .. x0+3 of one row as two packed words
// [f0 | f1 << 16], [f2 | f3 << 16]. Columns past the end repeat column nx-1
// (the clamped index), which is also what the right border of the window
// needs.
template <bool kVec>
__device__ __forceinline__ void grey_quad(const int16_t* __restrict__ row, int x0, int nx, unsigned LO2, unsigned HI2,
                                          int shift, unsigned M2, unsigned& A, unsigned& B) {
    unsigned w0, w1;
    if (kVec) {   // nx % 4 == 0 and 8-byte aligned rows
        const int xs = x0 < nx ? x0 : nx - 4;
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(row + xs));
        w0 = v.x;
        w1 = v.y;
    } else {
        const unsigned short* r = reinterpret_cast<const unsigned short*>(row);
        const int xa = min(x0, nx - 1), xb = min(x0 + 1, nx - 1), xc = min(x0 + 2, nx - 1), xd = min(x0 + 3, nx - 1);
        w0 = (unsigned)__ldg(r + xa) | ((unsigned)__ldg(r + xb) << 16);
        w1 = (unsigned)__ldg(r + xc) | ((unsigned)__ldg(r + xd) << 16);
    }
    A = grey2(w0, LO2, HI2, shift, M2);
    B = grey2(w1, LO2, HI2, shift, M2);
}

// Horizontal window sums of one row (summed over kDz-neighbourhood slices)
// for the thread's four columns, packed: Ha = [H0 | H1], Hb = [H2 | H3];
// and the centre slice's grey levels Fa, Fb.
template <int kDz, bool kVec>
__device__ __forceinline__ void row_sums(const Hist2dArgs& a, int z, int y, int x0, int lane, unsigned LO2,
                                         unsigned HI2, unsigned M2, unsigned& Ha, unsigned& Hb, unsigned& Fa,
                                         unsigned& Fb) {
    const long long plane = (long long)a.nx * a.ny;
    const int16_t* base = a.vol + (long long)y * a.nx;
    unsigned A, B;
    grey_quad<kVec>(base + z * plane, x0, a.nx, LO2, HI2, a.shift, M2, Fa, Fb);
    A = Fa;
    B = Fb;
    if (kDz) {
        const int zm = z > 0 ? z - 1 : 0, zp = z < a.nz - 1 ? z + 1 : a.nz - 1;
        unsigned A1, B1, A2, B2;
        grey_quad<kVec>(base + zm * plane, x0, a.nx, LO2, HI2, a.shift, M2, A1, B1);
        grey_quad<kVec>(base + zp * plane, x0, a.nx, LO2, HI2, a.shift, M2, A2, B2);
        A += A1 + A2;   // lanes stay below 3 * 255
        B += B1 + B2;
    }
    // neighbours: column x0 - 1 and x0 + 4 (clamped at the volume border)
    const bool left_in = x0 > 0, right_in = x0 + 4 < a.nx;
    unsigned gl = __shfl_up_sync(0xffffffffu, B, 1) >> 16;
    unsigned gr = __shfl_down_sync(0xffffffffu, A, 1) & 0xffffu;
    const bool need = (lane == 0 && left_in) || (lane == 31 && right_in);
    if (need) {
        const int xe = lane == 0 ? min(x0 - 1, a.nx - 1) : x0 + 4;   // idle lanes stay in bounds
        unsigned e = grey1(__ldg(base + z * plane + xe), a.lo, a.hi, a.shift);
        if (kDz) {
            const int zm = z > 0 ? z - 1 : 0, zp = z < a.nz - 1 ? z + 1 : a.nz - 1;
            e += grey1(__ldg(base + zm * plane + xe), a.lo, a.hi, a.shift) +
                 grey1(__ldg(base + zp * plane + xe), a.lo, a.hi, a.shift);
        }
        if (lane == 0) gl = e;
        else gr = e;
    }
    if (!left_in) gl = A & 0xffffu;    // column -1 is column 0
    if (!right_in) gr = B >> 16;       // column past the end repeats the last one
    const unsigned mid = (A >> 16) | (B << 16);   // [g1 | g2]
    Ha = ((A << 16) | gl) + A + mid;
    Hb = mid + B + ((B >> 16) | (gr << 16));
}

// Band-shaped shared histogram: entry (f, g) with d = g - f + kBand in
// [0, kBandW) lives at band[f * kBandStride + d].
__device__ __forceinline__ void count_voxel(int f, int g, int* band, int* gh, int L2) {
    const int d = g - f + kBand;
    if ((unsigned)d < (unsigned)kBandW) atomicAdd(band + f * kBandStride + d, 1);
    else atomicAdd(gh + f * L2 + g, 1);
}

__device__ void flush_band(int* band, int* gh, int L2) {
    const int nb = L2 * kBandStride;
    for (int i = threadIdx.x; i < nb; i += kH2Threads) {
        const int c = band[i];
        if (c) {
            const int f = i / kBandStride, d = i - f * kBandStride, g = f + d - kBand;   // d < kBandW: the pad stays 0
            atomicAdd(gh + f * L2 + g, c);
            band[i] = 0;
        }
    }
}

// ---- staged rows (the aligned path with the in-slice 3x3 window): each
// thread copies its own input words of a row two rows ahead into shared
// memory with cp.async, so the loads' latency overlaps the counting of the
// current row. A slot holds the thread's 8-byte word (columns x0 .. x0+3)
// and, for lanes 0 and 31, the 4-byte word holding the neighbouring column
// (x0-2 .. x0-1, x0+4 .. x0+5). Only the thread that copied a word reads it
// back, after its own cp.async.wait_group, so no barrier is needed; a slot is
// refilled one iteration after its last read. (Staging the three slices of
// the 3x3x3 window this way was measured slower than loading them directly:
// 179 against 164 us on 512x512x256; the in-slice form gains 6 %.)
constexpr int kH2Warps = kH2Threads / 32;
constexpr int kStageSlots = 3;
constexpr int kStageSlices = 1;
constexpr int kStageMainWords = kStageSlices * kH2Threads;          // uint2 per slot
constexpr int kStageEdgeWords = kStageSlices * kH2Warps * 2;        // unsigned per slot
constexpr int kStageBytes = kStageSlots * (kStageMainWords * 8 + kStageEdgeWords * 4);

__device__ __forceinline__ void h2_cp_async8(void* s, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g)
                 : "memory");
}
__device__ __forceinline__ void h2_cp_async4(void* s, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g)
                 : "memory");
}
__device__ __forceinline__ void h2_cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int kN>
__device__ __forceinline__ void h2_cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(kN) : "memory"); }

// Issues the copies of row y of slice z (clamped by the caller) into this
// thread's part of a slot: sw = the slot's main words + threadIdx.x, se = the
// slot's edge words + 2 * warp + (lane == 31).
__device__ __forceinline__ void stage_row(const Hist2dArgs& a, int z, int y, int x0, int lane, bool left_in,
                                          bool right_in, uint2* sw, unsigned* se) {
    const int16_t* r = a.vol + (long long)z * a.nx * a.ny + (long long)y * a.nx;
    const int xs = x0 < a.nx ? x0 : a.nx - 4;   // a quad past the row repeats the last one (never counted)
    const int xl = (x0 < a.nx ? x0 : a.nx) - 2;   // left neighbour word; past the row: columns nx-2, nx-1
    h2_cp_async8(sw, r + xs);
    if (lane == 0 && left_in) h2_cp_async4(se, r + xl);
    if (lane == 31 && right_in) h2_cp_async4(se, r + x0 + 4);
}

// row_sums<0, true> from a staged row (same results).
__device__ __forceinline__ void staged_row_sums(const Hist2dArgs& a, int lane, bool left_in, bool right_in,
                                                unsigned LO2, unsigned HI2, unsigned M2, const uint2* sw,
                                                const unsigned* se, unsigned& Ha, unsigned& Hb, unsigned& Fa,
                                                unsigned& Fb) {
    const uint2 w0 = sw[0];
    Fa = grey2(w0.x, LO2, HI2, a.shift, M2);
    Fb = grey2(w0.y, LO2, HI2, a.shift, M2);
    const unsigned A = Fa, B = Fb;
    unsigned gl = __shfl_up_sync(0xffffffffu, B, 1) >> 16;
    unsigned gr = __shfl_down_sync(0xffffffffu, A, 1) & 0xffffu;
    if ((lane == 0 && left_in) || (lane == 31 && right_in)) {
        const unsigned ww = se[0];
        const unsigned e = grey1(lane == 0 ? ((int)ww >> 16) : (int)(short)(ww & 0xffffu), a.lo, a.hi, a.shift);
        if (lane == 0) gl = e;
        else gr = e;
    }
    if (!left_in) gl = A & 0xffffu;    // column -1 is column 0
    if (!right_in) gr = B >> 16;       // column past the end repeats the last one
    const unsigned mid = (A >> 16) | (B << 16);
    Ha = ((A << 16) | gl) + A + mid;
    Hb = mid + B + ((B >> 16) | (gr << 16));
}

// Counts the voxels of one output row from the window sums of its rows
// y - 1, y, y + 1 and its centre grey levels.
template <unsigned kDiv>
__device__ __forceinline__ void count_row(unsigned Ta, unsigned Tb, unsigned F0a, unsigned F0b, int x0, int nx,
                                          int* band, int* gh, int L2) {
    if (x0 + 3 < nx) {   // the thread's four columns are all inside the row
        count_voxel((int)(F0a & 0xffffu), (int)((Ta & 0xffffu) / kDiv), band, gh, L2);
        count_voxel((int)(F0a >> 16), (int)((Ta >> 16) / kDiv), band, gh, L2);
        count_voxel((int)(F0b & 0xffffu), (int)((Tb & 0xffffu) / kDiv), band, gh, L2);
        count_voxel((int)(F0b >> 16), (int)((Tb >> 16) / kDiv), band, gh, L2);
    } else if (x0 < nx) {
        count_voxel((int)(F0a & 0xffffu), (int)((Ta & 0xffffu) / kDiv), band, gh, L2);
        if (x0 + 1 < nx) count_voxel((int)(F0a >> 16), (int)((Ta >> 16) / kDiv), band, gh, L2);
        if (x0 + 2 < nx) count_voxel((int)(F0b & 0xffffu), (int)((Tb & 0xffffu) / kDiv), band, gh, L2);
    }
}

template <int kDz, bool kVec>
__global__ void __launch_bounds__(kH2Threads, 2) k_hist2d(const Hist2dArgs a) {
    extern __shared__ int band[];
    // the row staging ring follows the band (16-byte aligned)
    uint2* stage_main = reinterpret_cast<uint2*>(band + ((a.L2 * kBandStride + 3) & ~3));
    unsigned* stage_edge = reinterpret_cast<unsigned*>(stage_main + kStageSlots * kStageMainWords);
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < a.L2 * kBandStride; i += kH2Threads) band[i] = 0;
    __syncthreads();
    constexpr unsigned kDiv = kDz ? 27u : 9u;
    const unsigned LO2 = ((unsigned)a.lo & 0xffffu) * 0x10001u;
    const unsigned HI2 = ((unsigned)a.hi & 0xffffu) * 0x10001u;
    const unsigned M2 = (0xffffu >> a.shift) * 0x10001u;
    const int group = tid / a.qw, cq = tid - group * a.qw;
    const int rows_per_tile = (kH2Threads / a.qw) * kH2RowsPerGroup;
    const long long t0 = (long long)blockIdx.x * a.ntiles / gridDim.x;
    const long long t1 = (long long)(blockIdx.x + 1) * a.ntiles / gridDim.x;
    int cur = -1;
    for (long long t = t0; t < t1; ++t) {
        const int xb = (int)(t % a.nxb);
        const long long r = t / a.nxb;
        const int yc = (int)(r % a.nyc);
        const int z = (int)(r / a.nyc);
        const int hidx = a.per_slice ? z : 0;
        if (hidx != cur) {
            if (cur >= 0) {
                __syncthreads();
                flush_band(band, a.ghist + (long long)cur * a.L2 * a.L2, a.L2);
                __syncthreads();
            }
            cur = hidx;
        }
        int* gh = a.ghist + (long long)hidx * a.L2 * a.L2;
        const int x0 = 4 * (xb * a.qw + cq);
        const int ys = yc * rows_per_tile + group * kH2RowsPerGroup;
        const int ye = min(ys + kH2RowsPerGroup, a.ny);
        if (ys >= a.ny) continue;   // uniform per warp: a warp lies in one group
        if constexpr (kVec && kDz == 0) {
            // input rows j = 0 .. nrows - 1 are rows ys - 1 + j (clamped);
            // output row ys + j - 2 is counted once input row j is summed
            const bool left_in = x0 > 0, right_in = x0 + 4 < a.nx;
            const int nrows = ye - ys + 2;
            uint2* sw0 = stage_main + threadIdx.x;
            unsigned* se0 = stage_edge + 2 * (threadIdx.x >> 5) + (lane == 31 ? 1 : 0);
            auto row_of = [&](int j) {
                const int y = ys - 1 + j;
                return y < 0 ? 0 : (y > a.ny - 1 ? a.ny - 1 : y);
            };
            stage_row(a, z, row_of(0), x0, lane, left_in, right_in, sw0, se0);
            h2_cp_async_commit();
            stage_row(a, z, row_of(1), x0, lane, left_in, right_in, sw0 + kStageMainWords,
                           se0 + kStageEdgeWords);
            h2_cp_async_commit();
            unsigned Hma = 0, Hmb = 0, H0a = 0, H0b = 0, F0a = 0, F0b = 0;
            for (int j = 0; j < nrows; ++j) {
                h2_cp_async_wait<1>();   // row j has landed (row j + 1 may still be in flight)
                const int sl = j % kStageSlots;
                unsigned Hna, Hnb, Fna, Fnb;
                staged_row_sums(a, lane, left_in, right_in, LO2, HI2, M2, sw0 + sl * kStageMainWords,
                                     se0 + sl * kStageEdgeWords, Hna, Hnb, Fna, Fnb);
                if (j + 2 < nrows) {
                    const int s2 = (j + 2) % kStageSlots;   // last read at iteration j - 1
                    stage_row(a, z, row_of(j + 2), x0, lane, left_in, right_in, sw0 + s2 * kStageMainWords,
                                   se0 + s2 * kStageEdgeWords);
                }
                h2_cp_async_commit();   // possibly empty: keeps one group per row
                if (j >= 2)
                    count_row<kDiv>(Hma + H0a + Hna, Hmb + H0b + Hnb, F0a, F0b, x0, a.nx, band, gh, a.L2);
                Hma = H0a; Hmb = H0b; H0a = Hna; H0b = Hnb; F0a = Fna; F0b = Fnb;
            }
            h2_cp_async_wait<0>();
        } else {
            unsigned Rma, Rmb, R0a, R0b, F0a, F0b, Fxa, Fxb;
            row_sums<kDz, kVec>(a, z, ys > 0 ? ys - 1 : 0, x0, lane, LO2, HI2, M2, Rma, Rmb, Fxa, Fxb);
            row_sums<kDz, kVec>(a, z, ys, x0, lane, LO2, HI2, M2, R0a, R0b, F0a, F0b);
            for (int y = ys; y < ye; ++y) {
                unsigned Rna, Rnb, Fna, Fnb;
                row_sums<kDz, kVec>(a, z, y + 1 < a.ny ? y + 1 : a.ny - 1, x0, lane, LO2, HI2, M2, Rna, Rnb, Fna,
                                    Fnb);
                // lanes below 9 * 765
                count_row<kDiv>(Rma + R0a + Rna, Rmb + R0b + Rnb, F0a, F0b, x0, a.nx, band, gh, a.L2);
                Rma = R0a; Rmb = R0b; R0a = Rna; R0b = Rnb; F0a = Fna; F0b = Fnb;
            }
        }
    }
    __syncthreads();
    if (cur >= 0) flush_band(band, a.ghist + (long long)cur * a.L2 * a.L2, a.L2);
}

// ------------------------------------------------------------ search

struct S2Args {
    const int* hist;      // [K][L2][L2]
    int L2;
    float q;
    const DfTables* T;
    int* PC;              // [K][L2][L2] counts, then quadrant-1 counts
    float2* PW;           // terms, then quadrant-1 term sums
    int* SC;              // [K][L2][L2] counts, then quadrant-2 counts
    float2* SW;
    // per row t, the row's running top (top.cuh): its best value (double-
    // float), the pair index t * (L2 - 1) + s (-1: no valid pair), its error
    // bound, and the largest value + bound among the row's other pairs
    float* rvh;           // [K][L2]
    float* rvl;
    float* rband;
    float* ru2;
    int* ri;
    float* curve;         // optional [K][L2-1][L2-1]
    int* t_out;           // [K][2] (t, s)
    int* t_bin;           // optional [K]: t alone, for the binarise pass
    float* phi_out;
    int* status;
    // window search (null / 0 otherwise)
    const int* cand;      // [K][topk] candidate cells
    int topk;
    unsigned char* cellflag;   // [K][kCells2d]
    int* winfo;           // [K] cells searched beyond the candidates
    long long K;          // histograms
    unsigned* check;      // checked build: first failing index check
};

__device__ __forceinline__ long long s2_off(const S2Args& a, int k) { return (long long)k * a.L2 * a.L2; }

// Inclusive block scans over the 256 threads (one value per thread).
struct ScanSmem {
    int c[kS2Threads / 32];
    F2 w[kS2Threads / 32];
};
__device__ __forceinline__ int warp_prefix_i32(int v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    return v;
}
__device__ __forceinline__ int warp_suffix_i32(int v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_down_sync(0xffffffffu, v, d);
        if (lane + d < 32) v += o;
    }
    return v;
}

__device__ void block_scan(int c, F2 w, bool suffix, ScanSmem& sm, int& c_out, F2& w_out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kW = kS2Threads / 32;
    int ci = suffix ? warp_suffix_i32(c, lane) : warp_prefix_i32(c, lane);
    F2 wi = suffix ? warp_suffix_f2(w, lane) : warp_prefix_f2(w, lane);
    const int edge = suffix ? 0 : 31;
    if (lane == edge) { sm.c[warp] = ci; sm.w[warp] = wi; }
    __syncthreads();
    // carry from the other warps, summed in a fixed order
    int cc = 0;
    F2 wc{0.f, 0.f};
    if (suffix) {
        for (int j = kW - 1; j > warp; --j) { cc += sm.c[j]; wc = f2_add(sm.w[j], wc); }
    } else {
        for (int j = 0; j < warp; ++j) { cc += sm.c[j]; wc = f2_add(wc, sm.w[j]); }
    }
    __syncthreads();
    c_out = ci + cc;
    w_out = suffix ? f2_add(wi, wc) : f2_add(wc, wi);
}

__global__ void __launch_bounds__(kS2Threads) k_s2_rows(const S2Args a) {
    __shared__ DfTables sdf;
    df_stage(&sdf, a.T, threadIdx.x, blockDim.x);
    __syncthreads();
    const DfTables* T = &sdf;
    __shared__ ScanSmem sm;
    const int k = blockIdx.y, i = blockIdx.x, s = threadIdx.x;
    const long long o = s2_off(a, k) + (long long)i * a.L2;
    const int h = s < a.L2 ? __ldg(a.hist + o + s) : 0;
    F2 w{0.f, 0.f};
    if (h > 0) w = a.q == 1.0f ? df_hlog2h<true>((unsigned)h, T) : df_pow_ratio<true>((unsigned)h, F2{kFixedLog2N, 0.f}, a.q, T);
    int c;
    F2 ws;
    block_scan(h, w, false, sm, c, ws);
    if (s < a.L2) { a.PC[o + s] = c; a.PW[o + s] = make_float2(ws.hi, ws.lo); }
    block_scan(h, w, true, sm, c, ws);
    if (s < a.L2) { a.SC[o + s] = c; a.SW[o + s] = make_float2(ws.hi, ws.lo); }
}

// Column scans: 32 columns x 32 row chunks per block (at most 8 rows per
// chunk for L2 <= 256). Each thread loads its chunk's cells together into
// registers, the chunk totals are exchanged through shared memory (summed
// in a fixed order), and the thread scans its chunk in registers: prefix
// over rows of the row prefixes, suffix over rows of the row suffixes.
constexpr int kColRows = 8;
__global__ void __launch_bounds__(1024) k_s2_cols(const S2Args a) {
    __shared__ int tcA[32][33], tcB[32][33];
    __shared__ F2 twA[32][33], twB[32][33];
    const int c = threadIdx.x & 31, r = threadIdx.x >> 5;
    const int k = blockIdx.y, s = blockIdx.x * 32 + c;
    const int rc = (a.L2 + 31) / 32, i0 = min(r * rc, a.L2), i1 = min(i0 + rc, a.L2);
    const long long o = s2_off(a, k);
    int pc[kColRows], sc[kColRows];
    F2 pw[kColRows], sw[kColRows];
#pragma unroll
    for (int j = 0; j < kColRows; ++j) {
        const int i = i0 + j;
        pc[j] = 0; sc[j] = 0;
        pw[j] = F2{0.f, 0.f}; sw[j] = F2{0.f, 0.f};
        if (s < a.L2 && i < i1) {
            const long long e = o + (long long)i * a.L2 + s;
            pc[j] = a.PC[e];
            sc[j] = a.SC[e];
            const float2 x = a.PW[e], y = a.SW[e];
            pw[j] = F2{x.x, x.y};
            sw[j] = F2{y.x, y.y};
        }
    }
    int ca = 0, cb = 0;
    F2 wa{0.f, 0.f}, wb{0.f, 0.f};
#pragma unroll
    for (int j = 0; j < kColRows; ++j) { ca += pc[j]; wa = f2_add(wa, pw[j]); }
#pragma unroll
    for (int j = kColRows - 1; j >= 0; --j) { cb += sc[j]; wb = f2_add(sw[j], wb); }
    tcA[r][c] = ca; twA[r][c] = wa;
    tcB[r][c] = cb; twB[r][c] = wb;
    __syncthreads();
    ca = 0; cb = 0;
    wa = F2{0.f, 0.f}; wb = F2{0.f, 0.f};
    for (int j = 0; j < r; ++j) { ca += tcA[j][c]; wa = f2_add(wa, twA[j][c]); }
    for (int j = 31; j > r; --j) { cb += tcB[j][c]; wb = f2_add(twB[j][c], wb); }
    if (s >= a.L2) return;
#pragma unroll
    for (int j = 0; j < kColRows; ++j) {
        ca += pc[j];
        wa = f2_add(wa, pw[j]);
        pc[j] = ca;
        pw[j] = wa;
    }
#pragma unroll
    for (int j = kColRows - 1; j >= 0; --j) {
        cb += sc[j];
        wb = f2_add(sw[j], wb);
        sc[j] = cb;
        sw[j] = wb;
    }
#pragma unroll
    for (int j = 0; j < kColRows; ++j) {
        const int i = i0 + j;
        if (i >= i1) break;
        const long long e = o + (long long)i * a.L2 + s;
        a.PC[e] = pc[j];
        a.PW[e] = make_float2(pw[j].hi, pw[j].lo);
        a.SC[e] = sc[j];
        a.SW[e] = make_float2(sw[j].hi, sw[j].lo);
    }
}

// Quadrant sums of pair (t, s): quadrant 1 at [t][s] of the prefix tables,
// quadrant 2 at [t+1][s+1] of the suffix tables.
struct Quad {
    int na, nb;
    F2 qa, qb;
};
__device__ __forceinline__ Quad quad_sums(const S2Args& a, int k, int t, int s) {
    const long long o = s2_off(a, k);
    const long long ea = o + (long long)t * a.L2 + s, eb = o + (long long)(t + 1) * a.L2 + (s + 1);
    const long long cells = a.K * a.L2 * a.L2;
    if (kCheckedBuild && !(in_range(ea, cells, a.check, kSite2dTables) && in_range(eb, cells, a.check, kSite2dTables)))
        return Quad{0, 0, F2{0.f, 0.f}, F2{0.f, 0.f}};
    const float2 x = a.PW[ea], y = a.SW[eb];
    return Quad{a.PC[ea], a.SC[eb], F2{x.x, x.y}, F2{y.x, y.y}};
}

__device__ __forceinline__ double eval64(const Quad& u, float q, const DfTables* T) {
    if (q == 1.0f) {
        const double la = df_to_double(df_log2_count<true>((unsigned)u.na, T));
        const double lb = df_to_double(df_log2_count<true>((unsigned)u.nb, T));
        return 0.6931471805599453 *
               ((la - df_to_double(u.qa) / (double)u.na) + (lb - df_to_double(u.qb) / (double)u.nb));
    }
    const F2 LN{kFixedLog2N, 0.f};
    const double pa = df_to_double(df_pow_ratio<true>((unsigned)u.na, LN, q, T));
    const double pb = df_to_double(df_pow_ratio<true>((unsigned)u.nb, LN, q, T));
    const double ab = (df_to_double(u.qa) / pa) * (df_to_double(u.qb) / pb);
    return (1.0 - ab) / ((double)q - 1.0);
}

__device__ __forceinline__ bool same_sums(const Quad& x, const Quad& y) {
    return x.na == y.na && x.nb == y.nb && x.qa.hi == y.qa.hi && x.qa.lo == y.qa.lo && x.qb.hi == y.qb.hi &&
           x.qb.lo == y.qb.lo;
}

struct RedSmem {
    float v[kS2Threads / 32];
    float u[kS2Threads / 32];
    int i[kS2Threads / 32];
    double dv[kS2Threads / 32];
    int n[kS2Threads / 32];
};

// Double-float objective of a pair and its error bound (top.cuh); false
// when a quadrant is empty.
__device__ __forceinline__ bool eval_df(const Quad& u, float q, const DfTables* T, F2& phi, float& band) {
    if (u.na <= 0 || u.nb <= 0) return false;
    const F2 LN{kFixedLog2N, 0.f};
    if (q == 1.0f) {
        const F2 la = df_log2_count<true>((unsigned)u.na, T), lb = df_log2_count<true>((unsigned)u.nb, T);
        const F2 sa = df_div(u.qa, df_from_u32((unsigned)u.na)), sb = df_div(u.qb, df_from_u32((unsigned)u.nb));
        phi = df_mul(df_add(df_add(la, f2_neg(sa)), df_add(lb, f2_neg(sb))), df_ln2());
        band = shannon_band_df(la.hi, sa.hi, lb.hi, sb.hi);
    } else {
        const F2 pa = df_pow_ratio<true>((unsigned)u.na, LN, q, T), pb = df_pow_ratio<true>((unsigned)u.nb, LN, q, T);
        const F2 ab = df_mul(df_div(u.qa, pa), df_div(u.qb, pb));
        phi = df_div(df_add(F2{1.0f, 0.f}, f2_neg(ab)), two_sum(q, -1.0f));
        band = tsallis_band_df(ab.hi, phi.hi, q);
    }
    return true;
}

// Per-warp tops, reduced by warp 0 into sm.t[0].
struct TopSmem {
    float vh[kS2Threads / 32], vl[kS2Threads / 32], band[kS2Threads / 32], u2[kS2Threads / 32];
    int i[kS2Threads / 32];
};
__device__ Top block_top2(Top tp, TopSmem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) tp = top_merge(tp, shfl_top(tp, d));
    if (lane == 0) {
        sm.vh[warp] = tp.v.hi; sm.vl[warp] = tp.v.lo; sm.band[warp] = tp.band; sm.u2[warp] = tp.u2; sm.i[warp] = tp.i;
    }
    __syncthreads();
    Top g{{-INFINITY, 0.f}, -1, 0.f, -INFINITY};
#pragma unroll
    for (int w = 0; w < kS2Threads / 32; ++w) g = top_merge(g, Top{{sm.vh[w], sm.vl[w]}, sm.i[w], sm.band[w], sm.u2[w]});
    __syncthreads();
    return g;
}

// One block per row t: the objective at every (t, s) in double-float, and
// the row's top.
__global__ void __launch_bounds__(kS2Threads) k_s2_eval(const S2Args a) {
    __shared__ DfTables sdf;
    df_stage(&sdf, a.T, threadIdx.x, blockDim.x);
    __syncthreads();
    const DfTables* T = &sdf;
    __shared__ TopSmem sm;
    const int k = blockIdx.y, t = blockIdx.x, s = threadIdx.x;
    const int m = a.L2 - 1;
    Top tp{{-INFINITY, 0.f}, -1, 0.f, -INFINITY};
    F2 phi{0.f, 0.f};
    float band = 0.f;
    bool ok = false;
    const bool wanted = !a.cellflag || a.cellflag[(long long)k * kCells2d + (t / kCell2d) * 64 + s / kCell2d];
    if (s < m && wanted) {
        ok = eval_df(quad_sums(a, k, t, s), a.q, T, phi, band);
        if (ok) tp = Top{phi, t * m + s, band, -INFINITY};
    }
    if (a.curve && s < m && wanted)
        a.curve[((long long)k * m + t) * m + s] = ok ? phi.hi + phi.lo : __int_as_float(0x7fc00000);
    const Top g = block_top2(tp, sm);
    if (s == 0) {
        const long long r = (long long)k * a.L2 + t;
        a.rvh[r] = g.v.hi;
        a.rvl[r] = g.v.lo;
        a.rband[r] = g.band;
        a.ru2[r] = g.u2;
        a.ri[r] = g.i;
    }
}

// Block reductions for the final kernel.
__device__ void red_argmax_d(double& v, int& i, RedSmem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_argmax(v, i);
    if (lane == 0) { sm.dv[warp] = v; sm.i[warp] = i; }
    __syncthreads();
    v = lane < kS2Threads / 32 ? sm.dv[lane] : 0.0;
    i = lane < kS2Threads / 32 ? sm.i[lane] : -1;
    warp_argmax(v, i);
    __syncthreads();
}
__device__ int red_min_i(int v, RedSmem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = __reduce_min_sync(0xffffffffu, v);
    if (lane == 0) sm.n[warp] = v;
    __syncthreads();
    v = lane < kS2Threads / 32 ? sm.n[lane] : 0x7fffffff;
    v = __reduce_min_sync(0xffffffffu, v);
    __syncthreads();
    return v;
}
// Two FP64 values of one partition computed from differently associated
// double-float sums agree to far better than this; distinct partitions
// closer than this are near-ties.
constexpr double kSamePartitionTol = 1e-10;

// One block per histogram: the maximum over the rows' tops; when another
// pair's bound reaches it, the pairs inside the bounds are re-ranked in FP64,
// and among pairs with the winner's quadrant counts and value the smallest
// (t, s) is returned.
// Status bits of a window search: the winner's cell among the candidates,
// and how many other cells had to be searched (saturating at 255).
__device__ __forceinline__ int window_bits(const S2Args& a, int k, int t, int s) {
    if (!a.cellflag) return 0;
    const int hit = a.cellflag[(long long)k * kCells2d + (t / kCell2d) * 64 + s / kCell2d] == 2;
    return (hit ? TSALLIS_STATUS_WINDOW_HIT : 0) | (min(a.winfo[k], 255) << TSALLIS_STATUS_FALLBACK_SHIFT);
}

// Upper bound of phi over the valid pairs of the cell [t0, t1] x [s0, s1]
// from the tables at its corners: N_1, Q_1 grow and N_2, Q_2 shrink with t
// and with s, so for q < 1 a b <= Q_1(t1,s1) Q_2(t0,s0) / (N_1(t0,s0)
// N_2(t1,s1))^q, for q > 1 a b >= Q_1(t0,s0) Q_2(t1,s1) / (N_1(t1,s1)
// N_2(t0,s0))^q, and at q = 1 each H_k <= log N_k(max) - Q_k(min) / N_k(max).
// Evaluated in double-float like the objective (FP32 instructions; FP64 is
// slow on this part); -inf when the cell holds no valid pair, +inf when a
// bound is unbounded.
__device__ float cell_bound(const S2Args& a, const DfTables* __restrict__ T, int k, int t0, int t1, int s0, int s1) {
    const long long o = s2_off(a, k);
    const long long a0 = o + (long long)t0 * a.L2 + s0, a1 = o + (long long)t1 * a.L2 + s1;
    const long long b_big = o + (long long)(t0 + 1) * a.L2 + (s0 + 1), b_small = o + (long long)(t1 + 1) * a.L2 + (s1 + 1);
    const int na0 = a.PC[a0], na1 = a.PC[a1], nb1 = a.SC[b_big], nb0 = a.SC[b_small];
    if (na1 <= 0 || nb1 <= 0) return -INFINITY;
    const float2 qa0f = a.PW[a0], qa1f = a.PW[a1], qb1f = a.SW[b_big], qb0f = a.SW[b_small];
    const F2 qa0{qa0f.x, qa0f.y}, qa1{qa1f.x, qa1f.y}, qb0{qb0f.x, qb0f.y}, qb1{qb1f.x, qb1f.y};
    if (a.q == 1.0f) {
        const F2 la = df_log2_count<true>((unsigned)na1, T), lb = df_log2_count<true>((unsigned)nb1, T);
        const F2 sa = df_div(qa0, df_from_u32((unsigned)na1)), sb = df_div(qb0, df_from_u32((unsigned)nb1));
        const F2 phi = df_mul(df_add(df_add(la, f2_neg(sa)), df_add(lb, f2_neg(sb))), df_ln2());
        return phi.hi + phi.lo;
    }
    const F2 LN{kFixedLog2N, 0.f};
    F2 ab;
    if (a.q < 1.0f) {
        if (na0 <= 0 || nb0 <= 0) return INFINITY;
        const F2 pa = df_pow_ratio<true>((unsigned)na0, LN, a.q, T), pb = df_pow_ratio<true>((unsigned)nb0, LN, a.q, T);
        ab = df_mul(df_div(qa1, pa), df_div(qb1, pb));
    } else {
        const F2 pa = df_pow_ratio<true>((unsigned)na1, LN, a.q, T), pb = df_pow_ratio<true>((unsigned)nb1, LN, a.q, T);
        ab = df_mul(df_div(qa0, pa), df_div(qb0, pb));
    }
    const F2 phi = df_div(df_add(F2{1.0f, 0.f}, f2_neg(ab)), two_sum(a.q, -1.0f));
    return phi.hi + phi.lo;
}

constexpr int kWindowParts = kCells2d / kS2Threads;   // blocks per histogram, one cell per thread

// Window search, kWindowParts blocks per histogram: the objective at every
// pair of the candidate cells (each block computes this maximum itself: 256
// pairs of 16 cells, one per thread), then a flag for each of the block's
// cells: 2 for a candidate, 1 when its bound reaches the candidates' maximum
// (less a margin far above the evaluation's error), 0 otherwise; only
// flagged cells are evaluated. winfo (zeroed by the caller) counts flag 1.
__global__ void __launch_bounds__(kS2Threads) k_s2_window(const S2Args a) {
    __shared__ DfTables sdf;
    df_stage(&sdf, a.T, threadIdx.x, blockDim.x);
    __syncthreads();
    const DfTables* T = &sdf;
    __shared__ unsigned cand_bits[kCells2d / 32];
    __shared__ float wbest[kS2Threads / 32];
    __shared__ int wcount[kS2Threads / 32];
    const int k = blockIdx.x / kWindowParts, part = blockIdx.x % kWindowParts;
    const int tid = threadIdx.x, m = a.L2 - 1;
    for (int i = tid; i < kCells2d / 32; i += kS2Threads) cand_bits[i] = 0u;
    __syncthreads();
    float best = -INFINITY;
    for (int i = tid; i < a.topk * kCell2d * kCell2d; i += kS2Threads) {
        const int c = a.cand[(long long)k * a.topk + i / (kCell2d * kCell2d)];
        if (!in_range(c, kCells2d, a.check, kSite2dCell) || c < 0 || c >= kCells2d) continue;
        if ((i & (kCell2d * kCell2d - 1)) == 0) atomicOr(&cand_bits[c >> 5], 1u << (c & 31));
        const int t = (c / 64) * kCell2d + (i & (kCell2d * kCell2d - 1)) / kCell2d;
        const int s = (c % 64) * kCell2d + (i & (kCell2d - 1));
        if (t >= m || s >= m) continue;
        F2 phi;
        float band;
        if (eval_df(quad_sums(a, k, t, s), a.q, T, phi, band)) best = fmaxf(best, phi.hi + phi.lo);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((tid & 31) == 0) wbest[tid >> 5] = best;
    __syncthreads();
    best = wbest[0];
    for (int w = 1; w < kS2Threads / 32; ++w) best = fmaxf(best, wbest[w]);
    const float thr = best - 1e-6f * fmaxf(fabsf(best), 1.0f);
    const int c = part * kS2Threads + tid;
    const int t0 = (c / 64) * kCell2d, s0 = (c % 64) * kCell2d;
    unsigned char f = 0;
    int searched = 0;
    if ((cand_bits[c >> 5] >> (c & 31)) & 1u) {
        f = 2;
    } else if (t0 < m && s0 < m) {
        const float u = cell_bound(a, T, k, t0, min(t0 + kCell2d - 1, m - 1), s0, min(s0 + kCell2d - 1, m - 1));
        if (u >= thr) {
            f = 1;
            searched = 1;
        }
    }
    a.cellflag[(long long)k * kCells2d + c] = f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) searched += __shfl_xor_sync(0xffffffffu, searched, o);
    if ((tid & 31) == 0) wcount[tid >> 5] = searched;
    __syncthreads();
    if (tid == 0) {
        int n = 0;
        for (int w = 0; w < kS2Threads / 32; ++w) n += wcount[w];
        if (n) atomicAdd(&a.winfo[k], n);
    }
}

__global__ void __launch_bounds__(kS2Threads) k_s2_final(const S2Args a) {
    __shared__ DfTables sdf;
    df_stage(&sdf, a.T, threadIdx.x, blockDim.x);
    __syncthreads();
    const DfTables* T = &sdf;
    __shared__ TopSmem tsm;
    __shared__ RedSmem sm;
    const int k = blockIdx.x, tid = threadIdx.x;
    const int m = a.L2 - 1;
    const long long ro = (long long)k * a.L2;
    Top tp{{-INFINITY, 0.f}, -1, 0.f, -INFINITY};
    for (int t = tid; t < m; t += kS2Threads)
        tp = top_merge(tp, Top{{a.rvh[ro + t], a.rvl[ro + t]}, a.ri[ro + t], a.rband[ro + t], a.ru2[ro + t]});
    const Top g = block_top2(tp, tsm);
    if (g.i < 0) {
        if (tid == 0) {
            a.t_out[2 * k] = -1;
            a.t_out[2 * k + 1] = -1;
            if (a.t_bin) a.t_bin[k] = -1;
            a.phi_out[k] = 0.f;
            a.status[k] = TSALLIS_ERR_NO_VALID_THRESHOLD;
        }
        return;
    }
    const float lower = g.v.hi - g.band;
    if (!(g.u2 >= lower)) {
        if (tid == 0) {
            a.t_out[2 * k] = g.i / m;
            a.t_out[2 * k + 1] = g.i % m;
            if (a.t_bin) a.t_bin[k] = g.i / m;
            a.phi_out[k] = g.v.hi + g.v.lo;
            a.status[k] = TSALLIS_OK | window_bits(a, k, g.i / m, g.i % m);
        }
        return;
    }
    // rows holding a pair inside the bounds (uniform over the block)
    auto row_in = [&](int t) {
        return a.ri[ro + t] >= 0 && (a.rvh[ro + t] + a.rband[ro + t] >= lower || a.ru2[ro + t] >= lower);
    };
    // A pair whose table sums equal its left or upper neighbour's exactly
    // has that smaller pair's partition and value, so it is neither the
    // maximiser nor the canonical pair and gets no FP64 evaluation (most
    // pairs of a plateau; members of one partition whose sums differ in the
    // last bits, from differently associated scans, are still compared).
    auto repeats = [&](const Quad& u, int t, int s) {
        return (s > 0 && same_sums(u, quad_sums(a, k, t, s - 1))) ||
               (t > 0 && same_sums(u, quad_sums(a, k, t - 1, s)));
    };
    double dv = 0.0;
    int di = -1;
    for (int t = 0; t < m; ++t) {
        if (!row_in(t)) continue;
        for (int s = tid; s < m; s += kS2Threads) {
            const Quad u = quad_sums(a, k, t, s);
            F2 phi;
            float band;
            if (eval_df(u, a.q, T, phi, band) && phi.hi + band >= lower && !repeats(u, t, s))
                argmax_merge(dv, di, eval64(u, a.q, T), t * m + s);
        }
    }
    red_argmax_d(dv, di, sm);
    if (di < 0) {   // the maximum is inside its own bound; kept as a guard
        di = g.i;
        dv = eval64(quad_sums(a, k, g.i / m, g.i % m), a.q, T);
    }
    const int wt = di / m, ws = di - wt * m;
    const Quad uw = quad_sums(a, k, wt, ws);
    const double tol = kSamePartitionTol * fmax(fabs(dv), 1.0);
    // canonical pair: the smallest (t, s) with the winner's partition and value
    int ci = 0x7fffffff;
    for (int t = 0; t < m && t <= wt; ++t) {
        if (!row_in(t)) continue;
        for (int s = tid; s < m; s += kS2Threads) {
            if (t * m + s >= di) break;
            const Quad u = quad_sums(a, k, t, s);
            if (u.na != uw.na || u.nb != uw.nb) continue;
            F2 phi;
            float band;
            if (eval_df(u, a.q, T, phi, band) && phi.hi + band >= lower && !repeats(u, t, s) &&
                fabs(eval64(u, a.q, T) - dv) <= tol)
                ci = min(ci, t * m + s);
        }
    }
    ci = min(red_min_i(ci, sm), di);
    if (tid == 0) {
        const int t = ci / m, s = ci - (ci / m) * m;
        a.t_out[2 * k] = t;
        a.t_out[2 * k + 1] = s;
        if (a.t_bin) a.t_bin[k] = t;
        a.phi_out[k] = (float)dv;
        a.status[k] = TSALLIS_OK | TSALLIS_STATUS_RERANKED | window_bits(a, k, t, s);
    }
}

}  // namespace

// ------------------------------------------------------------ host side

// The band, then the row-staging ring (used by the per-slice form only; one size for every form).
int hist2d_smem_bytes(int L2) { return ((L2 * kBandStride + 3) & ~3) * (int)sizeof(int) + kStageBytes; }

cudaError_t seg2d_prepare() {
    const int smem = hist2d_smem_bytes(256);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_hist2d<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_hist2d<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_hist2d<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_hist2d<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_hist2d(const Hist2dLaunch& p, cudaStream_t s) {
    Hist2dArgs a;
    a.vol = p.vol;
    a.nx = p.nx;
    a.ny = p.ny;
    a.nz = p.nz;
    a.lo = p.lo;
    a.hi = p.lo + p.L - 1 < 32767 ? p.lo + p.L - 1 : 32767;
    a.shift = p.shift;
    a.L2 = p.L >> p.shift;
    a.per_slice = p.per_slice;
    const int nq = (p.nx + 3) / 4;
    a.qw = nq >= 128 ? 128 : ((nq + 31) / 32) * 32;
    a.nxb = (nq + a.qw - 1) / a.qw;
    const int rows_per_tile = (kH2Threads / a.qw) * kH2RowsPerGroup;
    a.nyc = (p.ny + rows_per_tile - 1) / rows_per_tile;
    a.ntiles = (long long)p.nz * a.nyc * a.nxb;
    a.ghist = p.hist;
    const bool window3d = !p.per_slice && p.nz > 1;
    const bool vec = (p.nx % 4) == 0 && ((uintptr_t)p.vol & 7u) == 0;
    long long grid = (long long)p.sm_count * p.blocks_per_sm;
    if (grid > a.ntiles) grid = a.ntiles;
    if (grid < 1) grid = 1;
    const int smem = hist2d_smem_bytes(a.L2);
    if (window3d) {
        if (vec) k_hist2d<1, true><<<(int)grid, kH2Threads, smem, s>>>(a);
        else k_hist2d<1, false><<<(int)grid, kH2Threads, smem, s>>>(a);
    } else {
        if (vec) k_hist2d<0, true><<<(int)grid, kH2Threads, smem, s>>>(a);
        else k_hist2d<0, false><<<(int)grid, kH2Threads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t hist2d_occupancy(int* blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_hist2d<1, true>, kH2Threads,
                                                         hist2d_smem_bytes(256));
}

size_t search2d_scratch_bytes(int L2, long long K) {
    const size_t cells = (size_t)K * L2 * L2;
    return cells * (2 * sizeof(int) + 2 * sizeof(float2)) + (size_t)K * L2 * 5 * sizeof(float) + 256;
}

namespace {
S2Args s2_args(const Search2dLaunch& p) {
    const int L2 = p.L2;
    const size_t cells = (size_t)p.K * L2 * L2;
    unsigned char* b = static_cast<unsigned char*>(p.scratch);
    S2Args a;
    a.hist = p.hist;
    a.L2 = L2;
    a.q = p.q;
    a.T = static_cast<const DfTables*>(p.tables);
    a.PW = reinterpret_cast<float2*>(b);
    a.SW = a.PW + cells;
    a.PC = reinterpret_cast<int*>(a.SW + cells);
    a.SC = a.PC + cells;
    float* rows = reinterpret_cast<float*>(a.SC + cells);
    a.rvh = rows;
    a.rvl = rows + (size_t)p.K * L2;
    a.rband = rows + 2 * (size_t)p.K * L2;
    a.ru2 = rows + 3 * (size_t)p.K * L2;
    a.ri = reinterpret_cast<int*>(rows + 4 * (size_t)p.K * L2);
    a.curve = p.curve;
    a.t_out = p.t;
    a.t_bin = p.t_bin;
    a.phi_out = p.phi;
    a.status = p.status;
    a.cand = p.cand;
    a.topk = p.topk;
    a.cellflag = p.cellflag;
    a.winfo = p.winfo;
    a.K = p.K;
    a.check = p.check;
    return a;
}
}  // namespace

cudaError_t launch_search2d_tables(const Search2dLaunch& p, cudaStream_t s) {
    const S2Args a = s2_args(p);
    k_s2_rows<<<dim3(p.L2, (unsigned)p.K), kS2Threads, 0, s>>>(a);
    k_s2_cols<<<dim3((p.L2 + 31) / 32, (unsigned)p.K), 1024, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_search2d_window(const Search2dLaunch& p, cudaStream_t s) {
    if (p.L2 != 256 || !p.cand || !p.cellflag || !p.winfo || p.topk < 1) return cudaErrorInvalidValue;
    if (cudaMemsetAsync(p.winfo, 0, (size_t)p.K * sizeof(int), s) != cudaSuccess) return cudaGetLastError();
    k_s2_window<<<(unsigned)(p.K * kWindowParts), kS2Threads, 0, s>>>(s2_args(p));
    return cudaGetLastError();
}

cudaError_t launch_search2d_finish(const Search2dLaunch& p, cudaStream_t s) {
    const S2Args a = s2_args(p);
    k_s2_eval<<<dim3(p.L2 - 1, (unsigned)p.K), kS2Threads, 0, s>>>(a);
    k_s2_final<<<(unsigned)p.K, kS2Threads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_search2d(const Search2dLaunch& p, cudaStream_t s) {
    const cudaError_t e = launch_search2d_tables(p, s);
    return e != cudaSuccess ? e : launch_search2d_finish(p, s);
}

}  // namespace tsl
