// The 2-D search as the paper's GPU code organises it (section III, Table 4:
// one thread per threshold pair, 256 blocks of 256 threads for 256 grey
// levels): the thread of pair (t, s) sums its two quadrants directly,
// A = {i <= t, j <= s} and B = {i > t, j > s}, with no prefix sums or
// summed-area tables, O(L^2) work per pair and O(L^4) per histogram. Kept
// as a comparison point for the summed-area search of seg2d.cu and as a
// second, independently organised implementation of the same objective.
//
// Per histogram k and grey threshold t, one block; thread s holds pair
// (t, s). Row i of the histogram and of its term table (h^q, or h ln h at
// q = 1, as a pair of floats hi + lo) is staged in shared memory and every
// thread adds its part of the row: j <= s when i <= t, j > s when i > t
// (all threads read the same element at a time, a broadcast). Counts are
// summed exactly in integers. Each row's part of a quadrant's terms is a
// compensated FP32 sum (two-sum of the hi parts, their rounding errors and
// the lo parts gathered in a second float); the row sums are added in FP64.
// That bounds the relative error of a quadrant sum (kSumRelErr below), and
// each pair's objective, formed in FP64, carries a bound derived from it.
//
// The final kernel takes the largest lower bound (value - bound) over all
// pairs; every pair whose upper bound reaches it may be the maximiser. Each
// such pair is mapped to the smallest pair of its partition (rows t'+1..t
// and columns s'+1..s empty: the same quadrants), and these candidates are
// evaluated again in plain FP64 from the histogram. The largest FP64 value
// wins, the smallest (t, s) among equal values.
#include <math.h>

#include "checked.cuh"
#include "kernels.h"
#include "tsallis.h"

namespace tsl {
namespace {

constexpr int kBruteThreads = 256;
constexpr int kBruteWarps = kBruteThreads / 32;
constexpr int kMaxPairs = 255 * 255;

// Relative error bound of a quadrant sum. A term hi + lo is within
// 2^-48 + 2^-51 relative of h^q. In a row's compensated sum of n <= 256
// positive terms with total R, each two-sum error and each lo is at most
// 2^-24 R, so the second float stays below 2k 2^-24 R after k terms and its
// own roundings add at most (n^2 + 3n) 2^-48 R < 2.4e-10 R. The FP64 sum of
// at most 256 rows adds 256 * 2^-53. Taken with margin:
constexpr double kSumRelErr = 3e-10;

struct BruteArgs {
    const int* hist;        // [K][L2][L2]
    const float2* T;        // [K][L2][L2] terms (hi, lo)
    int L2;
    float q;
    float* curve;           // optional [K][L2-1][L2-1]
    double* upper;          // [K][L2-1][L2-1] value + bound; -inf for invalid pairs
    double* best_lo;        // [K][L2-1] per t: the largest value - bound over s
    int* t_out;             // [K][2]
    int* t_bin;             // optional [K]
    float* phi_out;
    int* status;
    long long K;
    unsigned* check;        // checked build: first failing index check
};

__global__ void k_brute_terms(const int* hist, long long n, float q, float2* T) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int h = hist[i];
        double v = 0.0;
        if (h > 0) v = (q == 1.0f) ? (double)h * log((double)h) : pow((double)h, (double)q);
        const float hi = (float)v;
        T[i] = make_float2(hi, (float)(v - (double)hi));
    }
}

// r + c += x.hi + x.lo: Knuth's two-sum of the hi parts; the exact rounding
// error and the lo part go to c.
__device__ __forceinline__ void comp_add(float& r, float& c, float2 x) {
    const float t = r + x.x;
    const float z = t - r;
    c += ((r - (t - z)) + (x.x - z)) + x.y;
    r = t;
}

// The objective in FP64 from exact counts and quadrant sums, and (when err
// is given) a bound on its error when SA and SB are within kSumRelErr
// relative. q = 1: ln N_A - S_A / N_A + ln N_B - S_B / N_B (S = sum h ln h);
// else (1 - a b) / (q - 1), a = S_A / N_A^q, b = S_B / N_B^q.
__device__ __forceinline__ double objective(double NA, double NB, double SA, double SB, float qf, double* err) {
    if (qf == 1.0f) {
        const double ra = SA / NA, rb = SB / NB, la = log(NA), lb = log(NB);
        const double phi = (la - ra) + (lb - rb);
        if (err) *err = kSumRelErr * (ra + rb) + 1e-14 * (fabs(la) + fabs(lb) + ra + rb);
        return phi;
    }
    const double q = (double)qf;
    const double ab = (SA / pow(NA, q)) * (SB / pow(NB, q));
    const double phi = (1.0 - ab) / (q - 1.0);
    if (err) {
        // d phi = -(b da + a db) / (q - 1), |da| <= eps a, |db| <= eps b
        const double g = ab / fabs(q - 1.0);
        *err = 2.5 * kSumRelErr * g + 1e-14 * (fabs(phi) + g);
    }
    return phi;
}

__global__ void __launch_bounds__(kBruteThreads) k_brute_pairs(const BruteArgs a) {
    __shared__ float2 sT[256];
    __shared__ int sH[256];
    __shared__ double red[kBruteWarps];
    const int t = blockIdx.x, k = blockIdx.y, s = threadIdx.x;
    const int L2 = a.L2, m = L2 - 1;
    const long long base = (long long)k * L2 * L2;
    unsigned int nA = 0, nB = 0;            // a histogram holds fewer than 2^31 voxels
    double SA = 0.0, SB = 0.0;
    for (int i = 0; i < L2; ++i) {
        __syncthreads();
        const bool row_ok = in_range(base + (long long)i * L2 + L2 - 1, a.K * L2 * L2, a.check, kSite2dBrute);
        for (int j = threadIdx.x; j < L2; j += kBruteThreads) {
            sT[j] = row_ok ? a.T[base + (long long)i * L2 + j] : make_float2(0.f, 0.f);
            sH[j] = row_ok ? a.hist[base + (long long)i * L2 + j] : 0;
        }
        __syncthreads();
        if (s < m) {
            float r = 0.f, c = 0.f;
            if (i <= t) {
                for (int j = 0; j <= s; ++j) {
                    nA += (unsigned)sH[j];
                    comp_add(r, c, sT[j]);
                }
                SA += (double)r + (double)c;
            } else {
                for (int j = s + 1; j < L2; ++j) {
                    nB += (unsigned)sH[j];
                    comp_add(r, c, sT[j]);
                }
                SB += (double)r + (double)c;
            }
        }
    }
    const bool ok = s < m && nA > 0 && nB > 0;
    double phi = 0.0, err = 0.0;
    if (ok) phi = objective((double)nA, (double)nB, SA, SB, a.q, &err);
    if (s < m) {
        const long long o = ((long long)k * m + t) * m + s;
        if (a.curve) a.curve[o] = ok ? (float)phi : __int_as_float(0x7fc00000);
        a.upper[o] = ok ? phi + err : -INFINITY;
    }
    // the block's largest lower bound
    double v = ok ? phi - err : -INFINITY;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, d));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kBruteWarps; ++w) v = fmax(v, red[w]);
        a.best_lo[(long long)k * m + t] = v;
    }
}

// One block per histogram: candidates, then their FP64 re-rank.
__global__ void __launch_bounds__(kBruteThreads) k_brute_final(const BruteArgs a) {
    __shared__ unsigned cand[(kMaxPairs + 31) / 32];
    __shared__ int row_ne[256], last_row[256], last_col[256];
    __shared__ double red_v[kBruteWarps];
    __shared__ int red_i[kBruteWarps];
    const int k = blockIdx.x, L2 = a.L2, m = L2 - 1, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const long long base = (long long)k * L2 * L2;
    const int* h = a.hist + base;
    const float2* T = a.T + base;

    // the largest lower bound over all pairs
    double lmax = -INFINITY;
    for (int t = tid; t < m; t += kBruteThreads) lmax = fmax(lmax, a.best_lo[(long long)k * m + t]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, d));
    if (lane == 0) red_v[warp] = lmax;
    for (int i = tid; i < L2; i += kBruteThreads) row_ne[i] = 0;
    for (int i = tid; i < (m * m + 31) / 32; i += kBruteThreads) cand[i] = 0u;
    __syncthreads();
    lmax = red_v[0];
    for (int w = 1; w < kBruteWarps; ++w) lmax = fmax(lmax, red_v[w]);
    if (lmax == -INFINITY) {   // no pair splits the histogram into two non-empty quadrants
        if (tid == 0) {
            a.t_out[2 * k] = -1;
            a.t_out[2 * k + 1] = -1;
            if (a.t_bin) a.t_bin[k] = -1;
            a.phi_out[k] = 0.f;
            a.status[k] = TSALLIS_ERR_NO_VALID_THRESHOLD;
        }
        return;
    }
    // occupied rows and columns (thread j reads column j: coalesced rows)
    bool col_ne = false;
    for (int i = 0; i < L2; ++i) {
        const bool nz = tid < L2 && h[(long long)i * L2 + tid] > 0;
        col_ne |= nz;
        if (__any_sync(0xffffffffu, nz) && lane == 0) atomicOr(&row_ne[i], 1);
    }
    __syncthreads();
    if (tid < L2) last_col[tid] = col_ne ? tid : -1;
    if (tid < L2) last_row[tid] = row_ne[tid] ? tid : -1;
    __syncthreads();
    if (tid == 0) {
        for (int i = 1; i < L2; ++i) {
            last_row[i] = max(last_row[i], last_row[i - 1]);
            last_col[i] = max(last_col[i], last_col[i - 1]);
        }
    }
    __syncthreads();
    // pairs that may be the maximiser, as the smallest pair of their partition
    const double* up = a.upper + (long long)k * m * m;
    for (int p = tid; p < m * m; p += kBruteThreads) {
        if (up[p] >= lmax) {
            const int t = p / m, s = p - t * m;
            const int c = last_row[t] * m + last_col[s];   // both >= 0: the pair is valid
            atomicOr(&cand[c >> 5], 1u << (c & 31));
        }
    }
    __syncthreads();
    // FP64 re-rank: warp w takes bitmap words w, w + 8, ... (increasing pairs
    // within a warp, so a strictly larger value is needed to replace its best)
    double bv = -INFINITY;
    int bi = -1;
    for (int w = warp; w < (m * m + 31) / 32; w += kBruteWarps) {
        unsigned bits = cand[w];
        while (bits) {
            const int c = w * 32 + __ffs(bits) - 1;
            bits &= bits - 1;
            const int t = c / m, s = c - t * m;
            long long nA = 0, nB = 0;
            double SA = 0.0, SB = 0.0;
            for (int i = 0; i < L2; ++i) {
                const bool in_a = i <= t;   // row i meets A in columns 0..s, B in s+1..L2-1
                const int j1 = in_a ? s + 1 : L2;
                for (int j = (in_a ? 0 : s + 1) + lane; j < j1; j += 32) {
                    const int n = h[(long long)i * L2 + j];
                    if (n == 0) continue;
                    const float2 x = T[(long long)i * L2 + j];
                    const double tv = (double)x.x + (double)x.y;
                    if (in_a) { nA += n; SA += tv; }
                    else { nB += n; SB += tv; }
                }
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                nA += __shfl_xor_sync(0xffffffffu, nA, d);
                nB += __shfl_xor_sync(0xffffffffu, nB, d);
                SA += __shfl_xor_sync(0xffffffffu, SA, d);
                SB += __shfl_xor_sync(0xffffffffu, SB, d);
            }
            const double phi = objective((double)nA, (double)nB, SA, SB, a.q, nullptr);
            if (nA > 0 && nB > 0 && (bi < 0 || phi > bv)) { bv = phi; bi = c; }
        }
    }
    if (lane == 0) {
        red_v[warp] = bv;
        red_i[warp] = bi;
    }
    __syncthreads();
    if (tid != 0) return;
    for (int w = 1; w < kBruteWarps; ++w) {
        const double v2 = red_v[w];
        const int i2 = red_i[w];
        if (i2 >= 0 && (bi < 0 || v2 > bv || (v2 == bv && i2 < bi))) { bv = v2; bi = i2; }
    }
    if (bi < 0) {   // cannot happen: the pair of the largest lower bound is a candidate
        a.t_out[2 * k] = -1;
        a.t_out[2 * k + 1] = -1;
        if (a.t_bin) a.t_bin[k] = -1;
        a.phi_out[k] = 0.f;
        a.status[k] = TSALLIS_ERR_NO_VALID_THRESHOLD;
        return;
    }
    const int t = bi / m, s = bi - t * m;
    a.t_out[2 * k] = t;
    a.t_out[2 * k + 1] = s;
    if (a.t_bin) a.t_bin[k] = t;
    a.phi_out[k] = (float)bv;
    a.status[k] = TSALLIS_OK;
}

size_t align256b(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t search2d_brute_scratch_bytes(int L2, long long K) {
    const size_t m = (size_t)(L2 > 1 ? L2 - 1 : 1);
    return align256b((size_t)K * L2 * L2 * sizeof(float2)) + align256b((size_t)K * m * m * sizeof(double)) +
           (size_t)K * m * sizeof(double);
}

cudaError_t launch_search2d_brute(const Search2dLaunch& p, cudaStream_t s) {
    const int L2 = p.L2;
    if (L2 < 2 || L2 > kBruteThreads || p.K < 1 || p.K > 65535) return cudaErrorInvalidValue;
    const size_t m = (size_t)(L2 - 1);
    unsigned char* b = static_cast<unsigned char*>(p.scratch);
    BruteArgs a;
    a.hist = p.hist;
    float2* T = reinterpret_cast<float2*>(b);
    b += align256b((size_t)p.K * L2 * L2 * sizeof(float2));
    a.upper = reinterpret_cast<double*>(b);
    b += align256b((size_t)p.K * m * m * sizeof(double));
    a.best_lo = reinterpret_cast<double*>(b);
    a.T = T;
    a.L2 = L2;
    a.q = p.q;
    a.curve = p.curve;
    a.t_out = p.t;
    a.t_bin = p.t_bin;
    a.phi_out = p.phi;
    a.status = p.status;
    a.K = p.K;
    a.check = p.check;
    const long long n = p.K * L2 * L2;
    k_brute_terms<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p.hist, n, p.q, T);
    dim3 grid((unsigned)(L2 - 1), (unsigned)p.K);
    k_brute_pairs<<<grid, kBruteThreads, 0, s>>>(a);
    k_brute_final<<<(unsigned)p.K, kBruteThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace tsl
