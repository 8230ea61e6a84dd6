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
// q = 1) is staged in shared memory and every thread adds its part of the
// row: j <= s when i <= t, j > s when i > t (all threads read the same
// element at a time, a broadcast). Counts are summed exactly in integers;
// terms are FP32 (the paper's precision) summed with an error-free
// transformation (two-sum) so that the sum carries its rounding error; each
// pair's objective H_A + H_B + (1-q) H_A H_B is then formed in FP64. The
// block keeps its best s (smallest s among equal values), a second kernel
// the best t (smallest t among equal values): the smallest (t, s) overall.
#include <math.h>

#include "checked.cuh"
#include "kernels.h"
#include "tsallis.h"

namespace tsl {
namespace {

constexpr int kBruteThreads = 256;

struct BruteArgs {
    const int* hist;        // [K][L2][L2]
    const float* T;         // [K][L2][L2] terms
    int L2;
    float q;
    float* curve;           // optional [K][L2-1][L2-1]
    double* best_phi;       // [K][L2-1]
    int* best_s;            // [K][L2-1]
    int* t_out;             // [K][2]
    int* t_bin;             // optional [K]
    float* phi_out;
    int* status;
    long long K;
    unsigned* check;        // checked build: first failing index check
};

__global__ void k_brute_terms(const int* hist, long long n, float q, float* T) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int h = hist[i];
        double v = 0.0;
        if (h > 0) v = (q == 1.0f) ? (double)h * log((double)h) : pow((double)h, (double)q);
        T[i] = (float)v;
    }
}

// s += x with the rounding error accumulated in c (Knuth's two-sum).
__device__ __forceinline__ void two_sum_add(float& s, float& c, float x) {
    const float t = s + x;
    const float z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
}

__global__ void __launch_bounds__(kBruteThreads) k_brute_pairs(const BruteArgs a) {
    __shared__ float sT[256];
    __shared__ int sH[256];
    __shared__ double red_v[kBruteThreads / 32];
    __shared__ int red_s[kBruteThreads / 32];
    const int t = blockIdx.x, k = blockIdx.y, s = threadIdx.x;
    const int L2 = a.L2, m = L2 - 1;
    const long long base = (long long)k * L2 * L2;
    unsigned int nA = 0, nB = 0;            // a histogram holds fewer than 2^31 voxels
    float sa = 0.f, ca = 0.f, sb = 0.f, cb = 0.f;
    for (int i = 0; i < L2; ++i) {
        __syncthreads();
        const bool row_ok = in_range(base + (long long)i * L2 + L2 - 1, a.K * L2 * L2, a.check, kSite2dBrute);
        for (int j = threadIdx.x; j < L2; j += kBruteThreads) {
            sT[j] = row_ok ? a.T[base + (long long)i * L2 + j] : 0.f;
            sH[j] = row_ok ? a.hist[base + (long long)i * L2 + j] : 0;
        }
        __syncthreads();
        if (s < m) {
            if (i <= t) {
                for (int j = 0; j <= s; ++j) {
                    nA += (unsigned)sH[j];
                    two_sum_add(sa, ca, sT[j]);
                }
            } else {
                for (int j = s + 1; j < L2; ++j) {
                    nB += (unsigned)sH[j];
                    two_sum_add(sb, cb, sT[j]);
                }
            }
        }
    }
    double phi = -INFINITY;
    bool ok = false;
    if (s < m && nA > 0 && nB > 0) {
        const double SA = (double)sa + (double)ca, SB = (double)sb + (double)cb;
        const double q = (double)a.q, NA = (double)nA, NB = (double)nB;
        double HA, HB;
        if (a.q == 1.0f) {
            // Shannon limit: H = ln N - (1/N) sum h ln h
            HA = log(NA) - SA / NA;
            HB = log(NB) - SB / NB;
            phi = HA + HB;
        } else {
            // H = (1 - sum (h/N)^q) / (q - 1)
            HA = (1.0 - SA / pow(NA, q)) / (q - 1.0);
            HB = (1.0 - SB / pow(NB, q)) / (q - 1.0);
            phi = HA + HB + (1.0 - q) * HA * HB;
        }
        ok = true;
    }
    if (a.curve && s < m)
        a.curve[((long long)k * m + t) * m + s] = ok ? (float)phi : __int_as_float(0x7fc00000);
    // block maximum over s, smallest s among equal values
    double v = ok ? phi : -INFINITY;
    int si = ok ? s : -1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int s2 = __shfl_xor_sync(0xffffffffu, si, o);
        if (s2 >= 0 && (si < 0 || v2 > v || (v2 == v && s2 < si))) { v = v2; si = s2; }
    }
    if ((threadIdx.x & 31) == 0) {
        red_v[threadIdx.x >> 5] = v;
        red_s[threadIdx.x >> 5] = si;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kBruteThreads / 32; ++w) {
            const double v2 = red_v[w];
            const int s2 = red_s[w];
            if (s2 >= 0 && (si < 0 || v2 > v || (v2 == v && s2 < si))) { v = v2; si = s2; }
        }
        a.best_phi[(long long)k * m + t] = v;
        a.best_s[(long long)k * m + t] = si;
    }
}

__global__ void __launch_bounds__(kBruteThreads) k_brute_final(const BruteArgs a) {
    __shared__ double red_v[kBruteThreads / 32];
    __shared__ int red_t[kBruteThreads / 32];
    const int k = blockIdx.x, m = a.L2 - 1;
    double v = -INFINITY;
    int ti = -1;
    for (int t = threadIdx.x; t < m; t += kBruteThreads) {
        const int s2 = a.best_s[(long long)k * m + t];
        const double v2 = a.best_phi[(long long)k * m + t];
        if (s2 >= 0 && (ti < 0 || v2 > v)) { v = v2; ti = t; }   // t ascends within a thread
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int t2 = __shfl_xor_sync(0xffffffffu, ti, o);
        if (t2 >= 0 && (ti < 0 || v2 > v || (v2 == v && t2 < ti))) { v = v2; ti = t2; }
    }
    if ((threadIdx.x & 31) == 0) {
        red_v[threadIdx.x >> 5] = v;
        red_t[threadIdx.x >> 5] = ti;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < kBruteThreads / 32; ++w) {
        const double v2 = red_v[w];
        const int t2 = red_t[w];
        if (t2 >= 0 && (ti < 0 || v2 > v || (v2 == v && t2 < ti))) { v = v2; ti = t2; }
    }
    if (ti < 0) {
        a.t_out[2 * k] = -1;
        a.t_out[2 * k + 1] = -1;
        if (a.t_bin) a.t_bin[k] = -1;
        a.phi_out[k] = 0.f;
        a.status[k] = TSALLIS_ERR_NO_VALID_THRESHOLD;
        return;
    }
    a.t_out[2 * k] = ti;
    a.t_out[2 * k + 1] = a.best_s[(long long)k * m + ti];
    if (a.t_bin) a.t_bin[k] = ti;
    a.phi_out[k] = (float)v;
    a.status[k] = TSALLIS_OK;
}

size_t align256b(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t search2d_brute_scratch_bytes(int L2, long long K) {
    return align256b((size_t)K * L2 * L2 * sizeof(float)) + align256b((size_t)K * L2 * sizeof(double)) +
           (size_t)K * L2 * sizeof(int);
}

cudaError_t launch_search2d_brute(const Search2dLaunch& p, cudaStream_t s) {
    const int L2 = p.L2;
    if (L2 < 2 || L2 > kBruteThreads || p.K < 1 || p.K > 65535) return cudaErrorInvalidValue;
    unsigned char* b = static_cast<unsigned char*>(p.scratch);
    BruteArgs a;
    a.hist = p.hist;
    float* T = reinterpret_cast<float*>(b);
    b += align256b((size_t)p.K * L2 * L2 * sizeof(float));
    a.best_phi = reinterpret_cast<double*>(b);
    b += align256b((size_t)p.K * L2 * sizeof(double));
    a.best_s = reinterpret_cast<int*>(b);
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
