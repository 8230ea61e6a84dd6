// Device building blocks shared by the kernels of the thresholding path.
//
// Method: maximum Tsallis entropy threshold (section II-C "Segmentation",
// "Tsallis entropy"), 1-D reading: for a threshold t, class 1 holds levels
// 0..t and class 2 levels t+1..L-1. With counts h_i, N_1 = sum_{i<=t} h_i,
// Q_1 = sum_{i<=t} h_i^q (and the same over i > t for class 2),
//     sum_{i in class k} (p_i / P_k)^q = Q_k / N_k^q,
// the normalisation p_i = h_i / N cancels, and the pseudo-additive objective
//     phi = H_1 + H_2 + (1 - q) H_1 H_2,  H_k = (1 - Q_k / N_k^q) / (q - 1)
// equals (1 - a b) / (q - 1) with a = Q_1 / N_1^q, b = Q_2 / N_2^q.
// At q = 1 (Shannon limit) H_k = ln N_k - (sum h ln h) / N_k and phi = H_1 + H_2.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tsl {

constexpr int kMaxBins = 4096;  // equals kMaxLevels of kernels.h

// ------------------------------------------------------------ compensated FP32
// A value held as an unevaluated sum hi + lo (Knuth's TwoSum error-free
// transformation). All summands on this path are >= 0.
struct F2 {
    float hi, lo;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ F2 f2_add(F2 x, F2 y) {
    F2 s = two_sum(x.hi, y.hi);
    float lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    float hi = __fadd_rn(s.hi, lo);                 // renormalise (fast two-sum)
    return {hi, __fsub_rn(lo, __fsub_rn(hi, s.hi))};
}

__device__ __forceinline__ float f2_val(F2 x) { return __fadd_rn(x.hi, x.lo); }

__device__ __forceinline__ F2 shfl_up_f2(F2 v, int d) {
    return {__shfl_up_sync(0xffffffffu, v.hi, d), __shfl_up_sync(0xffffffffu, v.lo, d)};
}
__device__ __forceinline__ F2 shfl_down_f2(F2 v, int d) {
    return {__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d)};
}

// Inclusive warp scans.
__device__ __forceinline__ long long warp_prefix_i64(long long v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        long long o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    return v;
}
__device__ __forceinline__ F2 warp_prefix_f2(F2 v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        F2 o = shfl_up_f2(v, d);
        if (lane >= d) v = f2_add(o, v);
    }
    return v;
}
__device__ __forceinline__ F2 warp_suffix_f2(F2 v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        F2 o = shfl_down_f2(v, d);
        if (lane + d < 32) v = f2_add(v, o);
    }
    return v;
}
// (value, index) maximum; equal values keep the smaller index.
template <typename T>
__device__ __forceinline__ void argmax_merge(T& v, int& i, T ov, int oi) {
    if (oi >= 0 && (i < 0 || ov > v || (ov == v && oi < i))) { v = ov; i = oi; }
}
template <typename T>
__device__ __forceinline__ void warp_argmax(T& v, int& i) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, v, d);
        int oi = __shfl_xor_sync(0xffffffffu, i, d);
        argmax_merge(v, i, ov, oi);
    }
}

// ------------------------------------------------------------ error band
// Bound on |phi_fp32 - phi_exact| used to decide which thresholds may still
// beat the FP32 maximiser. The class sums come from double-float sums, so
// rounding them to float costs 0.5 ulp each; the class powers (N_k/N)^q use
// powf, which CUDA documents to 4 ulp, on a ratio carrying 1.5 ulp (two
// int->float roundings and a division), i.e. 4 + 1.5 q ulp; the two
// divisions and the product add 0.5 ulp each. So ab is within
// (10.5 + 3 q) ulp, 1 ulp <= 2^-23 relative, and
//     |dphi| <= |ab| * (10.5 + 3 q) 2^-23 / |q - 1| + 1 ulp of phi.
// The constants below carry a further factor of two as margin.
__device__ __forceinline__ float tsallis_err(float ab, float phi, float q) {
    float rel = 2.51e-6f + 7.16e-7f * q;
    return rel * fabsf(ab) / fabsf(q - 1.0f) + 2.4e-7f * fabsf(phi);
}
// Shannon limit, in bits: H_k / ln 2 = log2 N_k - S_k / N_k. log2f is within
// 1 ulp, S_k / N_k within 1.5 ulp, each subtraction and the final scaling
// within 0.5 ulp; the bound below is several times that.
__device__ __forceinline__ float shannon_err(float la, float sa, float lb, float sb, float phi_bits) {
    return 1.0e-6f * (fabsf(la) + fabsf(sa) + fabsf(lb) + fabsf(sb) + fabsf(phi_bits) + 1.0f);
}

// ------------------------------------------------------------ 1-D search
// One thread block searches one histogram of L <= 4096 levels.
constexpr int kSearchThreads = 512;
constexpr int kBinsPerThread = kMaxBins / kSearchThreads;  // 8
constexpr int kSearchWarps = kSearchThreads / 32;

struct SearchSmem {
    long long cnt_pre[kSearchWarps];
    F2 w_pre[kSearchWarps];
    F2 w_suf[kSearchWarps];
    float red_v[kSearchWarps];
    int red_i[kSearchWarps];
    double red_dv[kSearchWarps];
    long long total;
    float best_err;
    int nlevels;        // non-empty levels (compaction)
    int flag;
    // per-warp running tops of the table search
    float top_vh[kSearchWarps], top_vl[kSearchWarps], top_band[kSearchWarps], top_u2[kSearchWarps];
    int top_i[kSearchWarps];
};

struct SearchResult {
    int t;          // -1 when no threshold is valid
    float phi;
    int status;     // tsallis_status | extra bits
};


// ------------------------------------------------------------ streaming tiles

__device__ __forceinline__ void st_stream(void* p, uint2 v) {
    asm volatile("st.global.cs.v2.u32 [%0], {%1,%2};" ::"l"(p), "r"(v.x), "r"(v.y) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

}  // namespace tsl
