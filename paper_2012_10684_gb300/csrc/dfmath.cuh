// Double-float ("float-float") arithmetic on the FP32 pipe.
//
// A value is an unevaluated sum hi + lo of two floats (about 48 significant
// bits). GB300 has a very low FP64 rate, so every O(L) high-precision step of
// the search (terms h^q, their sums) runs here instead, and FP64 is kept for
// the final comparison of a few near-tied candidates.
//
// Building blocks: Knuth's TwoSum and the FMA-based TwoProduct error-free
// transformations (Dekker 1971; Ogita, Rump & Oishi 2005). log2 and exp2 are
// table-driven in the manner of P. T. P. Tang (ACM TOMS 15 (1989) 144-157 and
// 16 (1990) 378-400): a 128-entry reciprocal table reduces the log argument
// to |r| <= 2^-8, a 65-entry 2^(j/64) table reduces the exp argument to
// |s| <= 2^-7, and short Taylor series finish both. Relative error of
// df_pow_ratio is below 1e-12 for counts below 2^31 and q in (0, 4]
// (tested on the GPU against numpy's double-precision power).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace tsl {

// Tables, filled on the host in double precision and split into float
// pairs. Stored in global memory; kernels copy them into shared memory
// (df_stage) before use, since every power reads them at diverging indices
// on its dependent path, where a global load costs a round trip to L2.
struct DfTables {
    float4 lg[128];  // x: float(1 / c_j), c_j = 1 + (j + 0.5) / 128; y, z: -log2(x) as hi, lo
    float2 ex[65];   // 2^((j - 32) / 64) as hi, lo
    const float2* lt;   // log2(h) as hi, lo for 0 <= h <= lt_max (built on the device)
    int lt_max;
};

// Copies the tables (global memory) into dst (shared memory); threads
// tid = 0 .. n-1 of the caller take part, and the caller synchronises them
// before the copy is used. The big log2 table stays in global memory.
__device__ __forceinline__ void df_stage(DfTables* dst, const DfTables* __restrict__ src, int tid, int n) {
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    for (int i = tid; i < (int)(sizeof(DfTables) / sizeof(int)); i += n) d[i] = __ldg(s + i);
}

__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ F2 two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// Accurate addition for operands of any sign.
__device__ __forceinline__ F2 df_add(F2 x, F2 y) {
    F2 s = two_sum(x.hi, y.hi);
    F2 t = two_sum(x.lo, y.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ F2 df_mul(F2 x, F2 y) {
    F2 p = two_prod(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ F2 df_mul_f(F2 x, float y) {
    F2 p = two_prod(x.hi, y);
    return fast_two_sum(p.hi, __fmaf_rn(x.lo, y, p.lo));
}

__device__ __forceinline__ double df_to_double(F2 x) { return (double)x.hi + (double)x.lo; }

// An unsigned count as an exact float pair (h < 2^32).
__device__ __forceinline__ F2 df_from_u32(unsigned h) {
    float hf = __uint2float_rn(h);
    // h - hf is exact in int arithmetic; hf <= 2^32 so compare in 64 bits
    long long d = (long long)h - (long long)hf;
    return {hf, (float)d};
}

// log(2) and log2(e) as float pairs.
__device__ __forceinline__ F2 df_ln2() { return {0.693147182464599609375f, -1.904654323148236e-09f}; }
__device__ __forceinline__ F2 df_log2e() { return {1.44269502162933349609375f, 1.925963033500011e-08f}; }

// log2(h) for an integer h >= 1.
static __device__ __noinline__ F2 df_log2_u32(unsigned h, const DfTables* __restrict__ T) {
    if (h == 1u) return {0.f, 0.f};
    F2 hh = df_from_u32(h);
    const int e = ((__float_as_int(hh.hi) >> 23) & 0xff) - 127;
    const float sc = __int_as_float((127 - e) << 23);    // 2^-e, exact
    const float mh = hh.hi * sc, ml = hh.lo * sc;       // m = h / 2^e in [1, 2)
    int j = (int)((mh - 1.0f) * 128.0f);
    j = j > 127 ? 127 : j;
    const float4 tj = T->lg[j];
    // r = m * inv_j - 1, |r| <= 2^-8
    F2 p = two_prod(mh, tj.x);
    F2 r = fast_two_sum(__fsub_rn(p.hi, 1.0f), __fmaf_rn(ml, tj.x, p.lo));
    // ln(1 + r) = r - r^2/2 + r^3 (1/3 - r/4 + r^2/5); truncation < 2^-48 / 6
    F2 r2 = df_mul(r, r);
    F2 ln1p = df_add(r, F2{-0.5f * r2.hi, -0.5f * r2.lo});
    const float rh = r.hi;
    const float c = rh * rh * rh * __fmaf_rn(rh, __fmaf_rn(rh, 0.2f, -0.25f), 0.333333343267f);
    ln1p = df_add(ln1p, F2{c, 0.f});
    F2 l2 = df_mul(ln1p, df_log2e());
    F2 res = df_add(F2{(float)e, 0.f}, F2{tj.y, tj.z});
    return df_add(res, l2);
}

// 2^y for -126 < y < 127. Returns a float pair (the low part may lose bits
// when y is near the bottom of that range).
__device__ __forceinline__ F2 df_exp2(F2 y, const DfTables* __restrict__ T) {
    const float k = rintf(y.hi);
    F2 f = fast_two_sum(__fsub_rn(y.hi, k), y.lo);       // |f| <= 1/2 + tiny
    const float jf = rintf(f.hi * 64.0f);                 // -32..32
    F2 s = fast_two_sum(__fsub_rn(f.hi, jf * 0.015625f), f.lo);  // exact hi difference (Sterbenz)
    F2 x = df_mul(s, df_ln2());                           // |x| <= ln2 / 128
    // exp(x) = 1 + x + x^2/2 + x^3 (1/6 + x/24 + x^2/120); truncation < 4e-17
    F2 x2 = df_mul(x, x);
    F2 ex = df_add(F2{1.0f, 0.f}, x);
    ex = df_add(ex, F2{0.5f * x2.hi, 0.5f * x2.lo});
    const float xh = x.hi;
    const float tail = xh * xh * xh * __fmaf_rn(xh, __fmaf_rn(xh, 8.33333376795e-3f, 4.16666679084e-2f),
                                               0.166666671634f);
    ex = df_add(ex, F2{tail, 0.f});
    const float2 tj = T->ex[(int)jf + 32];
    F2 r = df_mul(F2{tj.x, tj.y}, ex);
    const int ki = (int)k;
    return {ldexpf(r.hi, ki), ldexpf(r.lo, ki)};
}

// log2(h) of a count. kTable: counts up to lt_max are read from the table
// in global memory; otherwise log2 is computed in registers. Both give the
// same bits (the table is filled by df_log2_u32). The table saves
// instructions where a load is cheap (a search kernel that runs alone);
// computing avoids a dependent global load where the memory system is busy
// (the search inside the streaming kernel).
template <bool kTable>
__device__ __forceinline__ F2 df_log2_count(unsigned h, const DfTables* __restrict__ T) {
    if (kTable && h <= (unsigned)T->lt_max) {
        const float2 v = __ldg(&T->lt[h]);
        return {v.x, v.y};
    }
    return df_log2_u32(h, T);
}

// Terms are carried scaled by 2^64: for q <= 4 and N < 2^31 the smallest
// term (1/N)^q is above 2^-124, so scaled terms and their low parts stay in
// the normal float range. The scale cancels in every ratio Q_k / (N_k/N)^q.
constexpr float kTermScale = 18446744073709551616.0f;  // 2^64
constexpr int kTermScaleLog2 = 64;

// 2^64 (h / N)^q for integers 1 <= h <= N, given LN = log2(N). Kept out of
// line: it is called from several places and its body is long.
template <bool kTable>
static __device__ __noinline__ F2 df_pow_ratio(unsigned h, F2 LN, float q, const DfTables* __restrict__ T) {
    F2 lh = df_log2_count<kTable>(h, T);
    F2 d = df_add(lh, F2{-LN.hi, -LN.lo});                // log2(h / N) <= 0
    F2 y = df_add(df_mul_f(d, q), F2{(float)kTermScaleLog2, 0.f});
    return df_exp2(y, T);
}

// h * log2(h) as a float pair (the Shannon-limit term, in bits).
template <bool kTable>
__device__ __forceinline__ F2 df_hlog2h(unsigned h, const DfTables* __restrict__ T) {
    if (h <= 1u) return {0.f, 0.f};
    return df_mul(df_from_u32(h), df_log2_count<kTable>(h, T));
}

// FP32 class power 2^64 (n / N)^q for the objective's first pass. Small
// counts use the log2 table and exp2f with a first-order correction for the
// low part of the exponent (within 3.5 ulp: exp2f is documented to 2 ulp);
// larger ones use powf (documented to 4 ulp, plus 1.5 q ulp from rounding
// n / N). Both stay inside the error band used by the search.
template <bool kTable>
__device__ __forceinline__ float class_pow_f32(long long n, float fN, F2 LN, float q, const DfTables* __restrict__ T) {
    if (n <= (long long)T->lt_max) {
        const F2 y = df_mul_f(df_add(df_log2_count<kTable>((unsigned)n, T), F2{-LN.hi, -LN.lo}), q);
        return exp2f(y.hi) * __fmaf_rn(y.lo, 0.693147182f, 1.0f) * kTermScale;
    }
    return powf((float)n / fN, q) * kTermScale;
}

}  // namespace tsl
