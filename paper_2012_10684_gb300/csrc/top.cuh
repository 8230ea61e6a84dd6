// Double-float objective helpers shared by the searches that evaluate the
// objective in double-float (the per-slice table search of search1d.cuh and
// the cluster kernel): division, comparison, a running maximum that also
// tracks how close the other candidates come, and error bounds.
#pragma once
#include "common.cuh"
#include "dfmath.cuh"

namespace tsl {

__device__ __forceinline__ F2 f2_neg(F2 x) { return {-x.hi, -x.lo}; }

// x / y for double-float values (y != 0): one correction step on the
// float quotient.
__device__ __forceinline__ F2 df_div(F2 x, F2 y) {
    const float q1 = __fdiv_rn(x.hi, y.hi);
    const F2 r = df_add(x, f2_neg(df_mul_f(y, q1)));
    const float q2 = __fdiv_rn(r.hi, y.hi);
    return fast_two_sum(q1, q2);
}

// x / y as df_div, with the fast float quotient (__fdividef, within 2 ulp)
// in both steps: the correction step still recovers the double-float
// quotient, whose relative error grows from about 2^-47 to a few 2^-45, far
// inside the bounds below. For normal |y| < 2^126 (the searches' class
// powers 2^64 (n/N)^q and counts).
__device__ __forceinline__ F2 df_div_fast(F2 x, F2 y) {
    const float q1 = __fdividef(x.hi, y.hi);
    const F2 r = df_add(x, f2_neg(df_mul_f(y, q1)));
    const float q2 = __fdividef(r.hi, y.hi);
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ bool df_gt(F2 a, F2 b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

// Running top of (value, level) pairs: the largest value (smallest level on
// equal values), its error bound, and the largest value + bound among all
// other pairs seen (u2), which decides whether anything else can still beat
// the top. A pair whose value equals the top's exactly (a threshold on a
// plateau of empty levels gives the very same sums, hence the same value)
// does not raise u2: the smallest index already settles that tie.
struct Top {
    F2 v;
    int i;       // level, -1: none
    float band;
    float u2;    // max (value + bound) over the other pairs; -inf: none
};

__device__ __forceinline__ Top top_merge(Top a, Top b) {
    if (b.i < 0) return a;
    if (a.i < 0) return b;
    const bool a_wins = df_gt(a.v, b.v) || (!df_gt(b.v, a.v) && a.i < b.i);
    Top w = a_wins ? a : b;
    const Top l = a_wins ? b : a;
    const bool same = l.v.hi == w.v.hi && l.v.lo == w.v.lo;
    w.u2 = fmaxf(fmaxf(w.u2, l.u2), same ? -INFINITY : l.v.hi + l.band);
    return w;
}

__device__ __forceinline__ Top shfl_top(Top t, int d) {
    Top o;
    o.v.hi = __shfl_xor_sync(0xffffffffu, t.v.hi, d);
    o.v.lo = __shfl_xor_sync(0xffffffffu, t.v.lo, d);
    o.i = __shfl_xor_sync(0xffffffffu, t.i, d);
    o.band = __shfl_xor_sync(0xffffffffu, t.band, d);
    o.u2 = __shfl_xor_sync(0xffffffffu, t.u2, d);
    return o;
}

// Bounds on the error of the double-float objective. Terms (h/N)^q and the
// class powers are within 1e-12 relative (dfmath.cuh); a double-float sum
// of at most 4096 positive terms adds at most 4096 * 2^-47 < 3e-11
// relative; the quotients and products add a few 2^-47 (a few 2^-45 with
// df_div_fast). So a b' is within about 7e-11 relative, and the bounds below
// (1e-10) cover it.
__device__ __forceinline__ float tsallis_band_df(float ab, float phi, float q) {
    return 1e-10f * fabsf(ab) / fabsf(q - 1.0f) + 1e-12f * fabsf(phi) + 1e-30f;
}
__device__ __forceinline__ float shannon_band_df(float la, float sa, float lb, float sb) {
    return 1e-10f * (fabsf(la) + fabsf(sa) + fabsf(lb) + fabsf(sb) + 1.0f);
}

}  // namespace tsl
