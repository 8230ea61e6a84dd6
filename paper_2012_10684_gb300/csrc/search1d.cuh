// 1-D exhaustive threshold search, one thread block per histogram.
//
// Section II-C ("Tsallis entropy"), 1-D reading. Steps, all inside the block:
//   1. each thread owns 8 consecutive levels; h^q (or h ln h at q = 1) in
//      FP32, exact int64 counts;
//   2. block-wide exclusive prefix scan of counts and of the compensated
//      (hi, lo) sums of h^q, and a separate suffix scan for class 2 (class-2
//      sums are never formed as total minus class-1 sums);
//   3. phi(t) for every valid t with its error bound, block argmax with the
//      smallest t among equal values;
//   4. if any threshold giving a different partition lies within the error
//      bands of the maximum, recompute phi for all of those candidates in
//      FP64 (FP64 h^q, FP64 scans) and take their argmax;
//   5. canonical t: the smallest t giving the same class-1 count (empty
//      levels between classes do not change the partition).
#pragma once
#include "common.cuh"
#include "../../include/tsallis.h"

namespace tsl {

__device__ __forceinline__ float term_f32(int h, float q, bool shannon) {
    if (h <= 0) return 0.f;
    float x = (float)h;
    return shannon ? x * logf(x) : powf(x, q);
}
__device__ __forceinline__ double term_f64(int h, double q, bool shannon) {
    if (h <= 0) return 0.0;
    double x = (double)h;
    return shannon ? x * log(x) : pow(x, q);
}

// Block argmax over (value, index) pairs held one per thread; result in
// sm.red_v[0] / sm.red_i[0] after the call (all threads synchronised).
__device__ __forceinline__ void block_argmax_f(float v, int i, SearchSmem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_argmax(v, i);
    if (lane == 0) { sm.red_v[warp] = v; sm.red_i[warp] = i; }
    __syncthreads();
    if (warp == 0) {
        v = lane < kSearchWarps ? sm.red_v[lane] : 0.f;
        i = lane < kSearchWarps ? sm.red_i[lane] : -1;
        warp_argmax(v, i);
        if (lane == 0) { sm.red_v[0] = v; sm.red_i[0] = i; }
    }
    __syncthreads();
}
__device__ __forceinline__ void block_argmax_d(double v, int i, SearchSmem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_argmax(v, i);
    if (lane == 0) { sm.red_dv[warp] = v; sm.red_i[warp] = i; }
    __syncthreads();
    if (warp == 0) {
        v = lane < kSearchWarps ? sm.red_dv[lane] : 0.0;
        i = lane < kSearchWarps ? sm.red_i[lane] : -1;
        warp_argmax(v, i);
        if (lane == 0) { sm.red_dv[0] = v; sm.red_i[0] = i; }
    }
    __syncthreads();
}
__device__ __forceinline__ int block_min_i(int v, SearchSmem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = __reduce_min_sync(0xffffffffu, v);
    if (lane == 0) sm.red_i[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < kSearchWarps ? sm.red_i[lane] : 0x7fffffff;
        v = __reduce_min_sync(0xffffffffu, v);
        if (lane == 0) sm.canon_t = v;
    }
    __syncthreads();
    return sm.canon_t;
}

__device__ SearchResult search1d_block(const int32_t* __restrict__ h, int L, float q, float* __restrict__ curve,
                                       SearchSmem& sm) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool shannon = (q == 1.0f);
    const int base = tid * kBinsPerThread;

    // ---- 1. counts and FP32 terms of this thread's levels
    int hv[kBinsPerThread];
    float a0[kBinsPerThread];  // term h^q; later the error band
    float a1[kBinsPerThread];  // class-1 sum Q_1(t); later phi(t)
    long long c = 0;
    F2 w{0.f, 0.f};
#pragma unroll
    for (int k = 0; k < kBinsPerThread; ++k) {
        int i = base + k;
        hv[k] = i < L ? __ldcg(h + i) : 0;
        a0[k] = term_f32(hv[k], q, shannon);
        c += hv[k];
        w = f2_add_f(w, a0[k]);
    }

    // ---- 2. block scans of thread totals
    long long c_inc = warp_prefix_i64(c, lane);
    F2 w_inc = warp_prefix_f2(w, lane);
    F2 w_sinc = warp_suffix_f2(w, lane);
    if (lane == 31) { sm.cnt_pre[warp] = c_inc; sm.w_pre[warp] = w_inc; }
    if (lane == 0) sm.w_suf[warp] = w_sinc;
    __syncthreads();
    if (warp == 0) {
        long long cw = lane < kSearchWarps ? sm.cnt_pre[lane] : 0;
        F2 ww = lane < kSearchWarps ? sm.w_pre[lane] : F2{0.f, 0.f};
        F2 ws = lane < kSearchWarps ? sm.w_suf[lane] : F2{0.f, 0.f};
        long long ci = warp_prefix_i64(cw, lane);
        F2 wi = warp_prefix_f2(ww, lane);
        F2 si = warp_suffix_f2(ws, lane);
        long long ce = __shfl_up_sync(0xffffffffu, ci, 1);
        F2 we = shfl_up_f2(wi, 1);
        F2 se = shfl_down_f2(si, 1);
        if (lane == 0) { ce = 0; we = F2{0.f, 0.f}; }
        if (lane == 31) se = F2{0.f, 0.f};
        if (lane == kSearchWarps - 1) sm.total = ci;
        __syncwarp();
        if (lane < kSearchWarps) { sm.cnt_pre[lane] = ce; sm.w_pre[lane] = we; sm.w_suf[lane] = se; }
    }
    __syncthreads();
    const long long N = sm.total;
    long long c_before = __shfl_up_sync(0xffffffffu, c_inc, 1);
    F2 w_before = shfl_up_f2(w_inc, 1);
    F2 w_after = shfl_down_f2(w_sinc, 1);
    if (lane == 0) { c_before = 0; w_before = F2{0.f, 0.f}; }
    if (lane == 31) w_after = F2{0.f, 0.f};
    c_before += sm.cnt_pre[warp];
    w_before = f2_add(sm.w_pre[warp], w_before);
    w_after = f2_add(w_after, sm.w_suf[warp]);

    // class-1 sums, forward
    {
        F2 s = w_before;
#pragma unroll
        for (int k = 0; k < kBinsPerThread; ++k) {
            s = f2_add_f(s, a0[k]);
            a1[k] = f2_val(s);
        }
    }
    // ---- 3. objective and error bound per threshold; class-2 sums backward
    float best_v = 0.f;
    int best_i = -1;
    {
        F2 sB = w_after;
        long long na = c_before + c;  // class-1 count through the last level of the thread
#pragma unroll
        for (int k = kBinsPerThread - 1; k >= 0; --k) {
            const int t = base + k;
            const long long nb = N - na;
            const bool valid = (t <= L - 2) && na > 0 && nb > 0;
            float f = 0.f, e = -1.f;  // e < 0 marks an invalid threshold
            if (valid) {
                const float qa = a1[k], qb = f2_val(sB);
                const float fa = (float)na, fb = (float)nb;
                if (shannon) {
                    float lna = logf(fa), lnb = logf(fb);
                    float sa = qa / fa, sb = qb / fb;
                    f = (lna - sa) + (lnb - sb);
                    e = shannon_err(lna, sa, lnb, sb, f);
                } else {
                    float ab = (qa / powf(fa, q)) * (qb / powf(fb, q));
                    f = (1.0f - ab) / (q - 1.0f);
                    e = tsallis_err(ab, f, q);
                }
                argmax_merge(best_v, best_i, f, t);
            }
            if (curve != nullptr && t <= L - 2) curve[t] = valid ? f : __int_as_float(0x7fc00000);
            sB = f2_add_f(sB, a0[k]);
            a0[k] = e;
            a1[k] = f;
            na -= hv[k];
        }
    }
    block_argmax_f(best_v, best_i, sm);
    const int t32 = sm.red_i[0];
    const float phi32 = sm.red_v[0];
    __syncthreads();
    if (t32 < 0) return SearchResult{-1, 0.f, TSALLIS_ERR_NO_VALID_THRESHOLD};

    // owner of t32 publishes its class-1 count and error band
    if (t32 >= base && t32 < base + kBinsPerThread) {
        long long na = c_before;
#pragma unroll
        for (int k = 0; k < kBinsPerThread; ++k) {
            na += hv[k];
            if (base + k == t32) { sm.best_na = na; sm.best_err = a0[k]; }
        }
    }
    __syncthreads();
    const long long na_best = sm.best_na;
    const float lower = phi32 - sm.best_err;

    // ---- 4. near-tie detection: another partition within the error bands
    bool tie = false;
    {
        long long na = c_before;
#pragma unroll
        for (int k = 0; k < kBinsPerThread; ++k) {
            na += hv[k];
            if (a0[k] >= 0.f && na != na_best && a1[k] + a0[k] >= lower) tie = true;
        }
    }
    const bool rerank = __syncthreads_or(tie) != 0;

    int status = TSALLIS_OK;
    float phi_out = phi32;
    long long na_win = na_best;
    if (rerank) {
        status |= TSALLIS_STATUS_RERANKED;
        const double qd = (double)q;
        double dT[kBinsPerThread];
        double dsum = 0.0;
#pragma unroll
        for (int k = 0; k < kBinsPerThread; ++k) {
            dT[k] = term_f64(hv[k], qd, shannon);
            dsum += dT[k];
        }
        double d_inc = warp_prefix_f64(dsum, lane);
        double d_sinc = warp_suffix_f64(dsum, lane);
        if (lane == 31) sm.d_pre[warp] = d_inc;
        if (lane == 0) sm.d_suf[warp] = d_sinc;
        __syncthreads();
        if (warp == 0) {
            double a = lane < kSearchWarps ? sm.d_pre[lane] : 0.0;
            double b = lane < kSearchWarps ? sm.d_suf[lane] : 0.0;
            double ai = warp_prefix_f64(a, lane);
            double bi = warp_suffix_f64(b, lane);
            double ae = __shfl_up_sync(0xffffffffu, ai, 1);
            double be = __shfl_down_sync(0xffffffffu, bi, 1);
            if (lane == 0) ae = 0.0;
            if (lane == 31) be = 0.0;
            __syncwarp();
            if (lane < kSearchWarps) { sm.d_pre[lane] = ae; sm.d_suf[lane] = be; }
        }
        __syncthreads();
        double d_before = __shfl_up_sync(0xffffffffu, d_inc, 1);
        double d_after = __shfl_down_sync(0xffffffffu, d_sinc, 1);
        if (lane == 0) d_before = 0.0;
        if (lane == 31) d_after = 0.0;
        d_before += sm.d_pre[warp];
        d_after += sm.d_suf[warp];
        // class-1 sums forward, then candidates backward with class-2 sums
        double dA[kBinsPerThread];
        {
            double s = d_before;
#pragma unroll
            for (int k = 0; k < kBinsPerThread; ++k) {
                s += dT[k];
                dA[k] = s;
            }
        }
        double bv = 0.0;
        int bi = -1;
        {
            double sB = d_after;
            long long na = c_before + c;
#pragma unroll
            for (int k = kBinsPerThread - 1; k >= 0; --k) {
                const long long nb = N - na;
                if (a0[k] >= 0.f && a1[k] + a0[k] >= lower) {
                    const double QA = dA[k], QB = sB;
                    double f;
                    if (shannon) {
                        f = (log((double)na) - QA / (double)na) + (log((double)nb) - QB / (double)nb);
                    } else {
                        double ab = (QA / pow((double)na, qd)) * (QB / pow((double)nb, qd));
                        f = (1.0 - ab) / (qd - 1.0);
                    }
                    argmax_merge(bv, bi, f, base + k);
                }
                sB += dT[k];  // level k joins class 2 for threshold k-1
                na -= hv[k];
            }
        }
        block_argmax_d(bv, bi, sm);
        const int tw = sm.red_i[0];
        phi_out = (float)sm.red_dv[0];
        __syncthreads();
        if (tw >= base && tw < base + kBinsPerThread) {
            long long na = c_before;
#pragma unroll
            for (int k = 0; k < kBinsPerThread; ++k) {
                na += hv[k];
                if (base + k == tw) sm.best_na = na;
            }
        }
        __syncthreads();
        na_win = sm.best_na;
    }

    // ---- 5. canonical threshold: smallest t with the winning class-1 count
    int tmin = 0x7fffffff;
    {
        long long na = c_before;
#pragma unroll
        for (int k = 0; k < kBinsPerThread; ++k) {
            na += hv[k];
            if (a0[k] >= 0.f && na == na_win && base + k < tmin) tmin = base + k;
        }
    }
    const int t_final = block_min_i(tmin, sm);
    return SearchResult{t_final, phi_out, status};
}

}  // namespace tsl
