// 1-D exhaustive threshold search, one thread block per histogram.
//
// Section II-C ("Tsallis entropy"), 1-D reading. With N the total count,
// every term is scaled by N^-q (and by the constant 2^64 of dfmath.cuh,
// which cancels in every ratio):
//     w_i = (h_i / N)^q,  Q_1(t) = sum_{i<=t} w_i,  Q_2(t) = sum_{i>t} w_i,
//     a = Q_1 / (N_1/N)^q,  b = Q_2 / (N_2/N)^q,  phi = (1 - a b) / (q - 1),
// which is H_1 + H_2 + (1 - q) H_1 H_2 with H_k = (1 - sum (p_i/P_k)^q)/(q-1).
// At q = 1 (Shannon limit) w_i = h_i log2 h_i and
//     phi = ln 2 * [(log2 N_1 - Q_1/N_1) + (log2 N_2 - Q_2/N_2)].
//
// Steps, all inside the block (512 threads):
//   1. compaction of the non-empty levels (see search1d_block), exact int64
//      prefix sums of their counts (gives N and N_1);
//   2. terms w_i as double-float pairs (dfmath.cuh), kept in shared memory;
//      double-float prefix and suffix scans (class-2 sums are summed from
//      the right, never formed as total minus class-1 sums);
//   3. phi(t) in FP32 from the rounded sums, with a rigorous error bound,
//      and the block argmax (smallest t among equal values);
//   4. every threshold with a different partition whose FP32 value lies
//      within the error bands of the maximum is a candidate; if there is
//      one, all candidates are re-evaluated in FP64 from the double-float
//      sums (class powers (N_k/N)^q also in double-float), and the FP64
//      argmax wins;
//   5. canonical t: the smallest t with the winning partition, which is the
//      non-empty level the winning entry stands for.
#pragma once
#include "common.cuh"
#include "dfmath.cuh"
#include "top.cuh"
#include "../../include/tsallis.h"

namespace tsl {

// The 512 threads that run a search synchronise through a barrier policy:
// the whole block (standalone search kernel) or a named barrier shared only
// by the search warps of the fused kernel.
struct BlockSync {
    __device__ static void sync() { __syncthreads(); }
    __device__ static int tid() { return threadIdx.x; }
};
template <int kBarrier, int kFirstThread>
struct NamedSync {
    __device__ static void sync() { asm volatile("bar.sync %0, %1;" ::"n"(kBarrier), "n"(kSearchThreads) : "memory"); }
    __device__ static int tid() { return (int)threadIdx.x - kFirstThread; }
};

// Block-wide OR of a predicate through shared memory.
template <class Sync>
__device__ __forceinline__ bool block_any(bool p, SearchSmem& sm) {
    if (Sync::tid() == 0) sm.flag = 0;
    Sync::sync();
    if (p) sm.flag = 1;
    Sync::sync();
    const bool r = sm.flag != 0;
    Sync::sync();
    return r;
}

// The block's top from the per-warp tops in shared memory (after the barrier
// that published them), in every warp at once: lane l reads warp l mod 16's
// top and four xor-shuffle rounds merge them. top_merge only compares and
// takes maxima, so the result is the serial merge's, bit for bit; a
// duplicated entry merges with itself unchanged.
__device__ __forceinline__ Top block_top_of(const SearchSmem& sm) {
    const int w = threadIdx.x & (kSearchWarps - 1);
    Top g{{sm.top_vh[w], sm.top_vl[w]}, sm.top_i[w], sm.top_band[w], sm.top_u2[w]};
#pragma unroll
    for (int d = kSearchWarps / 2; d > 0; d >>= 1) g = top_merge(g, shfl_top(g, d));
    return g;
}

// Block argmax over (value, index) pairs held one per thread; result in
// sm.red_v[0] / sm.red_i[0] after the call (all threads synchronised).
template <class Sync>
__device__ __forceinline__ void block_argmax_f(float v, int i, SearchSmem& sm) {
    const int lane = Sync::tid() & 31, warp = Sync::tid() >> 5;
    warp_argmax(v, i);
    if (lane == 0) { sm.red_v[warp] = v; sm.red_i[warp] = i; }
    Sync::sync();
    if (warp == 0) {
        v = lane < kSearchWarps ? sm.red_v[lane] : 0.f;
        i = lane < kSearchWarps ? sm.red_i[lane] : -1;
        warp_argmax(v, i);
        if (lane == 0) { sm.red_v[0] = v; sm.red_i[0] = i; }
    }
    Sync::sync();
}
template <class Sync>
__device__ __forceinline__ void block_argmax_d(double v, int i, SearchSmem& sm) {
    const int lane = Sync::tid() & 31, warp = Sync::tid() >> 5;
    warp_argmax(v, i);
    if (lane == 0) { sm.red_dv[warp] = v; sm.red_i[warp] = i; }
    Sync::sync();
    if (warp == 0) {
        v = lane < kSearchWarps ? sm.red_dv[lane] : 0.0;
        i = lane < kSearchWarps ? sm.red_i[lane] : -1;
        warp_argmax(v, i);
        if (lane == 0) { sm.red_dv[0] = v; sm.red_i[0] = i; }
    }
    Sync::sync();
}
// Scratch (shared memory): sT[kMaxBins] float2 and sIC[kMaxBins] int2.
//
// Only non-empty levels matter: every threshold t in a run of empty levels
// between non-empty levels i_k and i_{k+1} gives the same partition as
// t = i_k, which is the smallest such t. So the levels are compacted to the
// list of non-empty ones (i_0 < i_1 < ... < i_{M-1}), the objective is
// evaluated once per entry k < M - 1 (threshold t = i_k), and the argmax over
// entries is already the canonical threshold.
template <class Sync>
__device__ SearchResult search1d_block(const int32_t* __restrict__ h, int L, float q, float* __restrict__ curve,
                                       SearchSmem& sm, float2* __restrict__ sT, int2* __restrict__ sIC,
                                       const DfTables* __restrict__ T) {
    const int tid = Sync::tid(), lane = tid & 31, warp = tid >> 5;
    const bool shannon = (q == 1.0f);

    // ---- 1. compaction of the non-empty levels, and the total count N
    {
        const int base = tid * kBinsPerThread;
        int hv[kBinsPerThread];
        int nz = 0;
        long long c = 0;
#pragma unroll
        for (int k = 0; k < kBinsPerThread; ++k) {
            const int i = base + k;
            hv[k] = i < L ? __ldcg(h + i) : 0;
            nz += hv[k] > 0;
            c += hv[k];
        }
        int nz_inc = nz;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, nz_inc, d);
            if (lane >= d) nz_inc += o;
        }
        long long csum = c;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) csum += __shfl_xor_sync(0xffffffffu, csum, d);
        if (lane == 31) sm.red_i[warp] = nz_inc;
        if (lane == 0) sm.cnt_pre[warp] = csum;
        Sync::sync();
        if (warp == 0) {
            const int v = lane < kSearchWarps ? sm.red_i[lane] : 0;
            int vi = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int o = __shfl_up_sync(0xffffffffu, vi, d);
                if (lane >= d) vi += o;
            }
            long long cs = lane < kSearchWarps ? sm.cnt_pre[lane] : 0;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, d);
            __syncwarp();
            if (lane < kSearchWarps) sm.red_i[lane] = vi - v;   // exclusive warp offsets
            if (lane == kSearchWarps - 1) sm.nlevels = vi;       // M
            if (lane == 0) sm.total = cs;
        }
        Sync::sync();
        int pos = sm.red_i[warp] + nz_inc - nz;
#pragma unroll
        for (int k = 0; k < kBinsPerThread; ++k)
            if (hv[k] > 0) sIC[pos++] = make_int2(base + k, hv[k]);
    }
    Sync::sync();
    const int M = sm.nlevels;
    const long long N = sm.total;
    if (curve != nullptr) {
        // empty class 1 below the first non-empty level
        const int first = M > 0 ? sIC[0].x : L;
        for (int t = tid; t < first && t < L - 1; t += kSearchThreads) curve[t] = __int_as_float(0x7fc00000);
    }
    if (M < 2) {
        if (curve != nullptr)
            for (int t = tid; t < L - 1; t += kSearchThreads) curve[t] = __int_as_float(0x7fc00000);
        Sync::sync();
        return SearchResult{-1, 0.f, TSALLIS_ERR_NO_VALID_THRESHOLD};
    }

    // ---- 2. each thread takes a contiguous run of at most 8 entries
    const int per = (M + kSearchThreads - 1) / kSearchThreads;
    const int j0 = min(tid * per, M), j1 = min(j0 + per, M);
    const F2 LN = shannon ? F2{0.f, 0.f} : df_log2_count<false>((unsigned)N, T);
    long long c = 0;
    F2 w{0.f, 0.f};
    for (int j = j0; j < j1; ++j) {
        const int cnt = sIC[j].y;
        const F2 tk = shannon ? df_hlog2h<false>((unsigned)cnt, T) : df_pow_ratio<false>((unsigned)cnt, LN, q, T);
        sT[j] = make_float2(tk.hi, tk.lo);
        c += cnt;
        w = f2_add(w, tk);
    }
    // block scans: counts (prefix), term sums (prefix and, separately, suffix)
    const long long c_inc = warp_prefix_i64(c, lane);
    const F2 w_inc = warp_prefix_f2(w, lane);
    const F2 w_sinc = warp_suffix_f2(w, lane);
    if (lane == 31) { sm.cnt_pre[warp] = c_inc; sm.w_pre[warp] = w_inc; }
    if (lane == 0) sm.w_suf[warp] = w_sinc;
    Sync::sync();
    if (warp == 0) {
        const long long cw = lane < kSearchWarps ? sm.cnt_pre[lane] : 0;
        const F2 ww = lane < kSearchWarps ? sm.w_pre[lane] : F2{0.f, 0.f};
        const F2 ws = lane < kSearchWarps ? sm.w_suf[lane] : F2{0.f, 0.f};
        const long long ci = warp_prefix_i64(cw, lane);
        const F2 wi = warp_prefix_f2(ww, lane);
        const F2 si = warp_suffix_f2(ws, lane);
        long long ce = __shfl_up_sync(0xffffffffu, ci, 1);
        F2 we = shfl_up_f2(wi, 1);
        F2 se = shfl_down_f2(si, 1);
        if (lane == 0) { ce = 0; we = F2{0.f, 0.f}; }
        if (lane == 31) se = F2{0.f, 0.f};
        __syncwarp();
        if (lane < kSearchWarps) { sm.cnt_pre[lane] = ce; sm.w_pre[lane] = we; sm.w_suf[lane] = se; }
    }
    Sync::sync();
    long long c_before = __shfl_up_sync(0xffffffffu, c_inc, 1);
    F2 w_before = shfl_up_f2(w_inc, 1);
    F2 w_after = shfl_down_f2(w_sinc, 1);
    if (lane == 0) { c_before = 0; w_before = F2{0.f, 0.f}; }
    if (lane == 31) w_after = F2{0.f, 0.f};
    c_before += sm.cnt_pre[warp];
    w_before = f2_add(sm.w_pre[warp], w_before);
    w_after = f2_add(w_after, sm.w_suf[warp]);

    // ---- 3. FP32 objective per entry (threshold at its level) and error band
    float qa_f[kBinsPerThread], phi[kBinsPerThread], err[kBinsPerThread];  // err < 0: invalid
    {
        F2 sA = w_before;
#pragma unroll
        for (int k = 0; k < kBinsPerThread; ++k) {
            if (j0 + k < j1) {
                const float2 tk = sT[j0 + k];
                sA = f2_add(sA, F2{tk.x, tk.y});
            }
            qa_f[k] = f2_val(sA);
        }
    }
    float best_v = 0.f;
    int best_i = -1;
    {
        const float fN = (float)N;
        F2 sB = w_after;
        long long na = c_before + c;
#pragma unroll 1
        for (int k = kBinsPerThread - 1; k >= 0; --k) {
            const int j = j0 + k;
            float f = 0.f, e = -1.f;
            if (j < j1) {
                const long long nb = N - na;
                if (j < M - 1) {   // class 2 is non-empty
                    const float qa = qa_f[k], qb = f2_val(sB);
                    const float fa = (float)na, fb = (float)nb;
                    if (shannon) {
                        const float ua = log2f(fa), ub = log2f(fb);
                        const float va = qa / fa, vb = qb / fb;
                        const float fb2 = (ua - va) + (ub - vb);
                        f = 0.693147182f * fb2;
                        e = shannon_err(ua, va, ub, vb, fb2);
                    } else {
                        // class powers scaled like the terms (2^64)
                        const float ab = (qa / class_pow_f32<false>(na, fN, LN, q, T)) * (qb / class_pow_f32<false>(nb, fN, LN, q, T));
                        f = (1.0f - ab) / (q - 1.0f);
                        e = tsallis_err(ab, f, q);
                    }
                    argmax_merge(best_v, best_i, f, j);
                }
                const float2 tk = sT[j];
                sB = f2_add(sB, F2{tk.x, tk.y});
                na -= sIC[j].y;
            }
            phi[k] = f;
            err[k] = e;
        }
    }
    if (curve != nullptr) {
        for (int k = 0; k < kBinsPerThread; ++k) {
            const int j = j0 + k;
            if (j >= j1) break;
            const int tb = sIC[j].x, te = (j + 1 < M) ? sIC[j + 1].x : L - 1;
            const float v = err[k] >= 0.f ? phi[k] : __int_as_float(0x7fc00000);
            for (int t = tb; t < te && t < L - 1; ++t) curve[t] = v;
        }
    }
    block_argmax_f<Sync>(best_v, best_i, sm);
    const int j32 = sm.red_i[0];
    const float phi32 = sm.red_v[0];
    Sync::sync();
    if (j32 >= j0 && j32 < j1) {
#pragma unroll
        for (int k = 0; k < kBinsPerThread; ++k)
            if (j0 + k == j32) sm.best_err = err[k];
    }
    Sync::sync();
    const float lower = phi32 - sm.best_err;

    // ---- 4. candidates: other entries (other partitions) inside the error bands
    bool tie = false;
#pragma unroll
    for (int k = 0; k < kBinsPerThread; ++k)
        if (err[k] >= 0.f && j0 + k != j32 && phi[k] + err[k] >= lower) tie = true;
    const bool rerank = block_any<Sync>(tie, sm);

    int status = TSALLIS_OK;
    float phi_out = phi32;
    int jwin = j32;
    if (rerank) {
        status |= TSALLIS_STATUS_RERANKED;
        double bv = 0.0;
        int bi = -1;
        F2 sA = w_before;
        long long na = c_before;
        for (int k = 0; k < kBinsPerThread; ++k) {
            const int j = j0 + k;
            if (j >= j1) break;
            const float2 tk = sT[j];
            sA = f2_add(sA, F2{tk.x, tk.y});
            na += sIC[j].y;
            if (!(err[k] >= 0.f && phi[k] + err[k] >= lower)) continue;
            F2 sB = w_after;
            for (int i = j1 - 1; i > j; --i) {
                const float2 ti = sT[i];
                sB = f2_add(sB, F2{ti.x, ti.y});
            }
            const long long nb = N - na;
            double f;
            if (shannon) {
                const double la = df_to_double(df_log2_count<false>((unsigned)na, T));
                const double lb = df_to_double(df_log2_count<false>((unsigned)nb, T));
                f = 0.6931471805599453 * ((la - df_to_double(sA) / (double)na) + (lb - df_to_double(sB) / (double)nb));
            } else {
                const double pa = df_to_double(df_pow_ratio<false>((unsigned)na, LN, q, T));
                const double pb = df_to_double(df_pow_ratio<false>((unsigned)nb, LN, q, T));
                const double ab = (df_to_double(sA) / pa) * (df_to_double(sB) / pb);
                f = (1.0 - ab) / ((double)q - 1.0);
            }
            argmax_merge(bv, bi, f, j);
        }
        block_argmax_d<Sync>(bv, bi, sm);
        jwin = sm.red_i[0];
        phi_out = (float)sm.red_dv[0];
        Sync::sync();
    }
    const int t_final = sIC[jwin].x;
    Sync::sync();   // sIC / sT may be reused by the caller after this
    return SearchResult{t_final, phi_out, status};
}

// ------------------------------------------------------------ table search
//
// The exhaustive search for a histogram whose total count N is fixed in
// advance (one slice of known size): the double-float terms 2^64 (n / N)^q
// for every count n = 0..N are read from a table (Tp, built once per N and
// q; at q = 1 the table holds n log2 n). The non-empty levels are compacted
// first (an empty level gives the same partition as the non-empty level
// below it, whose value is the smaller t), so each thread evaluates a short
// run of entries, and a thread's table reads are issued together: the terms
// Tp[h_i] for the class sums, then the class powers Tp[N_1] and Tp[N_2].
// Class-1 and (separately, from the right) class-2 sums in double-float, the
// objective in double-float with an error bound at every non-empty level
// with a non-empty class 2, the smallest level on equal values, and FP64 for
// the levels whose bound reaches the maximum's. Four barriers (six with a
// re-rank), against the dozen of search1d_block, and no transcendental
// functions but log2 at q = 1. Scratch (shared memory): sIC[kMaxBins]
// (level, count) and sW[kMaxBins] (terms).
template <class Sync>
__device__ SearchResult search1d_fast(const int32_t* __restrict__ h, int L, float q, const float2* __restrict__ Tp,
                                      long long N, SearchSmem& sm, int2* __restrict__ sIC, float2* __restrict__ sW,
                                      const DfTables* __restrict__ T) {
    const int tid = Sync::tid(), lane = tid & 31, warp = tid >> 5;
    const bool shannon = (q == 1.0f);
    // ---- 1. compaction of the non-empty levels
    const int base = tid * kBinsPerThread;
    int hv[kBinsPerThread];
    if (base + kBinsPerThread <= L && ((L & 3) == 0)) {
        const int4 a0 = __ldcg(reinterpret_cast<const int4*>(h + base));
        const int4 a1 = __ldcg(reinterpret_cast<const int4*>(h + base) + 1);
        hv[0] = a0.x; hv[1] = a0.y; hv[2] = a0.z; hv[3] = a0.w; hv[4] = a1.x; hv[5] = a1.y; hv[6] = a1.z; hv[7] = a1.w;
    } else {
#pragma unroll
        for (int k = 0; k < kBinsPerThread; ++k) hv[k] = base + k < L ? __ldcg(h + base + k) : 0;
    }
    int nz = 0;
#pragma unroll
    for (int k = 0; k < kBinsPerThread; ++k) nz += hv[k] > 0;
    int nz_inc = nz;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, nz_inc, d);
        if (lane >= d) nz_inc += o;
    }
    if (lane == 31) sm.red_i[warp] = nz_inc;
    Sync::sync();   // 1
    int M = 0, pos = nz_inc - nz;
#pragma unroll
    for (int w = 0; w < kSearchWarps; ++w) {
        const int v = sm.red_i[w];
        if (w < warp) pos += v;
        M += v;
    }
#pragma unroll
    for (int k = 0; k < kBinsPerThread; ++k)
        if (hv[k] > 0) sIC[pos++] = make_int2(base + k, hv[k]);
    Sync::sync();   // 2
    if (M < 2) return SearchResult{-1, 0.f, TSALLIS_ERR_NO_VALID_THRESHOLD};

    // ---- 2. this thread's entries (a contiguous run of at most 8), four at
    // a time: terms gathered together and kept in sW, run sums
    const int per = (M + kSearchThreads - 1) / kSearchThreads;
    const int j0 = min(tid * per, M), j1 = min(j0 + per, M);
    long long c = 0;
    F2 run{0.f, 0.f};
    for (int g = j0; g < j1; g += 4) {
        int cn[4];
        float2 tw[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) cn[u] = g + u < j1 ? sIC[g + u].y : 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) tw[u] = cn[u] > 0 ? __ldg(Tp + cn[u]) : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (g + u < j1) sW[g + u] = tw[u];
            c += cn[u];
            run = f2_add(run, F2{tw[u].x, tw[u].y});
        }
    }
    // exclusive count and term prefix, exclusive term suffix
    long long ci = c;
    F2 pi = run, si = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long oc = __shfl_up_sync(0xffffffffu, ci, d);
        const F2 op = shfl_up_f2(pi, d);
        const F2 os = shfl_down_f2(si, d);
        if (lane >= d) { ci += oc; pi = f2_add(op, pi); }
        if (lane + d < 32) si = f2_add(si, os);
    }
    if (lane == 31) { sm.cnt_pre[warp] = ci; sm.w_pre[warp] = pi; }
    if (lane == 0) sm.w_suf[warp] = si;
    Sync::sync();   // 3
    long long c_before = __shfl_up_sync(0xffffffffu, ci, 1);
    F2 w_before = shfl_up_f2(pi, 1);
    F2 w_after = shfl_down_f2(si, 1);
    if (lane == 0) { c_before = 0; w_before = F2{0.f, 0.f}; }
    if (lane == 31) w_after = F2{0.f, 0.f};
    {
        // the 16 warps' totals scanned in four shuffle rounds (lane l holds
        // warp l mod 16's), then this warp's exclusive prefix and suffix
        const int wl = lane & (kSearchWarps - 1);
        long long cw = sm.cnt_pre[wl];
        F2 pw = sm.w_pre[wl], sw = sm.w_suf[wl];
#pragma unroll
        for (int d = 1; d < kSearchWarps; d <<= 1) {
            const long long oc = __shfl_up_sync(0xffffffffu, cw, d);
            const F2 op = shfl_up_f2(pw, d);
            const F2 os = shfl_down_f2(sw, d);
            if (wl >= d) { cw += oc; pw = f2_add(op, pw); }
            if (wl + d < kSearchWarps) sw = f2_add(sw, os);
        }
        const int lp = (warp + kSearchWarps - 1) & (kSearchWarps - 1), ls = (warp + 1) & (kSearchWarps - 1);
        const long long cx = __shfl_sync(0xffffffffu, cw, lp);
        const F2 px{__shfl_sync(0xffffffffu, pw.hi, lp), __shfl_sync(0xffffffffu, pw.lo, lp)};
        const F2 sx{__shfl_sync(0xffffffffu, sw.hi, ls), __shfl_sync(0xffffffffu, sw.lo, ls)};
        if (warp > 0) {
            c_before += cx;
            w_before = f2_add(px, w_before);
        }
        if (warp < kSearchWarps - 1) w_after = f2_add(w_after, sx);
    }
    // class-2 sums from the right: sW[j] becomes Q_2 at entry j
    {
        F2 rs = w_after;
        for (int j = j1 - 1; j >= j0; --j) {
            const float2 w = sW[j];
            sW[j] = make_float2(rs.hi, rs.lo);
            rs = f2_add(F2{w.x, w.y}, rs);
        }
    }

    // ---- 3. the objective at each entry, left to right (class-1 sums from
    // the left), terms and class powers gathered two entries at a time;
    // mode 1 takes the entries whose bound reaches `lower` in FP64 (re-rank)
    const F2 qm1 = two_sum(q, -1.0f);
    // 1 / (q - 1) once, so that each objective multiplies instead of dividing
    const F2 rqm1 = shannon ? F2{0.f, 0.f} : df_div(F2{1.0f, 0.f}, qm1);
    auto sweep = [&](int mode, float lower, Top& tp, double& bv, int& bi) {
        F2 qa = w_before;
        long long na = c_before;
        for (int g = j0; g < j1; g += 2) {
            int cn[2];
            long long nag[2];
            float2 tw[2], pa[2], pb[2];
            long long nn = na;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                cn[u] = g + u < j1 ? sIC[g + u].y : 0;
                nn += cn[u];
                nag[u] = nn;
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const bool ok = !shannon && cn[u] > 0 && N - nag[u] > 0;
                tw[u] = cn[u] > 0 ? __ldg(Tp + cn[u]) : make_float2(0.f, 0.f);
                pa[u] = ok ? __ldg(Tp + nag[u]) : make_float2(1.f, 0.f);
                pb[u] = ok ? __ldg(Tp + (N - nag[u])) : make_float2(1.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int j = g + u;
                if (j >= j1) break;
                qa = f2_add(qa, F2{tw[u].x, tw[u].y});
                na = nag[u];
                const long long nb = N - na;
                if (nb <= 0) continue;
                const float2 qb2 = sW[j];
                const F2 QB{qb2.x, qb2.y};
                F2 phi, la{0.f, 0.f}, lb{0.f, 0.f};
                float band;
                if (shannon) {
                    la = df_log2_count<true>((unsigned)na, T);
                    lb = df_log2_count<true>((unsigned)nb, T);
                    const F2 sa = df_div_fast(qa, df_from_u32((unsigned)na)),
                             sb = df_div_fast(QB, df_from_u32((unsigned)nb));
                    phi = df_mul(df_add(df_add(la, f2_neg(sa)), df_add(lb, f2_neg(sb))), df_ln2());
                    band = shannon_band_df(la.hi, sa.hi, lb.hi, sb.hi);
                } else {
                    const F2 ab =
                        df_mul(df_div_fast(qa, F2{pa[u].x, pa[u].y}), df_div_fast(QB, F2{pb[u].x, pb[u].y}));
                    phi = df_mul(df_add(F2{1.0f, 0.f}, f2_neg(ab)), rqm1);
                    band = tsallis_band_df(ab.hi, phi.hi, q);
                }
                const int lev = sIC[j].x;
                if (mode == 0) {
                    tp = top_merge(Top{phi, lev, band, -INFINITY}, tp);
                } else if (phi.hi + band >= lower) {
                    // FP64 (a slow pipe here) only for the entries the bounds leave in play
                    const double f =
                        shannon ? 0.6931471805599453 * ((df_to_double(la) - df_to_double(qa) / (double)na) +
                                                        (df_to_double(lb) - df_to_double(QB) / (double)nb))
                                : (1.0 - (df_to_double(qa) / ((double)pa[u].x + (double)pa[u].y)) *
                                             (df_to_double(QB) / ((double)pb[u].x + (double)pb[u].y))) /
                                      ((double)q - 1.0);
                    argmax_merge(bv, bi, f, lev);
                }
            }
        }
    };
    Top tp{{-INFINITY, 0.f}, -1, 0.f, -INFINITY};
    double bv = -INFINITY;
    int bi = -1;
    sweep(0, 0.f, tp, bv, bi);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) tp = top_merge(tp, shfl_top(tp, d));
    if (lane == 0) {
        sm.top_vh[warp] = tp.v.hi;
        sm.top_vl[warp] = tp.v.lo;
        sm.top_i[warp] = tp.i;
        sm.top_band[warp] = tp.band;
        sm.top_u2[warp] = tp.u2;
    }
    Sync::sync();   // 4
    Top gt = block_top_of(sm);
    if (gt.i < 0) {
        Sync::sync();
        return SearchResult{-1, 0.f, TSALLIS_ERR_NO_VALID_THRESHOLD};
    }
    if (!(gt.u2 >= gt.v.hi - gt.band)) {
        Sync::sync();   // sIC / sW / sm may be reused by the caller after this
        return SearchResult{gt.i, gt.v.hi + gt.v.lo, TSALLIS_OK};
    }
    // ---- 4. near ties: FP64 from the same double-float sums and powers
    sweep(1, gt.v.hi - gt.band, tp, bv, bi);
    block_argmax_d<Sync>(bv, bi, sm);
    const int t_win = sm.red_i[0];
    const float phi_win = (float)sm.red_dv[0];
    Sync::sync();
    return SearchResult{t_win, phi_win, TSALLIS_OK | TSALLIS_STATUS_RERANKED};
}

// ------------------------------------------------------------ window search
//
// The exact search started from a window of candidate levels (a proposer's
// ranking). The terms, sums and per-level objective are those of the table
// search above, with the terms computed rather than read from a table. The
// objective is first evaluated at the canonical thresholds of the candidates
// (a candidate at an empty level stands for the non-empty level below it,
// which gives the same partition). Then, for every block of 64 levels, a
// bound on the objective over the block follows from the class sums at its
// two ends, because N_1 and Q_1 grow and N_2 and Q_2 shrink as t grows:
//   q < 1:  a b' <= Q_1(hi) Q_2(lo) / ((N_1(lo) N_2(hi)) / N^2)^q,
//           phi = (a b' - 1) / (1 - q) grows with a b';
//   q > 1:  a b' >= Q_1(lo) Q_2(hi) / ((N_1(hi) N_2(lo)) / N^2)^q,
//           phi = (1 - a b') / (q - 1) falls with a b';
//   q = 1:  H_1 <= log N_1(hi) - S_1(lo) / N_1(hi) and
//           H_2 <= log N_2(lo) - S_2(hi) / N_2(lo) (S = sum h log h >= 0).
// Every block whose bound reaches the window's maximum (less its error
// bound) is searched exhaustively, so the result is the exhaustive search's
// result. A block with an empty class 1 at its start or an empty class 2 at
// its end has no finite bound and is always searched.
struct WindowSmem {
    long long na_lo[64], na_hi[64];
    float qa_lo[64][2], qa_hi[64][2], qb_lo[64][2], qb_hi[64][2];
    unsigned char fallback[64];
    unsigned char sel[kMaxBins];   // bit 0: proposed level; bit 1: evaluated in the window
    int nfb;
};

__device__ __forceinline__ float window_block_bound(const WindowSmem& ws, int b, long long N, F2 LN, float q,
                                                    const DfTables* __restrict__ T) {
    const long long na_lo = ws.na_lo[b], na_hi = ws.na_hi[b];
    const long long nb_lo = N - na_lo, nb_hi = N - na_hi;
    if (na_hi <= 0 || nb_lo <= 0) return -INFINITY;   // no threshold of the block has two classes
    const F2 qa_lo{ws.qa_lo[b][0], ws.qa_lo[b][1]}, qa_hi{ws.qa_hi[b][0], ws.qa_hi[b][1]};
    const F2 qb_lo{ws.qb_lo[b][0], ws.qb_lo[b][1]}, qb_hi{ws.qb_hi[b][0], ws.qb_hi[b][1]};
    F2 u;
    if (q == 1.0f) {
        const F2 la = df_log2_count<false>((unsigned)na_hi, T), lb = df_log2_count<false>((unsigned)nb_lo, T);
        const F2 sa = df_div(qa_lo, df_from_u32((unsigned)na_hi)), sb = df_div(qb_hi, df_from_u32((unsigned)nb_lo));
        u = df_mul(df_add(df_add(la, f2_neg(sa)), df_add(lb, f2_neg(sb))), df_ln2());
    } else if (q < 1.0f) {
        if (na_lo <= 0 || nb_hi <= 0) return INFINITY;
        const F2 pa = df_pow_ratio<false>((unsigned)na_lo, LN, q, T), pb = df_pow_ratio<false>((unsigned)nb_hi, LN, q, T);
        const F2 ab = df_mul(df_div(qa_hi, pa), df_div(qb_lo, pb));
        u = df_div(df_add(ab, F2{-1.0f, 0.f}), two_sum(1.0f, -q));
    } else {
        const F2 pa = df_pow_ratio<false>((unsigned)na_hi, LN, q, T), pb = df_pow_ratio<false>((unsigned)nb_lo, LN, q, T);
        const F2 ab = df_mul(df_div(qa_lo, pa), df_div(qb_hi, pb));
        u = df_div(df_add(F2{1.0f, 0.f}, f2_neg(ab)), two_sum(q, -1.0f));
    }
    const float v = u.hi + u.lo;
    return v + 1e-9f * fabsf(v) + 1e-30f;   // the bound's own rounding
}

template <class Sync>
__device__ SearchResult search1d_window(const int32_t* __restrict__ h, int L, float q, const int32_t* __restrict__ cand,
                                        int ncand, SearchSmem& sm, WindowSmem& ws, float2* __restrict__ sW,
                                        float2* __restrict__ sQ, const DfTables* __restrict__ T) {
    const int tid = Sync::tid(), lane = tid & 31, warp = tid >> 5;
    const bool shannon = (q == 1.0f);
    const int base = tid * kBinsPerThread;

    int hv[kBinsPerThread];
    int c = 0, lastnz = -1;
#pragma unroll
    for (int k = 0; k < kBinsPerThread; ++k) {
        hv[k] = base + k < L ? __ldcg(h + base + k) : 0;
        c += hv[k];
        if (hv[k] > 0) lastnz = base + k;
        ws.sel[base + k] = 0;
    }
    // counts (prefix, total) and the last non-empty level before each thread
    long long ci = c;
    int li = lastnz;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long oc = __shfl_up_sync(0xffffffffu, ci, d);
        const int ol = __shfl_up_sync(0xffffffffu, li, d);
        if (lane >= d) { ci += oc; li = max(li, ol); }
    }
    if (lane == 31) { sm.cnt_pre[warp] = ci; sm.red_i[warp] = li; }
    Sync::sync();
    if (warp == 0) {
        const long long cw = lane < kSearchWarps ? sm.cnt_pre[lane] : 0;
        const int lw = lane < kSearchWarps ? sm.red_i[lane] : -1;
        long long cc = cw;
        int ll = lw;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long oc = __shfl_up_sync(0xffffffffu, cc, d);
            const int ol = __shfl_up_sync(0xffffffffu, ll, d);
            if (lane >= d) { cc += oc; ll = max(ll, ol); }
        }
        int le = __shfl_up_sync(0xffffffffu, ll, 1);
        if (lane == 0) le = -1;
        const long long tot = __shfl_sync(0xffffffffu, cc, kSearchWarps - 1);
        __syncwarp();
        if (lane < kSearchWarps) { sm.cnt_pre[lane] = cc - cw; sm.red_i[lane] = le; }
        if (lane == 0) sm.total = tot;
    }
    // proposed levels
    for (int i = tid; i < ncand; i += kSearchThreads) {
        const int t = cand[i];
        if (t >= 0 && t < L) ws.sel[t] = 1;
    }
    Sync::sync();
    const long long N = sm.total;
    long long c_before = __shfl_up_sync(0xffffffffu, ci, 1);
    int l_before = __shfl_up_sync(0xffffffffu, li, 1);
    if (lane == 0) { c_before = 0; l_before = -1; }
    c_before += sm.cnt_pre[warp];
    l_before = max(l_before, sm.red_i[warp]);
    // a proposed level stands for the last non-empty level at or below it
    {
        int last = l_before;
#pragma unroll
        for (int k = 0; k < kBinsPerThread; ++k) {
            if (hv[k] > 0) last = base + k;
            if ((ws.sel[base + k] & 1) && last >= 0) ws.sel[last] |= 2;
        }
    }

    // terms, running sums, block scans (as in the table search)
    const F2 LN = shannon ? F2{0.f, 0.f} : df_log2_count<false>((unsigned)N, T);
    F2 run{0.f, 0.f};
#pragma unroll
    for (int k = 0; k < kBinsPerThread; ++k) {
        F2 w{0.f, 0.f};
        if (hv[k] > 0) w = shannon ? df_hlog2h<false>((unsigned)hv[k], T) : df_pow_ratio<false>((unsigned)hv[k], LN, q, T);
        sW[base + k] = make_float2(w.hi, w.lo);
        run = f2_add(run, w);
        sQ[base + k] = make_float2(run.hi, run.lo);
    }
    F2 pi = run, si = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const F2 op = shfl_up_f2(pi, d);
        const F2 os = shfl_down_f2(si, d);
        if (lane >= d) pi = f2_add(op, pi);
        if (lane + d < 32) si = f2_add(si, os);
    }
    if (lane == 31) sm.w_pre[warp] = pi;
    if (lane == 0) sm.w_suf[warp] = si;
    Sync::sync();
    if (warp == 0) {
        F2 pp = lane < kSearchWarps ? sm.w_pre[lane] : F2{0.f, 0.f};
        F2 ss = lane < kSearchWarps ? sm.w_suf[lane] : F2{0.f, 0.f};
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const F2 op = shfl_up_f2(pp, d);
            const F2 os = shfl_down_f2(ss, d);
            if (lane >= d) pp = f2_add(op, pp);
            if (lane + d < 32) ss = f2_add(ss, os);
        }
        F2 pe = shfl_up_f2(pp, 1);
        if (lane == 0) pe = F2{0.f, 0.f};
        const F2 se = shfl_down_f2(ss, 1);
        __syncwarp();
        if (lane < kSearchWarps) { sm.w_pre[lane] = pe; sm.w_suf[lane] = se; }
    }
    Sync::sync();
    F2 w_before = shfl_up_f2(pi, 1);
    F2 w_after = shfl_down_f2(si, 1);
    if (lane == 0) w_before = F2{0.f, 0.f};
    if (lane == 31) w_after = F2{0.f, 0.f};
    w_before = f2_add(sm.w_pre[warp], w_before);
    w_after = f2_add(w_after, sm.w_suf[warp]);

    const F2 qm1 = two_sum(q, -1.0f);
    // objective at level k of this thread (valid: non-empty, class 2 non-empty)
    auto eval = [&](int k, long long na, F2 QA, F2 QB, F2& phi, float& band, double* f64) {
        const long long nb = N - na;
        if (shannon) {
            const F2 la = df_log2_count<false>((unsigned)na, T), lb = df_log2_count<false>((unsigned)nb, T);
            const F2 sa = df_div(QA, df_from_u32((unsigned)na)), sb = df_div(QB, df_from_u32((unsigned)nb));
            phi = df_mul(df_add(df_add(la, f2_neg(sa)), df_add(lb, f2_neg(sb))), df_ln2());
            band = shannon_band_df(la.hi, sa.hi, lb.hi, sb.hi);
            if (f64)
                *f64 = 0.6931471805599453 * ((df_to_double(la) - df_to_double(QA) / (double)na) +
                                             (df_to_double(lb) - df_to_double(QB) / (double)nb));
        } else {
            const F2 pa = df_pow_ratio<false>((unsigned)na, LN, q, T), pb = df_pow_ratio<false>((unsigned)nb, LN, q, T);
            const F2 ab = df_mul(df_div(QA, pa), df_div(QB, pb));
            phi = df_div(df_add(F2{1.0f, 0.f}, f2_neg(ab)), qm1);
            band = tsallis_band_df(ab.hi, phi.hi, q);
            if (f64)
                *f64 = (1.0 - (df_to_double(QA) / df_to_double(pa)) * (df_to_double(QB) / df_to_double(pb))) /
                       ((double)q - 1.0);
        }
    };
    // pass over this thread's levels, right to left; mode 0: the window,
    // and the class sums at the ends of each 64-level block; mode 1: the
    // window and the fallback blocks; mode 2: FP64 at levels within lower
    auto sweep = [&](int mode, float lower, Top& tp, double& bv, int& bi) {
        long long na = c_before + c;
        F2 rs{0.f, 0.f};
        const bool fb = mode >= 1 && ws.fallback[tid >> 3];
        for (int k = kBinsPerThread - 1; k >= 0; --k) {
            const F2 QA = f2_add(w_before, F2{sQ[base + k].x, sQ[base + k].y});
            const F2 QB = f2_add(rs, w_after);
            if (mode == 0 && k == 0 && (tid & 7) == 0) {
                ws.na_lo[tid >> 3] = na;
                ws.qa_lo[tid >> 3][0] = QA.hi; ws.qa_lo[tid >> 3][1] = QA.lo;
                ws.qb_lo[tid >> 3][0] = QB.hi; ws.qb_lo[tid >> 3][1] = QB.lo;
            }
            if (mode == 0 && k == kBinsPerThread - 1 && (tid & 7) == 7) {
                ws.na_hi[tid >> 3] = na;
                ws.qa_hi[tid >> 3][0] = QA.hi; ws.qa_hi[tid >> 3][1] = QA.lo;
                ws.qb_hi[tid >> 3][0] = QB.hi; ws.qb_hi[tid >> 3][1] = QB.lo;
            }
            const bool valid = hv[k] > 0 && N - na > 0;
            if (valid && ((ws.sel[base + k] & 2) || fb)) {
                F2 phi;
                float band;
                eval(k, na, QA, QB, phi, band, nullptr);
                if (mode < 2) {
                    tp = top_merge(Top{phi, base + k, band, -INFINITY}, tp);
                } else if (phi.hi + band >= lower) {
                    double f = 0.0;   // FP64 only inside the bounds (the same phi and band again)
                    eval(k, na, QA, QB, phi, band, &f);
                    argmax_merge(bv, bi, f, base + k);
                }
            }
            const float2 wk = sW[base + k];
            rs = f2_add(F2{wk.x, wk.y}, rs);
            na -= hv[k];
        }
    };
    auto block_top = [&](Top tp) -> Top {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) tp = top_merge(tp, shfl_top(tp, d));
        if (lane == 0) {
            sm.top_vh[warp] = tp.v.hi;
            sm.top_vl[warp] = tp.v.lo;
            sm.top_i[warp] = tp.i;
            sm.top_band[warp] = tp.band;
            sm.top_u2[warp] = tp.u2;
        }
        Sync::sync();
        Top g = block_top_of(sm);
        Sync::sync();
        return g;
    };
    double bv = -INFINITY;
    int bi = -1;
    Top tp{{-INFINITY, 0.f}, -1, 0.f, -INFINITY};
    sweep(0, 0.f, tp, bv, bi);
    const Top gw = block_top(tp);    // the window's maximum (also publishes the block ends)
    // blocks whose bound reaches the window's maximum
    if (tid < 64) {
        const float lower = gw.i >= 0 ? gw.v.hi - gw.band : -INFINITY;
        const F2 LNb = shannon ? F2{0.f, 0.f} : LN;
        ws.fallback[tid] = (64 * tid < L) && window_block_bound(ws, tid, N, LNb, q, T) >= lower;
    }
    if (tid == 0) ws.nfb = 0;
    Sync::sync();
    if (tid < 64 && ws.fallback[tid]) atomicAdd(&ws.nfb, 1);
    tp = Top{{-INFINITY, 0.f}, -1, 0.f, -INFINITY};
    sweep(1, 0.f, tp, bv, bi);
    const Top g = block_top(tp);
    const int nfb = ws.nfb;
    if (g.i < 0) {
        Sync::sync();
        return SearchResult{-1, 0.f, TSALLIS_ERR_NO_VALID_THRESHOLD | (nfb << 16)};
    }
    int t_win = g.i;
    float phi_win = g.v.hi + g.v.lo;
    int status = TSALLIS_OK;
    if (g.u2 >= g.v.hi - g.band) {
        sweep(2, g.v.hi - g.band, tp, bv, bi);
        block_argmax_d<Sync>(bv, bi, sm);
        t_win = sm.red_i[0];
        phi_win = (float)sm.red_dv[0];
        status |= TSALLIS_STATUS_RERANKED;
        Sync::sync();
    }
    if (ws.sel[t_win] & 2) status |= TSALLIS_STATUS_WINDOW_HIT;
    Sync::sync();
    return SearchResult{t_win, phi_win, status | (nfb << 16)};
}

}  // namespace tsl
