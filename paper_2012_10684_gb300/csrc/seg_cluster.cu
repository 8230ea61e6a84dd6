// Per-slice 1-D thresholding with the slice held on chip by a thread-block
// cluster (section II-C "Tsallis entropy" read in 1-D, and Algorithm 1).
//
// One cluster of kClusterCtas CTAs owns one slice at a time; each CTA owns
// one contiguous part of it (at most kPartVox voxels, 64 KB):
//   1. the part is copied from HBM into the CTA's shared memory by the bulk
//      copy engine (cp.async.bulk, in kChunks chunks, each completing on its
//      own mbarrier), and counted into the CTA's 4096-level histogram as the
//      chunks land;
//   2. the cluster's histograms are summed through distributed shared
//      memory: CTA r sums levels [512 r, 512 r + 512) of all eight (a
//      reduce-scatter), so each thread of the cluster holds one level;
//   3. the exhaustive search runs on all 4096 threads of the cluster, one
//      level per thread (below);
//   4. every CTA binarises its part from shared memory (Algorithm 1) and
//      streams the mask out.
// The volume is read from HBM exactly once and the mask written once
// (3 bytes per voxel), whatever the L2 does. Two CTAs of different clusters
// share an SM, so one streams while the other searches.
//
// Search (one level b per thread, class 1 = levels 0..b, class 2 = b+1..L-1):
// with w_i = 2^64 (h_i / N)^q (double-float, dfmath.cuh), the sums
// Q_1(b) = sum_{i<=b} w_i and Q_2(b) = sum_{i>b} w_i are double-float prefix
// and suffix scans (class-2 sums are summed from the right, never formed as
// total minus class-1), N_1 and N_2 are exact integers, and
//     phi(b) = (1 - a b') / (q - 1),  a = Q_1 / 2^64 (N_1/N)^q,  b' = Q_2 / 2^64 (N_2/N)^q,
// which equals H_1 + H_2 + (1 - q) H_1 H_2 (pseudo-additivity); q = 1 uses
// the Shannon limit. phi is evaluated in double-float at every non-empty
// level b with a non-empty class 2 (the canonical thresholds: an empty
// level gives the same partition as the non-empty level below it). The
// argmax (smallest b on equal values) is taken on the double-float values
// together with a bound on their error; when another level's value lies
// within the bounds of the maximum, those candidates are re-ranked in FP64.
#include <cmath>
#include <cstdint>

#include "common.cuh"
#include "dfmath.cuh"
#include "kernels.h"
#include "top.cuh"
#include "../../include/tsallis.h"

namespace tsl {

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kChunks = 4;
constexpr int kChunkVox = kClusterPartVox / kChunks;   // 8192 voxels, 16 KB
constexpr int kLevelsPerCta = kMaxBins / kClusterCtas;  // 512

static_assert(kLevelsPerCta == kThreads, "one level per thread");
static_assert(kChunkVox % 8 == 0, "chunks are whole 16-byte words");

// ------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// All threads of all CTAs of the cluster; release/acquire orders shared
// memory (local and distributed) around it.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of the same shared variable in CTA `rank` of the cluster.
__device__ __forceinline__ unsigned map_rank(unsigned local, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ int ld_cluster_s32(unsigned addr) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void st_cluster_u32(unsigned addr, unsigned v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bulk copy global -> this CTA's shared memory, completing on an mbarrier;
// the lines are marked evict-first in L2 (they are not read again).
__device__ __forceinline__ void bulk_load(unsigned dst, const void* src, unsigned bytes, unsigned bar,
                                          unsigned long long policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar), "l"(policy)
        : "memory");
}
__device__ __forceinline__ unsigned long long policy_evict_first() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void st_stream_v2(void* p, uint2 v) {
    asm volatile("st.global.cs.v2.u32 [%0], {%1,%2};" ::"l"(p), "r"(v.x), "r"(v.y) : "memory");
}

// ------------------------------------------------------------ shared memory

struct TotRec {       // one CTA's totals for the cluster-wide scans
    int count;
    float whi, wlo;
    int err;
};
struct TopRec {
    float vhi, vlo;
    int i;
    float band, u2;
    int pad[3];
};
struct DblRec {
    double v;
    int i;
    int pad;
};

struct SmemCtl {
    unsigned long long mbar[kChunks];
    TotRec tot[kClusterCtas];
    TopRec top[kClusterCtas];
    DblRec dbl[kClusterCtas];
    int zfirst;           // first slice of the cluster (broadcast once)
    int znext;            // next slice (broadcast every slice)
    int err;              // a chunk wait of this CTA ran out in this slice
    // block scans
    int wc[kWarps];
    F2 wp[kWarps];
    F2 ws[kWarps];
    Top wt[kWarps];
    double wd[kWarps];
    int wdi[kWarps];
};

__device__ __forceinline__ bool wait_chunk(unsigned bar, unsigned parity, unsigned long long t0,
                                           unsigned long long timeout_ns) {
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer_ns() - t0 > timeout_ns) return false;
    }
    return true;
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 2) k_slice_cluster(const ClusterArgs a) {
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    uint4* buf = reinterpret_cast<uint4*>(smem_dyn);                                  // the part
    int* hist = reinterpret_cast<int*>(smem_dyn + (size_t)kClusterPartVox * 2);       // 4096 levels
    __shared__ SmemCtl ctl;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned rank = cluster_rank();
    const long long S = a.slice_vox;
    const long long P = a.part_vox;
    const long long pstart = (long long)rank * P;
    const int plen = (int)(pstart >= S ? 0 : (S - pstart < P ? S - pstart : P));   // voxels of this part
    const int hi_v = a.lo + a.L - 1 > 32767 ? 32767 : a.lo + a.L - 1;
    const unsigned LO2 = ((unsigned)a.lo & 0xffffu) * 0x10001u;
    const unsigned HI2 = ((unsigned)hi_v & 0xffffu) * 0x10001u;
    int* histb = hist - a.lo;   // histb[v] is level v - lo
    __shared__ DfTables sdf;
    const DfTables* T = &sdf;
    const bool shannon = a.q == 1.0f;
    const F2 qm1 = two_sum(a.q, -1.0f);                  // q - 1, exact
    const int level = (int)rank * kLevelsPerCta + tid;   // this thread's level in the search
    const unsigned long long pol = policy_evict_first();
    const unsigned buf_s = smem_addr(buf);

    for (int i = tid; i < kMaxBins; i += kThreads) hist[i] = 0;
    df_stage(&sdf, static_cast<const DfTables*>(a.df_tables), tid, kThreads);
    if (tid == 0) {
        for (int c = 0; c < kChunks; ++c) mbar_init(smem_addr(&ctl.mbar[c]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        ctl.err = 0;
    }
    __syncthreads();
    const F2 LN = df_log2_count<false>((unsigned)S, T);   // log2 N, N = S voxels per slice (after the staging)
    if (rank == 0 && tid == 0) {
        const int z0 = (int)atomicAdd(&a.hdr->h_next, 1u);
        for (unsigned k = 0; k < kClusterCtas; ++k) st_cluster_u32(map_rank(smem_addr(&ctl.zfirst), k), (unsigned)z0);
    }
    cluster_sync();
    int z = ctl.zfirst;
    unsigned phase = 0;   // parity of the chunk mbarriers' current phase (all chunks advance together)

    // the chunks of this part that carry data
    auto chunk_len = [&](int c) -> int {
        const int s = c * kChunkVox;
        return s >= plen ? 0 : (plen - s < kChunkVox ? plen - s : kChunkVox);
    };
    // chunk c of slice zz is copied unless it is empty (or the test hook
    // withholds it); every thread evaluates this identically
    auto copied = [&](int zz, int c) -> bool {
        return chunk_len(c) > 0 && !((a.flags & 1u) && zz == 0 && rank == 0 && c == 0);
    };
    auto issue = [&](int zz) {
        if (tid == 0) {
            const int16_t* src = a.vol + (long long)zz * S + pstart;
            for (int c = 0; c < kChunks; ++c) {
                if (!copied(zz, c)) continue;
                const int n = chunk_len(c);
                const unsigned bar = smem_addr(&ctl.mbar[c]);
                mbar_arrive_expect_tx(bar, (unsigned)n * 2u);
                bulk_load(buf_s + (unsigned)c * kChunkVox * 2u, src + (long long)c * kChunkVox, (unsigned)n * 2u, bar,
                          pol);
            }
        }
    };
    if (z < a.nz) issue(z);

    while (z < a.nz) {
        // next slice index for the cluster (read by every CTA after the next barrier)
        if (rank == 0 && tid == 0) {
            const int zn = (int)atomicAdd(&a.hdr->h_next, 1u);
            for (unsigned k = 0; k < kClusterCtas; ++k) st_cluster_u32(map_rank(smem_addr(&ctl.znext), k), (unsigned)zn);
        }

        // ---- 1. histogram of the part, chunk by chunk as the copies land
        const unsigned long long t0 = globaltimer_ns();
        bool ok = true;
        for (int c = 0; c < kChunks; ++c) {
            const int n = chunk_len(c);
            if (n == 0) break;
            if (!wait_chunk(smem_addr(&ctl.mbar[c]), phase, t0, a.timeout_ns)) {
                ok = false;
                break;
            }
            const uint4* cb = buf + c * (kChunkVox / 8);
            for (int i = tid; i < (n >> 3); i += kThreads) {
                const uint4 r = cb[i];
                const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const unsigned cl = __vmins2(__vmaxs2(w[j], LO2), HI2);
                    atomicAdd(histb + (int)(short)(cl & 0xffffu), 1);
                    atomicAdd(histb + (((int)cl) >> 16), 1);
                }
            }
        }
        if (!ok) ctl.err = 1;   // benign race: every writer stores 1
        cluster_sync();   // #1: every histogram of the cluster is complete; znext visible
        const int znext = ctl.znext;

        // ---- 2. reduce-scatter: this thread's level summed over the cluster
        int cnt = 0;
        {
            const unsigned la = smem_addr(hist + level);
#pragma unroll
            for (unsigned k = 0; k < kClusterCtas; ++k) cnt += ld_cluster_s32(map_rank(la, k));
        }

        // ---- 3. term and CTA-level scans (counts; terms prefix and suffix)
        F2 w{0.f, 0.f};
        if (cnt > 0) w = shannon ? df_hlog2h<false>((unsigned)cnt, T) : df_pow_ratio<false>((unsigned)cnt, LN, a.q, T);
        int c_inc = cnt;
        F2 w_inc = w, w_sinc = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int oc = __shfl_up_sync(0xffffffffu, c_inc, d);
            const F2 op = shfl_up_f2(w_inc, d);
            const F2 os = shfl_down_f2(w_sinc, d);
            if (lane >= d) { c_inc += oc; w_inc = f2_add(op, w_inc); }
            if (lane + d < 32) w_sinc = f2_add(w_sinc, os);
        }
        if (lane == 31) { ctl.wc[warp] = c_inc; ctl.wp[warp] = w_inc; }
        if (lane == 0) ctl.ws[warp] = w_sinc;
        __syncthreads();
        if (warp == 0) {
            // scans over the warp totals: exclusive prefix and exclusive
            // suffix of each warp, and this CTA's totals
            const int cw = lane < kWarps ? ctl.wc[lane] : 0;
            int ci = cw;
            F2 pi = lane < kWarps ? ctl.wp[lane] : F2{0.f, 0.f};
            F2 si = lane < kWarps ? ctl.ws[lane] : F2{0.f, 0.f};
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int oc = __shfl_up_sync(0xffffffffu, ci, d);
                const F2 op = shfl_up_f2(pi, d);
                const F2 os = shfl_down_f2(si, d);
                if (lane >= d) { ci += oc; pi = f2_add(op, pi); }
                if (lane + d < 32) si = f2_add(si, os);
            }
            F2 pe = shfl_up_f2(pi, 1);
            if (lane == 0) pe = F2{0.f, 0.f};
            const F2 se = shfl_down_f2(si, 1);
            const int ctot = __shfl_sync(0xffffffffu, ci, kWarps - 1);
            const F2 wtot{__shfl_sync(0xffffffffu, pi.hi, kWarps - 1), __shfl_sync(0xffffffffu, pi.lo, kWarps - 1)};
            __syncwarp();
            if (lane < kWarps) {
                ctl.wc[lane] = ci - cw;
                ctl.wp[lane] = pe;
                ctl.ws[lane] = se;
            }
            // this CTA's totals into slot `rank` of every CTA of the cluster
            if (lane < kClusterCtas) {
                const unsigned base = map_rank(smem_addr(&ctl.tot[rank]), (unsigned)lane);
                st_cluster_u32(base + 0, (unsigned)ctot);
                st_cluster_u32(base + 4, __float_as_uint(wtot.hi));
                st_cluster_u32(base + 8, __float_as_uint(wtot.lo));
                st_cluster_u32(base + 12, (unsigned)ctl.err);
            }
        }
        __syncthreads();
        // this thread's local prefix (inclusive) and suffix (exclusive) within the CTA
        int n_loc = c_inc + ctl.wc[warp];
        F2 qa_loc = f2_add(ctl.wp[warp], w_inc);
        F2 sx = shfl_down_f2(w_sinc, 1);
        if (lane == 31) sx = F2{0.f, 0.f};
        F2 qb_loc = f2_add(sx, ctl.ws[warp]);
        cluster_sync();   // #3: totals of every CTA visible; every peer has read this CTA's histogram
        for (int i = tid; i < kMaxBins; i += kThreads) hist[i] = 0;
        if (tid == 0) ctl.err = 0;

        // ---- 4. class sums across the cluster, objective, error bound
        int errs = 0;
        long long n_before = 0;
        F2 w_before{0.f, 0.f}, w_after{0.f, 0.f};
#pragma unroll
        for (int k = 0; k < kClusterCtas; ++k) {
            const TotRec t = ctl.tot[k];
            errs |= t.err;
            if (k < (int)rank) { n_before += t.count; w_before = f2_add(w_before, F2{t.whi, t.wlo}); }
        }
#pragma unroll
        for (int k = kClusterCtas - 1; k > (int)rank; --k) w_after = f2_add(F2{ctl.tot[k].whi, ctl.tot[k].wlo}, w_after);
        const long long na = n_before + n_loc;
        const long long nb = S - na;
        const F2 QA = f2_add(w_before, qa_loc);
        const F2 QB = f2_add(qb_loc, w_after);
        const bool valid = cnt > 0 && nb > 0 && level <= a.L - 2;
        F2 my_phi{-INFINITY, 0.f};
        float my_band = 0.f;
        F2 ka{0.f, 0.f}, kb{0.f, 0.f};   // class powers 2^64 (N_k/N)^q, or log2 N_k (Shannon)
        if (valid) {
            if (shannon) {
                ka = df_log2_count<false>((unsigned)na, T);
                kb = df_log2_count<false>((unsigned)nb, T);
                const F2 sa = df_div(QA, df_from_u32((unsigned)na)), sb = df_div(QB, df_from_u32((unsigned)nb));
                const F2 bits = df_add(df_add(ka, f2_neg(sa)), df_add(kb, f2_neg(sb)));
                my_phi = df_mul(bits, df_ln2());
                my_band = shannon_band_df(ka.hi, sa.hi, kb.hi, sb.hi);
            } else {
                ka = df_pow_ratio<false>((unsigned)na, LN, a.q, T);
                kb = df_pow_ratio<false>((unsigned)nb, LN, a.q, T);
                const F2 ab = df_mul(df_div(QA, ka), df_div(QB, kb));
                my_phi = df_div(df_add(F2{1.0f, 0.f}, f2_neg(ab)), qm1);
                my_band = tsallis_band_df(ab.hi, my_phi.hi, a.q);
            }
        }
        Top tp{my_phi, valid ? level : -1, my_band, -INFINITY};
        // CTA top, then the cluster top (merged in rank order by every CTA)
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) tp = top_merge(tp, shfl_top(tp, d));
        if (lane == 0) ctl.wt[warp] = tp;
        __syncthreads();
        if (warp == 0) {
            Top t = lane < kWarps ? ctl.wt[lane] : Top{{-INFINITY, 0.f}, -1, 0.f, -INFINITY};
#pragma unroll
            for (int d = 8; d > 0; d >>= 1) t = top_merge(t, shfl_top(t, d));
            if (lane < kClusterCtas) {
                const unsigned base = map_rank(smem_addr(&ctl.top[rank]), (unsigned)lane);
                st_cluster_u32(base + 0, __float_as_uint(t.v.hi));
                st_cluster_u32(base + 4, __float_as_uint(t.v.lo));
                st_cluster_u32(base + 8, (unsigned)t.i);
                st_cluster_u32(base + 12, __float_as_uint(t.band));
                st_cluster_u32(base + 16, __float_as_uint(t.u2));
            }
        }
        cluster_sync();   // #4: every CTA's top visible
        Top g{{-INFINITY, 0.f}, -1, 0.f, -INFINITY};
#pragma unroll
        for (int k = 0; k < kClusterCtas; ++k) {
            const TopRec r = ctl.top[k];
            g = top_merge(g, Top{{r.vhi, r.vlo}, r.i, r.band, r.u2});
        }
        int t_win = g.i;
        float phi_win = g.v.hi + g.v.lo;
        int status = TSALLIS_OK;
        if (errs) {
            t_win = -1;
            phi_win = 0.f;
            status = TSALLIS_ERR_TIMEOUT;
        } else if (g.i < 0) {
            status = TSALLIS_ERR_NO_VALID_THRESHOLD;
            phi_win = 0.f;
        } else if (g.u2 >= g.v.hi - g.band) {
            // ---- 5. near ties: FP64 re-rank of every level inside the bounds
            const float lower = g.v.hi - g.band;
            double dv = -INFINITY;
            int di = -1;
            if (valid && my_phi.hi + my_band >= lower) {
                if (shannon)
                    dv = 0.6931471805599453 * ((df_to_double(ka) - df_to_double(QA) / (double)na) +
                                               (df_to_double(kb) - df_to_double(QB) / (double)nb));
                else
                    dv = (1.0 - (df_to_double(QA) / df_to_double(ka)) * (df_to_double(QB) / df_to_double(kb))) /
                         ((double)a.q - 1.0);
                di = level;
            }
            // CTA argmax in FP64 (smallest level on equal values)
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, dv, d);
                const int oi = __shfl_xor_sync(0xffffffffu, di, d);
                argmax_merge(dv, di, ov, oi);
            }
            if (lane == 0) { ctl.wd[warp] = dv; ctl.wdi[warp] = di; }
            __syncthreads();
            if (warp == 0) {
                double v = lane < kWarps ? ctl.wd[lane] : -INFINITY;
                int i = lane < kWarps ? ctl.wdi[lane] : -1;
#pragma unroll
                for (int d = 8; d > 0; d >>= 1) {
                    const double ov = __shfl_xor_sync(0xffffffffu, v, d);
                    const int oi = __shfl_xor_sync(0xffffffffu, i, d);
                    argmax_merge(v, i, ov, oi);
                }
                if (lane < kClusterCtas) {
                    const unsigned base = map_rank(smem_addr(&ctl.dbl[rank]), (unsigned)lane);
                    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
                    st_cluster_u32(base + 0, (unsigned)(bits & 0xffffffffu));
                    st_cluster_u32(base + 4, (unsigned)(bits >> 32));
                    st_cluster_u32(base + 8, (unsigned)i);
                }
            }
            cluster_sync();   // #5: every CTA's FP64 maximum visible
            double bv = -INFINITY;
            int bi = -1;
#pragma unroll
            for (int k = 0; k < kClusterCtas; ++k) argmax_merge(bv, bi, ctl.dbl[k].v, ctl.dbl[k].i);
            t_win = bi;
            phi_win = (float)bv;
            status = TSALLIS_OK | TSALLIS_STATUS_RERANKED;
        }

        // ---- 6. Algorithm 1 on this CTA's part, from shared memory
        {
            uint8_t* dst = a.mask + (long long)z * S + pstart;
            const bool none = t_win < 0;
            // level <= t  <=>  v <= lo + t (t below the top level); at the top every voxel
            const int T0 = (t_win >= a.L - 1) ? 32767 : (a.lo + t_win > 32767 ? 32767 : a.lo + t_win);
            const unsigned T2 = ((unsigned)T0 & 0xffffu) * 0x10001u;
            const bool le = a.polarity == 0;
            const int nv = plen >> 3;
            for (int i = tid; i < nv; i += kThreads) {
                uint2 m = make_uint2(0u, 0u);
                if (!none) {
                    const uint4 r = buf[i];
                    unsigned m0, m1, m2, m3;
                    if (le) {
                        m0 = __vcmples2(r.x, T2); m1 = __vcmples2(r.y, T2); m2 = __vcmples2(r.z, T2); m3 = __vcmples2(r.w, T2);
                    } else {
                        m0 = __vcmpgts2(r.x, T2); m1 = __vcmpgts2(r.y, T2); m2 = __vcmpgts2(r.z, T2); m3 = __vcmpgts2(r.w, T2);
                    }
                    m = make_uint2(__byte_perm(m0, m1, 0x6420) & 0x01010101u, __byte_perm(m2, m3, 0x6420) & 0x01010101u);
                }
                st_stream_v2(dst + (long long)i * 8, m);
            }
        }
        if (rank == 0 && tid == 0) {
            a.t_out[z] = t_win;
            a.phi_out[z] = phi_win;
            a.status[z] = status;
        }
        if (!ok) {
            // a chunk wait ran out: let copies still in flight land (bounded),
            // then start the chunk barriers afresh
            const unsigned long long t1 = globaltimer_ns();
            for (int c = 0; c < kChunks; ++c)
                if (copied(z, c)) wait_chunk(smem_addr(&ctl.mbar[c]), phase, t1, a.timeout_ns);
        }
        __syncthreads();   // every read of the part is done
        if (!ok && tid == 0) {
            for (int c = 0; c < kChunks; ++c) {
                mbar_inval(smem_addr(&ctl.mbar[c]));
                mbar_init(smem_addr(&ctl.mbar[c]), 1);
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        if (ok) phase ^= 1u;
        else phase = 0u;
        __syncthreads();
        z = znext;
        if (z < a.nz) {
            if (tid == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(z);
        }
    }

    // every peer is done with this CTA's shared memory
    cluster_sync();
    if (tid == 0) {
        __threadfence();
        const unsigned d = atomicAdd(&a.hdr->done, 1u);
        if (d == gridDim.x - 1) {
            // the last CTA resets the slice counter for the next launch
            a.hdr->h_next = 0;
            a.hdr->done = 0;
            __threadfence();
        }
    }
}

int slice_cluster_smem_bytes() { return kClusterPartVox * 2 + kMaxBins * (int)sizeof(int); }

cudaError_t slice_cluster_prepare() {
    return cudaFuncSetAttribute(k_slice_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                slice_cluster_smem_bytes());
}

cudaError_t slice_cluster_occupancy(int* max_clusters) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClusterCtas * 64);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = slice_cluster_smem_bytes();
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kClusterCtas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(max_clusters, k_slice_cluster, &cfg);
}

cudaError_t launch_slice_cluster(const ClusterArgs& a, int nclusters, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClusterCtas * nclusters);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = slice_cluster_smem_bytes();
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kClusterCtas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_slice_cluster, a);
}

}  // namespace tsl
