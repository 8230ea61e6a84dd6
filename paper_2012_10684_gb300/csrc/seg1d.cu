// 1-D thresholding path: histogram, search and binarise tiles driven by one
// persistent kernel with a work-item queue.
//
// Work items are taken in order from a global ticket counter. For uniform
// groups (slices of one volume, or the whole volume as one group) item k is
//   step s = k / (2 * ntiles), r = k % (2 * ntiles)
//   r <  ntiles : histogram tile r of group s
//   r >= ntiles : binarise tile of group s - lag (tiles in reverse order, so
//                 the most recently read part of the group is re-read first)
// A histogram tile builds a shared-memory histogram of its voxels and adds
// it to the group's histogram in global memory. The last tile of a group to
// arrive runs the search for that group and publishes the threshold. A
// binarise tile waits (bounded) for its group's threshold, then re-reads its
// voxels, which are still in L2 when the group is a slice, and writes the mask
// (Algorithm 1).
//
// No waits can deadlock: every histogram item is taken before any binarise
// item of the same group, and histogram items never wait.
#include "common.cuh"
#include "search1d.cuh"
#include "kernels.h"

namespace tsl {

constexpr int kSegThreads = kSearchThreads;  // 512

__device__ __forceinline__ long long lmin(long long a, long long b) { return a < b ? a : b; }

__device__ __forceinline__ void accumulate8(uint4 r, int lo, int L, int* __restrict__ sh, int copy, int C,
                                            unsigned& low) {
    const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int v0 = (int)(short)(w[j] & 0xffffu);
        const int v1 = ((int)w[j]) >> 16;
        const int b0 = level_of(v0, lo, L), b1 = level_of(v1, lo, L);
        if (b0 == 0) ++low; else atomicAdd(&sh[b0 * C + copy], 1);
        if (b1 == 0) ++low; else atomicAdd(&sh[b1 * C + copy], 1);
    }
}

// Histogram of n voxels at src into the shared histogram sh[L][C], then add
// it to gdst[L] and leave sh zeroed.
template <int C>
__device__ void hist_tile(const int16_t* __restrict__ src, long long n, int lo, int L, int* __restrict__ sh,
                          int* __restrict__ gdst) {
    const int tid = threadIdx.x;
    const int copy = (tid & 31) % C;
    unsigned low = 0;
    // scalar head up to 16-byte alignment
    const int head = (int)lmin(n, (long long)((((16 - ((uintptr_t)src & 15)) & 15)) >> 1));
    if (tid < head) {
        int b = level_of(src[tid], lo, L);
        if (b == 0) ++low; else atomicAdd(&sh[b * C + copy], 1);
    }
    const uint4* vsrc = reinterpret_cast<const uint4*>(src + head);
    const long long nv = (n - head) >> 3;
    long long i = tid;
    for (; i + 3 * kSegThreads < nv; i += 4 * kSegThreads) {
        uint4 r0 = ld_stream_keep(vsrc + i);
        uint4 r1 = ld_stream_keep(vsrc + i + kSegThreads);
        uint4 r2 = ld_stream_keep(vsrc + i + 2 * kSegThreads);
        uint4 r3 = ld_stream_keep(vsrc + i + 3 * kSegThreads);
        accumulate8(r0, lo, L, sh, copy, C, low);
        accumulate8(r1, lo, L, sh, copy, C, low);
        accumulate8(r2, lo, L, sh, copy, C, low);
        accumulate8(r3, lo, L, sh, copy, C, low);
    }
    for (; i < nv; i += kSegThreads) accumulate8(ld_stream_keep(vsrc + i), lo, L, sh, copy, C, low);
    // scalar tail
    const long long tail0 = head + (nv << 3);
    if (tail0 + tid < n) {
        int b = level_of(src[tail0 + tid], lo, L);
        if (b == 0) ++low; else atomicAdd(&sh[b * C + copy], 1);
    }
    // level 0 is counted in registers (the clamped air level is the hottest)
    low = __reduce_add_sync(0xffffffffu, low);
    if ((tid & 31) == 0 && low) atomicAdd(&sh[0], (int)low);
    __syncthreads();
    for (int b = tid; b < L; b += kSegThreads) {
        int s = 0;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            s += sh[b * C + c];
            sh[b * C + c] = 0;
        }
        if (s) atomicAdd(&gdst[b], s);
    }
    __syncthreads();
}

// Algorithm 1 on n voxels: mask = level <= t (polarity 0) or level >= t + 1
// (polarity 1), where level = clamp(v - lo, 0, L-1) >> shift. With
// 0 <= t <= (L-1 >> shift) - 1 both reduce to a compare of v with
// T = lo + ((t + 1) << shift) - 1. t < 0 gives zeros.
__device__ void bin_tile(const int16_t* __restrict__ src, uint8_t* __restrict__ dst, long long n, int t, int lo,
                         int L, int shift, int polarity) {
    const int tid = threadIdx.x;
    // thresholds at or above the top level put every voxel in class 1
    const int T = (t >= ((L - 1) >> shift)) ? 0x7fffffff : lo + ((t + 1) << shift) - 1;
    const bool none = t < 0;
    const unsigned want = polarity ? 0u : 1u;   // value written when v <= T
    auto fg = [&](int v) -> unsigned { return none ? 0u : ((v <= T) ? want : 1u - want); };
    const int head = (int)lmin(n, (long long)((((16 - ((uintptr_t)src & 15)) & 15)) >> 1));
    if (tid < head) dst[tid] = (uint8_t)fg(src[tid]);
    const uint4* vsrc = reinterpret_cast<const uint4*>(src + head);
    uint8_t* vdst = dst + head;
    const long long nv = (n - head) >> 3;
    auto one = [&](uint4 r, long long i) {
        const unsigned w[4] = {r.x, r.y, r.z, r.w};
        unsigned out[2] = {0u, 0u};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int v0 = (int)(short)(w[j] & 0xffffu);
            const int v1 = ((int)w[j]) >> 16;
            out[j >> 1] |= (fg(v0) | (fg(v1) << 8)) << ((j & 1) * 16);
        }
        st_stream(vdst + i * 8, make_uint2(out[0], out[1]));
    };
    long long i = tid;
    for (; i + 3 * kSegThreads < nv; i += 4 * kSegThreads) {
        uint4 r0 = ld_last_use(vsrc + i);
        uint4 r1 = ld_last_use(vsrc + i + kSegThreads);
        uint4 r2 = ld_last_use(vsrc + i + 2 * kSegThreads);
        uint4 r3 = ld_last_use(vsrc + i + 3 * kSegThreads);
        one(r0, i);
        one(r1, i + kSegThreads);
        one(r2, i + 2 * kSegThreads);
        one(r3, i + 3 * kSegThreads);
    }
    for (; i < nv; i += kSegThreads) one(ld_last_use(vsrc + i), i);
    const long long tail0 = head + (nv << 3);
    if (tail0 + tid < n) dst[tail0 + tid] = (uint8_t)fg(src[tail0 + tid]);
}

struct Item {
    int kind;   // 0 none, 1 histogram, 2 binarise
    int group;
    int tile;
};

__device__ __forceinline__ Item decode(const SegArgs& a, unsigned k) {
    Item it{0, 0, 0};
    if (a.worklist != nullptr) {
        WorkItem w = a.worklist[k];
        it.group = w.group;
        it.kind = (w.tile < 0) ? 2 : 1;
        it.tile = w.tile & 0x7fffffff;
        return it;
    }
    const unsigned nt = (unsigned)a.ntiles;
    if (a.phases == kPhaseHist || a.phases == kPhaseBin) {
        it.group = (int)(k / nt);
        it.tile = (int)(k % nt);
        it.kind = a.phases == kPhaseHist ? 1 : 2;
        if (it.kind == 2) it.tile = a.ntiles - 1 - it.tile;
        return it;
    }
    const unsigned s = k / (2 * nt), r = k % (2 * nt);
    if (r < nt) {
        if ((int)s < a.ngroups) { it.kind = 1; it.group = (int)s; it.tile = (int)r; }
    } else {
        const int g = (int)s - a.lag;
        if (g >= 0 && g < a.ngroups) { it.kind = 2; it.group = g; it.tile = a.ntiles - 1 - (int)(r - nt); }
    }
    return it;
}

template <int C>
__global__ void __launch_bounds__(kSegThreads, 2) k_segment1d(const SegArgs a) {
    extern __shared__ int4 smem_raw[];
    int* sh = reinterpret_cast<int*>(smem_raw);
    __shared__ SearchSmem ssm;
    __shared__ unsigned s_ticket;
    __shared__ int s_flag, s_t;
    const int tid = threadIdx.x;
    const int epoch = *(volatile int*)&a.hdr->epoch;

    for (int i = tid; i < a.L * C; i += kSegThreads) sh[i] = 0;
    __syncthreads();

    for (;;) {
        if (tid == 0) s_ticket = atomicAdd(&a.hdr->ticket, 1u);
        __syncthreads();
        const unsigned k = s_ticket;
        if (k >= a.nticket) break;
        const Item it = decode(a, k);
        if (it.kind != 0) {
            const int16_t* gvol;
            uint8_t* gmask;
            long long gn;
            if (a.groups != nullptr) {
                const GroupDesc gd = a.groups[it.group];
                gvol = gd.vol; gmask = gd.mask; gn = gd.nvox;
            } else {
                gvol = a.vol + (long long)it.group * a.group_vox;
                gmask = a.mask + (long long)it.group * a.group_vox;
                gn = a.group_vox;
            }
            const long long off = (long long)it.tile * a.tile_vox;
            const long long n = lmin((long long)a.tile_vox, gn - off);
            if (it.kind == 1) {
                int* gh = a.ghist + (long long)it.group * a.L;
                if (n > 0) hist_tile<C>(gvol + off, n, a.lo, a.L, sh, gh);
                if (a.phases & kPhaseSearch) {
                    __threadfence();
                    __syncthreads();
                    if (tid == 0) {
                        int last = 0;
                        const bool skip = (a.flags & 1u) && it.group == 0 && it.tile == 0;
                        if (skip) {
                            atomicExch(&a.hdr->err, 1);
                        } else {
                            const int gt = a.groups != nullptr ? a.groups[it.group].ntiles : a.ntiles;
                            last = atomicAdd(&a.arrive[it.group], 1) == gt - 1;
                        }
                        s_flag = last;
                    }
                    __syncthreads();
                    if (s_flag) {
                        __threadfence();
                        SearchResult r = search1d_block(gh, a.L, a.q,
                                                        a.curve ? a.curve + (long long)it.group * (a.L - 1) : nullptr,
                                                        ssm);
                        // leave the group's scratch histogram zeroed for the next launch
                        for (int b = tid; b < a.L; b += kSegThreads) gh[b] = 0;
                        if (tid == 0) {
                            a.t_out[it.group] = r.t;
                            a.phi_out[it.group] = r.phi;
                            a.status[it.group] = r.status;
                            a.arrive[it.group] = 0;
                        }
                        __threadfence();
                        __syncthreads();
                        if (tid == 0) st_release(&a.ready[it.group], epoch + 1);
                    }
                }
            } else {
                if (tid == 0) {
                    int t;
                    if (a.phases & kPhaseSearch) {
                        const unsigned long long t0 = globaltimer_ns();
                        unsigned ns = 32;
                        bool ok = true;
                        while (ld_acquire(&a.ready[it.group]) != epoch + 1) {
                            if (globaltimer_ns() - t0 > a.timeout_ns) { ok = false; break; }
                            __nanosleep(ns);
                            if (ns < 2048) ns <<= 1;
                        }
                        if (ok) {
                            t = __ldcg(&a.t_out[it.group]);
                        } else {
                            // recorded now, reported by the last block once
                            // nothing of this launch can still write the status
                            a.tmo[it.group] = epoch + 1;
                            atomicExch(&a.hdr->err, 1);
                            t = -2;
                        }
                    } else {
                        t = a.t_in[it.group];
                    }
                    s_t = t;
                }
                __syncthreads();
                const int t = s_t;
                if (t != -2 && n > 0) bin_tile(gvol + off, gmask + off, n, t, a.lo, a.L, a.bin_shift, a.polarity);
            }
        }
        __syncthreads();
    }

    // exit: the last block restores the scratch header for the next launch
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned d = atomicAdd(&a.hdr->done, 1u);
        s_flag = (d == gridDim.x - 1);
    }
    __syncthreads();
    if (s_flag) {
        __threadfence();
        if (*(volatile int*)&a.hdr->err && (a.phases & kPhaseSearch)) {
            // a wait ran out: report it, then clear every group's arrival
            // count and histogram
            for (int g = tid; g < a.ngroups; g += kSegThreads) {
                if (*(volatile int*)&a.tmo[g] == epoch + 1) {
                    a.t_out[g] = -1;
                    a.phi_out[g] = 0.f;
                    a.status[g] = 5; /* TSALLIS_ERR_TIMEOUT */
                }
                a.arrive[g] = 0;
            }
            const long long tot = (long long)a.ngroups * a.L;
            for (long long i = tid; i < tot; i += kSegThreads) a.ghist[i] = 0;
        }
        __syncthreads();
        if (tid == 0) {
            a.hdr->ticket = 0;
            a.hdr->done = 0;
            a.hdr->err = 0;
            a.hdr->epoch = epoch + 1;
            __threadfence();
        }
    }
}

__global__ void __launch_bounds__(kSearchThreads) k_search1d(const int32_t* __restrict__ hist, long long nh, int L,
                                                             float q, int32_t* __restrict__ t_out,
                                                             float* __restrict__ phi_out,
                                                             int32_t* __restrict__ status, float* __restrict__ curve) {
    __shared__ SearchSmem sm;
    for (long long g = blockIdx.x; g < nh; g += gridDim.x) {
        SearchResult r = search1d_block(hist + g * L, L, q, curve ? curve + g * (L - 1) : nullptr, sm);
        if (threadIdx.x == 0) {
            t_out[g] = r.t;
            phi_out[g] = r.phi;
            status[g] = r.status;
        }
        __syncthreads();
    }
}

int segment1d_threads() { return kSegThreads; }
int segment1d_smem_bytes(int L, int copies) { return L * copies * (int)sizeof(int); }

cudaError_t segment1d_occupancy(int copies, int L, int* blocks_per_sm) {
    const int smem = segment1d_smem_bytes(L, copies);
    switch (copies) {
        case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_segment1d<1>, kSegThreads, smem);
        case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_segment1d<2>, kSegThreads, smem);
        case 4: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_segment1d<4>, kSegThreads, smem);
        default: return cudaErrorInvalidValue;
    }
}

template <int C>
static cudaError_t launch_c(const SegArgs& a, int grid, cudaStream_t s) {
    const int smem = segment1d_smem_bytes(a.L, C);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_segment1d<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    k_segment1d<C><<<grid, kSegThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_segment1d(const SegArgs& a, int grid, int copies, cudaStream_t s) {
    switch (copies) {
        case 1: return launch_c<1>(a, grid, s);
        case 2: return launch_c<2>(a, grid, s);
        case 4: return launch_c<4>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_search1d(const int32_t* hist, long long nh, int L, float q, int32_t* t, float* phi,
                            int32_t* status, float* curve, cudaStream_t s) {
    if (nh <= 0) return cudaSuccess;
    const int grid = (int)(nh < 65535 ? nh : 65535);
    k_search1d<<<grid, kSearchThreads, 0, s>>>(hist, nh, L, q, t, phi, status, curve);
    return cudaGetLastError();
}

}  // namespace tsl
