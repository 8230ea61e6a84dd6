// Learned threshold proposer: a small network that reads a coarse view of
// a 4096-level histogram and ranks thresholds, so that the exact search can
// start from a window of candidates (the search itself, with the bounds that
// make it exact, is in search1d.cuh). The paper has no counterpart; the
// network is defined here:
//   features  x_k = log1p(sum of levels 16k..16k+15) / log1p(N), k < 256;
//   network   z1 = W1 x + b1, a1 = GELU(z1), z2 = W2 a1 + b2, a2 = GELU(z2),
//             z3 = W3 a2 + b3 (4096 logits), GELU(z) = z Phi(z);
//   training  mean soft-target cross-entropy of softmax(z3), Adam.
// Weights are kept in FP32 (the optimiser's copy) and bfloat16 (what the
// forward and backward passes multiply with); every product accumulates in
// FP32. Layout of the flat parameter vector: W1, b1, W2, b2, W3, b3, each
// matrix row-major [out][in].
//
// Every product runs on the tensor cores (mma.sync m16n8k16, bfloat16
// operands, FP32 accumulation). A bfloat16 operand (the weights) enters as
// it is; an FP32 operand (features, activations, gradients) is split into a
// bfloat16 pair hi + lo (hi = rn(v), lo = rn(v - hi), about 16 bits of v)
// and the product is taken as hi*hi + lo*hi, plus hi*lo when both operands
// are FP32; the error against the FP32 product of the same operands stays
// near 2^-16 relative, well inside the tests' tolerances. Training, batches
// above 64 rows and windows of more than 64 proposals use one tiled GEMM
// (k_gemm); inference of up to 64 rows is one cooperative kernel
// (k_mlp_infer): features, the three layers and the top-k, each weight
// matrix read once.
#include <cuda_bf16.h>
#include <cmath>
#include <cstdint>

#include "kernels.h"

namespace tsl {

namespace {

constexpr int BM = 64, BN = 64, BK2 = 32;
constexpr int kGemmThreads = 128;

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// One m16n8k16 product: c += a * b (a: 16 x 16 row-major, b: 16 x 8
// column-major, bfloat16 pairs; c: 16 x 8 FP32). Fragments (lane = 4 g + t):
// a[0] (row g, cols 2t, 2t+1), a[1] (row g + 8), a[2] (row g, cols 2t + 8, +9),
// a[3] (row g + 8, cols 2t + 8, +9); b[0] (rows k = 2t, 2t+1 of col g),
// b[1] (rows 2t + 8, +9); c[0], c[1] (row g, cols 2t, 2t+1), c[2], c[3]
// (row g + 8). The lower half of each pair holds the smaller index.
__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ unsigned bf16x2_bits(__nv_bfloat162 v) { return *reinterpret_cast<unsigned*>(&v); }
// Two FP32 values (x the smaller index) as bfloat16 pairs hi and lo.
__device__ __forceinline__ void split2(float x, float y, unsigned& hi, unsigned& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
    const float2 hf = __bfloat1622float2(h);
    hi = bf16x2_bits(h);
    lo = bf16x2_bits(__floats2bfloat162_rn(x - hf.x, y - hf.y));
}
__device__ __forceinline__ void split1(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// C[M][N] = sum_k A(m, k) B(k, n), then the epilogue.
//   kAT = 0: A(m, k) = A[m * lda + k];  1: A(m, k) = A[k * lda + m]     (FP32)
//   kBT = 0: B(k, n) = Wb[n * ldb + k]; 1: B(k, n) = Wb[k * ldb + n]   (bfloat16)
//         2: B(k, n) = Bf[k * ldb + n]                                  (FP32)
//   kEpi = 0: C = sum; 1: C = sum + bias[n]; 2: Z = sum + bias[n] and
//         C = GELU(Z); 3: C += sum (accumulate).
// A block computes a 64 x 64 tile with 4 warps (32 x 32 each: 2 x 4
// products of 16 x 8), staging 32-deep slices of both operands in shared
// memory as bfloat16 hi (and lo) parts, [row][k] with a padded stride.
constexpr int kTcPad = BK2 + 8;
template <int kAT, int kBT, int kEpi>
__global__ void __launch_bounds__(kGemmThreads) k_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                                       const __nv_bfloat16* __restrict__ Wb,
                                                       const float* __restrict__ Bf, int ldb,
                                                       const float* __restrict__ bias, float* __restrict__ C,
                                                       float* __restrict__ Z, int ldc) {
    constexpr bool kBsplit = kBT == 2;   // B is FP32: its lo part too
    __shared__ __align__(16) __nv_bfloat16 Ahi[BM][kTcPad], Alo[BM][kTcPad];
    __shared__ __align__(16) __nv_bfloat16 Bhi[BN][kTcPad], Blo[kBsplit ? BN : 1][kTcPad];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[2][4][4] = {};
    for (int k0 = 0; k0 < K; k0 += BK2) {
        for (int e = tid; e < BM * BK2; e += kGemmThreads) {
            int mm, kk;
            if (kAT == 0) { mm = e / BK2; kk = e % BK2; } else { kk = e / BM; mm = e % BM; }
            const int m = m0 + mm, k = k0 + kk;
            float v = 0.f;
            if (m < M && k < K) v = kAT == 0 ? A[(long long)m * lda + k] : A[(long long)k * lda + m];
            split1(v, Ahi[mm][kk], Alo[mm][kk]);
        }
        for (int e = tid; e < BK2 * BN; e += kGemmThreads) {
            int kk, nn;
            if (kBT == 0) { nn = e / BK2; kk = e % BK2; } else { kk = e / BN; nn = e % BN; }
            const int k = k0 + kk, n = n0 + nn;
            if (kBsplit) {
                const float v = (k < K && n < N) ? Bf[(long long)k * ldb + n] : 0.f;
                split1(v, Bhi[nn][kk], Blo[nn][kk]);
            } else {
                __nv_bfloat16 v = __float2bfloat16_rn(0.f);
                if (k < K && n < N) v = kBT == 0 ? Wb[(long long)n * ldb + k] : Wb[(long long)k * ldb + n];
                Bhi[nn][kk] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK2; ks += 16) {
            unsigned ah[2][4], al[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r = wm + mt * 16 + g, c = ks + 2 * t;
                ah[mt][0] = *reinterpret_cast<const unsigned*>(&Ahi[r][c]);
                ah[mt][1] = *reinterpret_cast<const unsigned*>(&Ahi[r + 8][c]);
                ah[mt][2] = *reinterpret_cast<const unsigned*>(&Ahi[r][c + 8]);
                ah[mt][3] = *reinterpret_cast<const unsigned*>(&Ahi[r + 8][c + 8]);
                al[mt][0] = *reinterpret_cast<const unsigned*>(&Alo[r][c]);
                al[mt][1] = *reinterpret_cast<const unsigned*>(&Alo[r + 8][c]);
                al[mt][2] = *reinterpret_cast<const unsigned*>(&Alo[r][c + 8]);
                al[mt][3] = *reinterpret_cast<const unsigned*>(&Alo[r + 8][c + 8]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int r = wn + nt * 8 + g, c = ks + 2 * t;
                const unsigned bh[2] = {*reinterpret_cast<const unsigned*>(&Bhi[r][c]),
                                        *reinterpret_cast<const unsigned*>(&Bhi[r][c + 8])};
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma_bf16(acc[mt][nt], ah[mt], bh);
                    mma_bf16(acc[mt][nt], al[mt], bh);
                }
                if (kBsplit) {
                    const unsigned bl[2] = {*reinterpret_cast<const unsigned*>(&Blo[r][c]),
                                            *reinterpret_cast<const unsigned*>(&Blo[r][c + 8])};
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) mma_bf16(acc[mt][nt], ah[mt], bl);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int m = m0 + wm + mt * 16 + g + (i >> 1) * 8;
                const int n = n0 + wn + nt * 8 + 2 * t + (i & 1);
                if (m >= M || n >= N) continue;
                const long long o = (long long)m * ldc + n;
                float v = acc[mt][nt][i];
                if (kEpi == 1 || kEpi == 2) v += bias[n];
                if (kEpi == 2) {
                    Z[o] = v;
                    v = gelu_f(v);
                }
                if (kEpi == 3) v += C[o];
                C[o] = v;
            }
}

template <int kAT, int kBT, int kEpi>
cudaError_t gemm(int M, int N, int K, const float* A, int lda, const __nv_bfloat16* Wb, const float* Bf, int ldb,
                 const float* bias, float* C, float* Z, int ldc, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    k_gemm<kAT, kBT, kEpi><<<grid, kGemmThreads, 0, s>>>(M, N, K, A, lda, Wb, Bf, ldb, bias, C, Z, ldc);
    return cudaGetLastError();
}

// Top k (k <= 64) of one row of 4096 logits per block, as warp argmax
// rounds: each of the 16 warps takes the k largest of its 256 keys (a lane
// holds 8; each round the warp's maximum is found by shuffles and its lane
// moves to its next key), then warp 0 takes the k largest of the 16 k
// candidates the same way. Keys are the order-preserving bits of the logit
// above the complemented index, so equal logits rank the smaller index
// first; the output is in descending order, as the bitonic kernel's.
constexpr int kTopkSmallMax = 64;
__device__ __forceinline__ unsigned long long topk_key(float v, int i) {
    unsigned u = __float_as_uint(v);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (unsigned)(0xffffffffu - (unsigned)i);
}
template <int kPer>
__device__ __forceinline__ void warp_topk_rounds(unsigned long long (&key)[kPer], int k, unsigned long long* out) {
    const int lane = threadIdx.x & 31;
    // each lane's keys in descending order, so its next key is key[pos]
#pragma unroll
    for (int i = 1; i < kPer; ++i)
#pragma unroll
        for (int j = i; j > 0; --j)
            if (key[j] > key[j - 1]) {
                const unsigned long long t = key[j];
                key[j] = key[j - 1];
                key[j - 1] = t;
            }
    int pos = 0;
    for (int r = 0; r < k; ++r) {
        unsigned long long head = 0ull;
#pragma unroll
        for (int i = 0; i < kPer; ++i)
            if (i == pos) head = key[i];
        unsigned long long best = head;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
            best = other > best ? other : best;
        }
        if (head == best && head != 0ull) ++pos;   // keys are distinct: one lane owns the maximum
        if (lane == 0) out[r] = best;
    }
}
// One row by a block of 512 threads (cand: 16 k keys, fin: k keys, in
// shared memory). Warps other than 0 return after the barrier.
__device__ void topk_row_small(const float* __restrict__ zr, int k, int32_t* __restrict__ outr,
                               unsigned long long* cand, unsigned long long* fin) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long key[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int i = warp * 256 + j * 32 + lane;
        key[j] = topk_key(zr[i], i);
    }
    warp_topk_rounds<8>(key, k, cand + warp * k);
    __syncthreads();
    if (warp != 0) return;
    // warp 0 merges the 16 k candidates in shared memory: lane l owns
    // candidates l, l + 32, ... and caches the largest it still holds; each
    // round takes the warp's maximum, and only the lane that held it (keys
    // are distinct) clears that candidate and looks for its next largest
    const int nc = 16 * k;
    auto rescan = [&](int& bi) {
        unsigned long long b = 0ull;
        bi = -1;
        for (int c = lane; c < nc; c += 32)
            if (cand[c] > b) { b = cand[c]; bi = c; }
        return b;
    };
    int bi;
    unsigned long long mine = rescan(bi);
    for (int r = 0; r < k; ++r) {
        unsigned long long best = mine;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
            best = other > best ? other : best;
        }
        if (lane == 0) fin[r] = best;
        if (mine == best && mine != 0ull) {
            cand[bi] = 0ull;
            mine = rescan(bi);
        }
        __syncwarp();
    }
    for (int r = lane; r < k; r += 32) outr[r] = (int32_t)(0xffffffffu - (unsigned)(fin[r] & 0xffffffffu));
}
__global__ void __launch_bounds__(512) k_topk_small(const float* __restrict__ z, int k, int32_t* __restrict__ out) {
    __shared__ unsigned long long cand[16 * kTopkSmallMax];   // warp w's k keys at [w * k, w * k + k)
    __shared__ unsigned long long fin[kTopkSmallMax];
    topk_row_small(z + (long long)blockIdx.x * kMlpOut, k, out + (long long)blockIdx.x * k, cand, fin);
}

// x[k] = log1p(sum of levels 16k..16k+15) / log1p(N) of one histogram, by
// the first 256 threads of the block (all threads reach the barriers).
__device__ void features_row(const int32_t* __restrict__ hrow, float* __restrict__ xrow, long long* part) {
    const bool on = threadIdx.x < kMlpIn;
    long long s = 0;
    if (on) {
        const int32_t* r = hrow + threadIdx.x * kMlpGroup;
#pragma unroll
        for (int j = 0; j < kMlpGroup; ++j) s += r[j];
    }
    long long w = s;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) w += __shfl_xor_sync(0xffffffffu, w, d);
    if (on && (threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = w;
    __syncthreads();
    long long n = 0;
#pragma unroll
    for (int i = 0; i < kMlpIn / 32; ++i) n += part[i];
    __syncthreads();
    const float den = log1pf((float)n);
    if (on) xrow[threadIdx.x] = n > 0 ? log1pf((float)s) / den : 0.f;
}

// x[h][k] for nh histograms; one block per histogram.
__global__ void __launch_bounds__(kMlpIn) k_features(const int32_t* __restrict__ hist, long long nh,
                                                       float* __restrict__ x) {
    __shared__ long long part[kMlpIn / 32];
    for (long long h = blockIdx.x; h < nh; h += gridDim.x) features_row(hist + h * kMlpOut, x + h * kMlpIn, part);
}

// Softmax cross-entropy against soft targets, one block per row: adds the
// row's loss / B to *loss and writes dL/dz = (softmax - y) / B.
__global__ void __launch_bounds__(256) k_softmax_ce(const float* __restrict__ z, const float* __restrict__ y, int B,
                                                    float* __restrict__ dz, float* __restrict__ loss) {
    __shared__ float red[8];
    const int row = blockIdx.x;
    const float* zr = z + (long long)row * kMlpOut;
    const float* yr = y + (long long)row * kMlpOut;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float m = -INFINITY;
    for (int i = threadIdx.x; i < kMlpOut; i += 256) m = fmaxf(m, zr[i]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
    if (lane == 0) red[warp] = m;
    __syncthreads();
    m = red[0];
#pragma unroll
    for (int i = 1; i < 8; ++i) m = fmaxf(m, red[i]);
    __syncthreads();
    float s = 0.f;
    for (int i = threadIdx.x; i < kMlpOut; i += 256) s += expf(zr[i] - m);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += red[i];
    __syncthreads();
    const float lse = m + logf(s);
    float l = 0.f;
    for (int i = threadIdx.x; i < kMlpOut; i += 256) {
        const float lp = zr[i] - lse;
        l -= yr[i] * lp;
        dz[(long long)row * kMlpOut + i] = (expf(lp) - yr[i]) / (float)B;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) l += __shfl_xor_sync(0xffffffffu, l, d);
    if (lane == 0) red[warp] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < 8; ++i) t += red[i];
        atomicAdd(loss, t / (float)B);
    }
}

// db[n] = sum over rows of d[r][n].
__global__ void k_colsum(const float* __restrict__ d, int rows, int n, float* __restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += d[(long long)r * n + c];
    db[c] = s;
}

// dz = da * GELU'(z), elementwise.
__global__ void k_gelu_bwd(const float* __restrict__ da, const float* __restrict__ z, float* __restrict__ dz,
                           long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dz[i] = da[i] * gelu_grad_f(z[i]);
}

// Adam with bias correction (c1 = 1 - beta1^t, c2 = 1 - beta2^t), then the
// bfloat16 copy.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ p16, long long n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        p16[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ p16, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p16[i] = __float2bfloat16_rn(p[i]);
}

// The k largest logits of each row (ties: the smaller level first), by a
// bitonic sort of (value, level) keys in shared memory; one block per row.
__global__ void __launch_bounds__(512) k_topk(const float* __restrict__ z, int k, int32_t* __restrict__ out) {
    __shared__ unsigned long long key[kMlpOut];
    const int row = blockIdx.x;
    for (int i = threadIdx.x; i < kMlpOut; i += 512) {
        unsigned u = __float_as_uint(z[(long long)row * kMlpOut + i]);
        u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);   // order-preserving
        key[i] = ((unsigned long long)u << 32) | (unsigned)(0xffffffffu - (unsigned)i);
    }
    __syncthreads();
    for (int size = 2; size <= kMlpOut; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < kMlpOut / 2; i += 512) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool desc = ((lo & size) == 0);
                const unsigned long long a = key[lo], b = key[hi];
                if ((a < b) == desc) { key[lo] = b; key[hi] = a; }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < k; i += 512)
        out[(long long)row * k + i] = (int32_t)(0xffffffffu - (unsigned)(key[i] & 0xffffffffu));
}

// 2-D form: x_f = log1p(count of the 16 x 16 block f of the 256 x 256
// grey x mean histogram) / log1p(N), f = 16 * (grey block) + mean block.
// Warp w takes the grey blocks w and w + 8: its lanes read each histogram
// row as 16-byte words (lane l: columns 8l .. 8l + 7, half of mean block
// l / 2), eight rows of loads in flight, and lane pairs combine their halves.
// kVec false: the same with 4-byte loads, for histograms not on a 16-byte
// boundary.
template <bool kVec>
__global__ void __launch_bounds__(kMlpIn) k_features2d(const int32_t* __restrict__ hist, long long nh,
                                                         float* __restrict__ x) {
    __shared__ long long part[kMlpIn / 32];
    __shared__ long long blk[256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (long long h = blockIdx.x; h < nh; h += gridDim.x) {
        long long tot = 0;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int bi = warp + 8 * q;
            const int32_t* r = hist + h * 65536ll + (bi * 16) * 256 + 8 * lane;
            long long s = 0;
#pragma unroll
            for (int i0 = 0; i0 < 16; i0 += 8) {
                int4 v[8][2];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int32_t* e = r + (i0 + i) * 256;
                    if constexpr (kVec) {
                        v[i][0] = __ldg(reinterpret_cast<const int4*>(e));
                        v[i][1] = __ldg(reinterpret_cast<const int4*>(e) + 1);
                    } else {
                        v[i][0] = make_int4(__ldg(e), __ldg(e + 1), __ldg(e + 2), __ldg(e + 3));
                        v[i][1] = make_int4(__ldg(e + 4), __ldg(e + 5), __ldg(e + 6), __ldg(e + 7));
                    }
                }
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    s += (long long)v[i][0].x + v[i][0].y + v[i][0].z + v[i][0].w + v[i][1].x + v[i][1].y + v[i][1].z +
                         v[i][1].w;
            }
            s += __shfl_xor_sync(0xffffffffu, s, 1);   // the two halves of mean block lane / 2
            if ((lane & 1) == 0) blk[bi * 16 + (lane >> 1)] = s;
            tot += s;
        }
        // each block's count appears twice in tot (both lanes of a pair)
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, d);
        if (lane == 0) part[warp] = tot / 2;
        __syncthreads();
        long long n = 0;
#pragma unroll
        for (int i = 0; i < kMlpIn / 32; ++i) n += part[i];
        const long long c = blk[threadIdx.x];
        __syncthreads();
        const float den = log1pf((float)n);
        x[h * kMlpIn + threadIdx.x] = n > 0 ? log1pf((float)c) / den : 0.f;
    }
}

// ------------------------------------------------------------ fused inference
//
// Up to 64 rows in one cooperative launch of kInferBlocks blocks of 512
// threads, in phases separated by bounded grid barriers:
//   0. (histograms given) the features of row b, by block b;
//   1. a1 = GELU(W1 x + b1): block b < 32 owns outputs 8b .. 8b + 7, its warp
//      w < 4 the rows 16w .. 16w + 15;
//   2. a2 = GELU(W2 a1 + b2), the same way;
//   3. z3 = W3 a2 + b3: block b owns outputs 64b .. 64b + 63, its warp w the
//      outputs 64b + 8 (w mod 8) .. + 7 of rows 16 (w / 8) + 32 q;
// the layer's input rows are staged in shared memory as bfloat16 hi and lo
// parts, and each warp loads all of its weight fragments before its first
// product (so the layer costs one memory latency, not one per k step);
//   4. (k > 0) the top k of row b, by block b.
// Each weight matrix is read from memory once. A barrier that runs out of
// time sets the error word and the kernel runs on: the outputs are then
// meaningless, but every candidate is still a valid level, which is all the
// window searches that use them need (their result is certified exact).
constexpr int kInferBlocks = 64, kInferThreads = 512, kInferRows = 64;
constexpr int kInferPad = kMlpHid + 8;   // shared-memory row stride of the staged activations (bfloat16)
constexpr int kInferSmem = 2 * kInferRows * kInferPad * 2;

struct InferArgs {
    const int32_t* hist;       // [B][4096], or null: x is given
    const float* x;            // [B][256] features (written by phase 0 when hist is given)
    float* xw;
    const __nv_bfloat16* w;    // parameters, bfloat16 (matrices)
    const float* p32;          // parameters, FP32 (biases)
    float* a1;                 // [B][256]
    float* a2;                 // [B][256]
    float* z3;                 // [B][4096] logits
    int B, k;
    int32_t* cand;             // [B][k]
    unsigned* sync;            // [0] barrier arrivals, [1] blocks done, [2] error
    unsigned long long timeout_ns;
};

__device__ __forceinline__ unsigned long long infer_clock() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier number `phase` (1, 2, ...): every block arrives once.
__device__ void infer_barrier(const InferArgs& a, unsigned phase) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&a.sync[0], 1u);
        const unsigned target = phase * gridDim.x;
        const unsigned long long t0 = infer_clock();
        for (unsigned spin = 0;; ++spin) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&a.sync[0]) : "memory");
            if (v >= target) break;
            // every 64 polls: the error word and the clock
            if ((spin & 63u) == 63u) {
                if (*(volatile unsigned*)&a.sync[2]) break;
                if (infer_clock() - t0 > a.timeout_ns) {
                    atomicExch(&a.sync[2], 1u);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Rows 0 .. B-1 of an FP32 [B][256] matrix into shared memory as bfloat16
// hi and lo parts (stride kInferPad; rows B .. 63 zero), by the whole block.
__device__ void infer_stage(const float* __restrict__ src, int B, __nv_bfloat16* Shi, __nv_bfloat16* Slo) {
    constexpr int kPer = kInferRows * (kMlpHid / 2) / kInferThreads;   // 16 pairs a thread, all loads in flight
    float2 v[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int e = threadIdx.x + j * kInferThreads;
        const int r = e / (kMlpHid / 2), c2 = (e % (kMlpHid / 2)) * 2;
        v[j] = r < B ? __ldcg(reinterpret_cast<const float2*>(src + (long long)r * kMlpHid + c2)) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int e = threadIdx.x + j * kInferThreads;
        const int r = e / (kMlpHid / 2), c2 = (e % (kMlpHid / 2)) * 2;
        unsigned hi, lo;
        split2(v[j].x, v[j].y, hi, lo);
        *reinterpret_cast<unsigned*>(Shi + r * kInferPad + c2) = hi;
        *reinterpret_cast<unsigned*>(Slo + r * kInferPad + c2) = lo;
    }
    __syncthreads();
}

// One warp: the 8 outputs n0 .. n0 + 7 of (W a)(rows 16 mt + 32 q, q < nq)
// with the staged rows of a, W bfloat16 [N][256] in global memory. Every
// weight fragment of the warp is loaded before the first product.
template <int kQ>
__device__ __forceinline__ void infer_tile(const __nv_bfloat16* __restrict__ W, int n0, int mt,
                                           const __nv_bfloat16* Shi, const __nv_bfloat16* Slo, float (&acc)[kQ][4],
                                           int nq) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const __nv_bfloat16* wr = W + (long long)(n0 + g) * kMlpHid + 2 * t;
    unsigned bw[kMlpHid / 16][2];
#pragma unroll
    for (int k = 0; k < kMlpHid / 16; ++k) {
        bw[k][0] = __ldg(reinterpret_cast<const unsigned*>(wr + 16 * k));
        bw[k][1] = __ldg(reinterpret_cast<const unsigned*>(wr + 16 * k + 8));
    }
#pragma unroll
    for (int q = 0; q < kQ; ++q)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[q][i] = 0.f;
#pragma unroll
    for (int k = 0; k < kMlpHid / 16; ++k) {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            if (q >= nq) break;
            const int r = 16 * mt + 32 * q + g, c = 16 * k + 2 * t;
            const unsigned ah[4] = {*reinterpret_cast<const unsigned*>(Shi + r * kInferPad + c),
                                    *reinterpret_cast<const unsigned*>(Shi + (r + 8) * kInferPad + c),
                                    *reinterpret_cast<const unsigned*>(Shi + r * kInferPad + c + 8),
                                    *reinterpret_cast<const unsigned*>(Shi + (r + 8) * kInferPad + c + 8)};
            const unsigned al[4] = {*reinterpret_cast<const unsigned*>(Slo + r * kInferPad + c),
                                    *reinterpret_cast<const unsigned*>(Slo + (r + 8) * kInferPad + c),
                                    *reinterpret_cast<const unsigned*>(Slo + r * kInferPad + c + 8),
                                    *reinterpret_cast<const unsigned*>(Slo + (r + 8) * kInferPad + c + 8)};
            mma_bf16(acc[q], ah, bw[k]);
            mma_bf16(acc[q], al, bw[k]);
        }
    }
}

__global__ void __launch_bounds__(kInferThreads) k_mlp_infer(const InferArgs a) {
    extern __shared__ __align__(16) unsigned char infer_smem[];
    __nv_bfloat16* Shi = reinterpret_cast<__nv_bfloat16*>(infer_smem);
    __nv_bfloat16* Slo = Shi + kInferRows * kInferPad;
    __shared__ long long part[kMlpIn / 32];
    __shared__ unsigned long long cand[16 * kTopkSmallMax];
    __shared__ unsigned long long fin[kTopkSmallMax];
    const int b = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int B = a.B;
    unsigned phase = 0;
    const float* x = a.x;
    if (a.hist) {
        if (b < B) features_row(a.hist + (long long)b * kMlpOut, a.xw + (long long)b * kMlpIn, part);
        infer_barrier(a, ++phase);
        x = a.xw;
    }
    // layers 1 and 2: block b < 32 owns outputs 8b .. 8b + 7; warp w < 4 the
    // rows 16w .. 16w + 15
    const bool hid = b < kMlpHid / 8;
    for (int layer = 0; layer < 2; ++layer) {
        const float* in = layer == 0 ? x : a.a1;
        float* out = layer == 0 ? a.a1 : a.a2;
        if (hid) infer_stage(in, B, Shi, Slo);
        if (hid && warp < 4 && warp * 16 < B) {
            float acc[1][4];
            infer_tile<1>(a.w + (layer == 0 ? kOffW1 : kOffW2), 8 * b, warp, Shi, Slo, acc, 1);
            const float* bias = a.p32 + (layer == 0 ? kOffB1 : kOffB2);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int row = 16 * warp + g + (i >> 1) * 8, n = 8 * b + 2 * t + (i & 1);
                if (row < B) out[(long long)row * kMlpHid + n] = gelu_f(acc[0][i] + bias[n]);
            }
        }
        infer_barrier(a, ++phase);
    }
    // layer 3: block b owns outputs 64b .. 64b + 63; warp w the outputs
    // 64b + 8 (w mod 8) .. + 7 of rows 16 (w / 8) + 32 q (q = 0, 1)
    infer_stage(a.a2, B, Shi, Slo);
    {
        const int n0 = 64 * b + 8 * (warp & 7), mt = warp >> 3;
        const int nq = B > 16 * mt ? ((B - 16 * mt + 31) / 32 < 2 ? (B - 16 * mt + 31) / 32 : 2) : 0;
        if (nq > 0) {
            float acc[2][4];
            infer_tile<2>(a.w + kOffW3, n0, mt, Shi, Slo, acc, nq);
            const float* b3 = a.p32 + kOffB3;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (q >= nq) break;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int row = 16 * mt + 32 * q + g + (i >> 1) * 8, n = n0 + 2 * t + (i & 1);
                    if (row < B) a.z3[(long long)row * kMlpOut + n] = acc[q][i] + b3[n];
                }
            }
        }
    }
    // the top k of each row
    if (a.k > 0) {
        infer_barrier(a, ++phase);
        if (b < B) topk_row_small(a.z3 + (long long)b * kMlpOut, a.k, a.cand + (long long)b * a.k, cand, fin);
    }
    // exit: the last block resets the barrier words for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&a.sync[1], 1u) == gridDim.x - 1) {
            a.sync[0] = 0u;
            a.sync[1] = 0u;
            a.sync[2] = 0u;
            __threadfence();
        }
    }
}

}  // namespace

cudaError_t mlp_features2d(const int32_t* hist, long long nh, float* x, cudaStream_t s) {
    if (nh <= 0) return cudaSuccess;
    const int grid = (int)(nh < 65535 ? nh : 65535);
    if (reinterpret_cast<uintptr_t>(hist) % 16 == 0)
        k_features2d<true><<<grid, kMlpIn, 0, s>>>(hist, nh, x);
    else
        k_features2d<false><<<grid, kMlpIn, 0, s>>>(hist, nh, x);
    return cudaGetLastError();
}

cudaError_t mlp_features(const int32_t* hist, long long nh, float* x, cudaStream_t s) {
    if (nh <= 0) return cudaSuccess;
    k_features<<<(int)(nh < 65535 ? nh : 65535), kMlpIn, 0, s>>>(hist, nh, x);
    return cudaGetLastError();
}

cudaError_t mlp_to_bf16(const float* p, void* p16, long long n, cudaStream_t s) {
    k_to_bf16<<<1024, 256, 0, s>>>(p, static_cast<__nv_bfloat16*>(p16), n);
    return cudaGetLastError();
}

cudaError_t mlp_forward(const MlpBuffers& b, const float* x, int B, cudaStream_t s) {
    const __nv_bfloat16* w = static_cast<const __nv_bfloat16*>(b.p16);
    cudaError_t e;
    if ((e = gemm<0, 0, 2>(B, kMlpHid, kMlpIn, x, kMlpIn, w + kOffW1, nullptr, kMlpIn, b.p32 + kOffB1, b.a1, b.z1,
                           kMlpHid, s)) != cudaSuccess) return e;
    if ((e = gemm<0, 0, 2>(B, kMlpHid, kMlpHid, b.a1, kMlpHid, w + kOffW2, nullptr, kMlpHid, b.p32 + kOffB2, b.a2,
                           b.z2, kMlpHid, s)) != cudaSuccess) return e;
    return gemm<0, 0, 1>(B, kMlpOut, kMlpHid, b.a2, kMlpHid, w + kOffW3, nullptr, kMlpHid, b.p32 + kOffB3, b.z3,
                         nullptr, kMlpOut, s);
}

cudaError_t mlp_backward(const MlpBuffers& b, const float* x, const float* y, int B, float* loss, cudaStream_t s) {
    const __nv_bfloat16* w = static_cast<const __nv_bfloat16*>(b.p16);
    float* g = b.grad;
    cudaError_t e;
    if ((e = cudaMemsetAsync(loss, 0, sizeof(float), s)) != cudaSuccess) return e;
    k_softmax_ce<<<B, 256, 0, s>>>(b.z3, y, B, b.d3, loss);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // layer 3
    if ((e = gemm<1, 2, 0>(kMlpOut, kMlpHid, B, b.d3, kMlpOut, nullptr, b.a2, kMlpHid, nullptr, g + kOffW3, nullptr,
                           kMlpHid, s)) != cudaSuccess) return e;
    k_colsum<<<(kMlpOut + 255) / 256, 256, 0, s>>>(b.d3, B, kMlpOut, g + kOffB3);
    if ((e = gemm<0, 1, 0>(B, kMlpHid, kMlpOut, b.d3, kMlpOut, w + kOffW3, nullptr, kMlpHid, nullptr, b.da, nullptr,
                           kMlpHid, s)) != cudaSuccess) return e;
    const long long nh = (long long)B * kMlpHid;
    k_gelu_bwd<<<256, 256, 0, s>>>(b.da, b.z2, b.dz, nh);
    // layer 2
    if ((e = gemm<1, 2, 0>(kMlpHid, kMlpHid, B, b.dz, kMlpHid, nullptr, b.a1, kMlpHid, nullptr, g + kOffW2, nullptr,
                           kMlpHid, s)) != cudaSuccess) return e;
    k_colsum<<<1, 256, 0, s>>>(b.dz, B, kMlpHid, g + kOffB2);
    if ((e = gemm<0, 1, 0>(B, kMlpHid, kMlpHid, b.dz, kMlpHid, w + kOffW2, nullptr, kMlpHid, nullptr, b.da, nullptr,
                           kMlpHid, s)) != cudaSuccess) return e;
    k_gelu_bwd<<<256, 256, 0, s>>>(b.da, b.z1, b.dz, nh);
    // layer 1
    if ((e = gemm<1, 2, 0>(kMlpHid, kMlpIn, B, b.dz, kMlpHid, nullptr, x, kMlpIn, nullptr, g + kOffW1, nullptr,
                           kMlpIn, s)) != cudaSuccess) return e;
    k_colsum<<<1, 256, 0, s>>>(b.dz, B, kMlpHid, g + kOffB1);
    return cudaGetLastError();
}

cudaError_t mlp_adam(const MlpBuffers& b, float lr, int step, cudaStream_t s) {
    const double b1 = 0.9, b2 = 0.999;
    k_adam<<<1024, 256, 0, s>>>(b.p32, b.grad, b.m, b.v, static_cast<__nv_bfloat16*>(b.p16), kMlpParams, lr,
                                (float)b1, (float)b2, 1e-8f, (float)(1.0 - std::pow(b1, step)),
                                (float)(1.0 - std::pow(b2, step)));
    return cudaGetLastError();
}

cudaError_t mlp_topk(const float* z, int B, int k, int32_t* out, cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    if (k >= 1 && k <= kTopkSmallMax) k_topk_small<<<B, 512, 0, s>>>(z, k, out);
    else k_topk<<<B, 512, 0, s>>>(z, k, out);
    return cudaGetLastError();
}

cudaError_t mlp_prepare() {
    return cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, kInferSmem);
}

cudaError_t mlp_infer(const MlpBuffers& b, const int32_t* hist, const float* x, float* xw, int B, int k,
                      int32_t* cand, unsigned* sync, unsigned long long timeout_ns, cudaStream_t s) {
    if (B < 1 || B > kInferRows || k < 0 || k > kTopkSmallMax || (!hist && !x) || (hist && !xw) || (k > 0 && !cand))
        return cudaErrorInvalidValue;
    InferArgs a;
    a.hist = hist;
    a.x = x;
    a.xw = xw;
    a.w = static_cast<const __nv_bfloat16*>(b.p16);
    a.p32 = b.p32;
    a.a1 = b.a1;
    a.a2 = b.a2;
    a.z3 = b.z3;
    a.B = B;
    a.k = k;
    a.cand = cand;
    a.sync = sync;
    a.timeout_ns = timeout_ns;
    // cooperative: the grid barriers need every block resident
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kInferBlocks);
    cfg.blockDim = dim3(kInferThreads);
    cfg.dynamicSmemBytes = kInferSmem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_mlp_infer, a);
}

}  // namespace tsl
