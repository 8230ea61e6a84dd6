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
// The products are small (a batch of at most a few thousand rows against
// 256 x 256 and 4096 x 256 weight matrices), so they run as one tiled
// shared-memory GEMM on the FP32 pipe with bfloat16 operands widened on
// load.
#include <cuda_bf16.h>
#include <cmath>
#include <cstdint>

#include "kernels.h"

namespace tsl {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;
constexpr int kGemmThreads = 256;

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// C[M][N] = sum_k A(m, k) B(k, n), then the epilogue.
//   kAT = 0: A(m, k) = A[m * lda + k];  1: A(m, k) = A[k * lda + m]     (FP32)
//   kBT = 0: B(k, n) = Wb[n * ldb + k]; 1: B(k, n) = Wb[k * ldb + n]   (bfloat16)
//         2: B(k, n) = Bf[k * ldb + n]                                  (FP32)
//   kEpi = 0: C = sum; 1: C = sum + bias[n]; 2: Z = sum + bias[n] and
//         C = GELU(Z); 3: C += sum (accumulate).
template <int kAT, int kBT, int kEpi>
__global__ void __launch_bounds__(kGemmThreads) k_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                                       const __nv_bfloat16* __restrict__ Wb,
                                                       const float* __restrict__ Bf, int ldb,
                                                       const float* __restrict__ bias, float* __restrict__ C,
                                                       float* __restrict__ Z, int ldc) {
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += BK) {
        // A tile: BM x BK, 4 elements per thread
        for (int e = threadIdx.x; e < BM * BK; e += kGemmThreads) {
            int mm, kk;
            if (kAT == 0) { mm = e / BK; kk = e % BK; } else { kk = e / BM; mm = e % BM; }
            const int m = m0 + mm, k = k0 + kk;
            float v = 0.f;
            if (m < M && k < K) v = kAT == 0 ? A[(long long)m * lda + k] : A[(long long)k * lda + m];
            As[kk][mm] = v;
        }
        // B tile: BK x BN
        for (int e = threadIdx.x; e < BK * BN; e += kGemmThreads) {
            int kk, nn;
            if (kBT == 0) { nn = e / BK; kk = e % BK; } else { kk = e / BN; nn = e % BN; }
            const int k = k0 + kk, n = n0 + nn;
            float v = 0.f;
            if (k < K && n < N) {
                if (kBT == 0) v = __bfloat162float(Wb[(long long)n * ldb + k]);
                else if (kBT == 1) v = __bfloat162float(Wb[(long long)k * ldb + n]);
                else v = Bf[(long long)k * ldb + n];
            }
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            const long long o = (long long)m * ldc + n;
            float v = acc[i][j];
            if (kEpi == 1 || kEpi == 2) v += bias[n];
            if (kEpi == 2) {
                Z[o] = v;
                v = gelu_f(v);
            }
            if (kEpi == 3) v += C[o];
            C[o] = v;
        }
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

// Forward layers for small batches (the searches' proposals: a few to 64
// rows per launch): C[m][n] = act(sum_k X[m][k] W[n][k] + bias[n]) with
// K = 256. A block owns 16 outputs of up to 64 rows; thread (m, g) computes
// outputs n0 + 4g .. n0 + 4g + 3 of row m. The rows' inputs are staged in
// shared memory 64 columns at a time with a padded stride (the 32 lanes of a
// warp read 32 rows of one column: distinct banks); the 16 weight rows are
// read as broadcasts. Epilogue as k_gemm's kEpi 1 (bias) and 2 (bias, Z,
// GELU).
constexpr int kSmallRows = 64, kSmallCols = 16, kSmallK = 64;
template <int kEpi>
__global__ void __launch_bounds__(256) k_gemm_small(int M, int N, const float* __restrict__ X,
                                                  const __nv_bfloat16* __restrict__ W,
                                                  const float* __restrict__ bias, float* __restrict__ C,
                                                  float* __restrict__ Z) {
    __shared__ float xs[kSmallRows][kSmallK + 1];
    __shared__ float ws[kSmallCols][kSmallK];
    const int m_local = threadIdx.x & (kSmallRows - 1), g = threadIdx.x >> 6;
    const int m0 = blockIdx.y * kSmallRows, n0 = blockIdx.x * kSmallCols;
    const int m = m0 + m_local;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < kMlpIn; k0 += kSmallK) {
        for (int e = threadIdx.x; e < kSmallRows * kSmallK; e += 256) {
            const int r = e / kSmallK, kk = e % kSmallK;
            xs[r][kk] = (m0 + r < M) ? X[(long long)(m0 + r) * kMlpIn + k0 + kk] : 0.f;
        }
        for (int e = threadIdx.x; e < kSmallCols * kSmallK; e += 256) {
            const int c = e / kSmallK, kk = e % kSmallK;
            ws[c][kk] = (n0 + c < N) ? __bfloat162float(W[(long long)(n0 + c) * kMlpIn + k0 + kk]) : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kSmallK; ++kk) {
            const float xv = xs[m_local][kk];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] = fmaf(xv, ws[g * 4 + j][kk], acc[j]);
        }
        __syncthreads();
    }
    if (m >= M) return;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int n = n0 + g * 4 + j;
        if (n >= N) continue;
        const long long o = (long long)m * N + n;
        float v = acc[j] + bias[n];
        if (kEpi == 2) {
            Z[o] = v;
            v = gelu_f(v);
        }
        C[o] = v;
    }
}

template <int kEpi>
cudaError_t gemm_small(int M, int N, const float* X, const __nv_bfloat16* W, const float* bias, float* C, float* Z,
                       cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    dim3 grid((N + kSmallCols - 1) / kSmallCols, (M + kSmallRows - 1) / kSmallRows);
    k_gemm_small<kEpi><<<grid, 256, 0, s>>>(M, N, X, W, bias, C, Z);
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
__global__ void __launch_bounds__(512) k_topk_small(const float* __restrict__ z, int k, int32_t* __restrict__ out) {
    __shared__ unsigned long long cand[16 * kTopkSmallMax];   // warp w's k keys at [w * k, w * k + k)
    __shared__ unsigned long long fin[kTopkSmallMax];
    const int row = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float* zr = z + (long long)row * kMlpOut;
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
    for (int r = lane; r < k; r += 32)
        out[(long long)row * k + r] = (int32_t)(0xffffffffu - (unsigned)(fin[r] & 0xffffffffu));
}

// x[h][k] = log1p(sum of levels 16k..16k+15) / log1p(N); one block per histogram.
__global__ void __launch_bounds__(kMlpIn) k_features(const int32_t* __restrict__ hist, long long nh,
                                                       float* __restrict__ x) {
    __shared__ long long part[kMlpIn / 32];
    for (long long h = blockIdx.x; h < nh; h += gridDim.x) {
        const int32_t* r = hist + h * kMlpOut + threadIdx.x * kMlpGroup;
        long long s = 0;
#pragma unroll
        for (int j = 0; j < kMlpGroup; ++j) s += r[j];
        long long w = s;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) w += __shfl_xor_sync(0xffffffffu, w, d);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = w;
        __syncthreads();
        long long n = 0;
#pragma unroll
        for (int i = 0; i < kMlpIn / 32; ++i) n += part[i];
        __syncthreads();
        const float den = log1pf((float)n);
        x[h * kMlpIn + threadIdx.x] = n > 0 ? log1pf((float)s) / den : 0.f;
    }
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
__global__ void __launch_bounds__(kMlpIn) k_features2d(const int32_t* __restrict__ hist, long long nh,
                                                         float* __restrict__ x) {
    __shared__ long long part[kMlpIn / 32];
    const int bi = threadIdx.x >> 4, bj = threadIdx.x & 15;
    for (long long h = blockIdx.x; h < nh; h += gridDim.x) {
        const int32_t* r = hist + h * 65536ll + (bi * 16) * 256 + bj * 16;
        long long s = 0;
        for (int i = 0; i < 16; ++i)
#pragma unroll
            for (int j = 0; j < 16; ++j) s += r[i * 256 + j];
        long long w = s;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) w += __shfl_xor_sync(0xffffffffu, w, d);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = w;
        __syncthreads();
        long long n = 0;
#pragma unroll
        for (int i = 0; i < kMlpIn / 32; ++i) n += part[i];
        __syncthreads();
        const float den = log1pf((float)n);
        x[h * kMlpIn + threadIdx.x] = n > 0 ? log1pf((float)s) / den : 0.f;
    }
}

}  // namespace

cudaError_t mlp_features2d(const int32_t* hist, long long nh, float* x, cudaStream_t s) {
    if (nh <= 0) return cudaSuccess;
    k_features2d<<<(int)(nh < 65535 ? nh : 65535), kMlpIn, 0, s>>>(hist, nh, x);
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
    if (B <= kSmallRows) {
        if ((e = gemm_small<2>(B, kMlpHid, x, w + kOffW1, b.p32 + kOffB1, b.a1, b.z1, s)) != cudaSuccess) return e;
        if ((e = gemm_small<2>(B, kMlpHid, b.a1, w + kOffW2, b.p32 + kOffB2, b.a2, b.z2, s)) != cudaSuccess) return e;
        return gemm_small<1>(B, kMlpOut, b.a2, w + kOffW3, b.p32 + kOffB3, b.z3, nullptr, s);
    }
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

}  // namespace tsl
