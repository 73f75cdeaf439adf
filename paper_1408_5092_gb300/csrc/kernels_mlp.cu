// Kernels of the learned block preconditioner's network: a 3-layer
// perceptron with bfloat16 weights (float32 master copies) and float32
// accumulation, trained with mean-squared error and Adam.
//
// One tiled GEMM kernel covers every product of training and inference:
//   C[m][n] = sum_k opA(m, k) * opB(k, n)  (+ bias[n]) (relu / relu-mask)
// with A, B float32 or bfloat16 and optional transposes.
#include <cuda_bf16.h>

#include "kernels.h"

namespace mpspt {
namespace {

constexpr int MT = 64, NTL = 64, KT = 16;

template <class TB>
__device__ __forceinline__ float ld(const TB* p, size_t i);
template <>
__device__ __forceinline__ float ld<float>(const float* p, size_t i) { return p[i]; }
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p, size_t i) {
    return __bfloat162float(p[i]);
}

// epi: 0 plain, 1 + bias, 2 + bias then relu, 3 multiply by (mask > 0)
template <class TB>
__global__ void __launch_bounds__(256) k_mlp_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                                  int ta, const TB* __restrict__ B, int ldb, int tb,
                                                  float* __restrict__ C, int ldc, const float* __restrict__ bias,
                                                  const float* __restrict__ mask, int epi) {
    __shared__ float As[KT][MT + 1];
    __shared__ float Bs[KT][NTL + 1];
    const int r0 = blockIdx.y * MT, c0 = blockIdx.x * NTL;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += KT) {
        for (int e = threadIdx.x; e < MT * KT; e += 256) {
            int i, kk;
            if (ta) { i = e % MT; kk = e / MT; } else { kk = e % KT; i = e / KT; }
            const int r = r0 + i, k = k0 + kk;
            float v = 0.f;
            if (r < M && k < K) v = ta ? A[(size_t)k * lda + r] : A[(size_t)r * lda + k];
            As[kk][i] = v;
        }
        for (int e = threadIdx.x; e < NTL * KT; e += 256) {
            int j, kk;
            if (tb) { kk = e % KT; j = e / KT; } else { j = e % NTL; kk = e / NTL; }
            const int c = c0 + j, k = k0 + kk;
            float v = 0.f;
            if (c < N && k < K) v = tb ? ld(B, (size_t)c * ldb + k) : ld(B, (size_t)k * ldb + c);
            Bs[kk][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty + 16 * i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + tx + 16 * j;
            if (c >= N) continue;
            float v = acc[i][j];
            if (epi == 1 || epi == 2) v += bias[c];
            if (epi == 2) v = fmaxf(v, 0.f);
            if (epi == 3) v = mask[(size_t)r * ldc + c] > 0.f ? v : 0.f;
            C[(size_t)r * ldc + c] = v;
        }
    }
}

// column sums: out[n] = sum_m A[m][n]
__global__ void k_colsum(int M, int N, const float* __restrict__ A, float* __restrict__ out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += A[(size_t)m * N + n];
    out[n] = s;
}

// dY = (Y - T) / B and the loss terms 0.5 |Y - T|^2 / B (per row)
__global__ void k_mse(int B, int N, const float* __restrict__ Y, const float* __restrict__ T,
                      float* __restrict__ dY, float* __restrict__ rowloss) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float l = 0.f;
    for (int n = 0; n < N; ++n) {
        const float d = Y[(size_t)b * N + n] - T[(size_t)b * N + n];
        dY[(size_t)b * N + n] = d / (float)B;
        l += 0.5f * d * d / (float)B;
    }
    rowloss[b] = l;
}

__global__ void k_adam(int n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ wb, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(int n, const float* __restrict__ w, __nv_bfloat16* __restrict__ wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

}  // namespace

void mlp_gemm(int M, int N, int K, const float* A, int lda, bool ta, const float* B, int ldb, bool tb,
              float* C, int ldc, const float* bias, const float* mask, int epi, cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    dim3 g((N + NTL - 1) / NTL, (M + MT - 1) / MT);
    count_launch();
    k_mlp_gemm<float><<<g, 256, 0, st>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, bias, mask, epi);
}

void mlp_gemm_bf16w(int M, int N, int K, const float* A, int lda, bool ta, const void* B, int ldb, bool tb,
                    float* C, int ldc, const float* bias, const float* mask, int epi, cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    dim3 g((N + NTL - 1) / NTL, (M + MT - 1) / MT);
    count_launch();
    k_mlp_gemm<__nv_bfloat16><<<g, 256, 0, st>>>(M, N, K, A, lda, ta, static_cast<const __nv_bfloat16*>(B), ldb,
                                                  tb, C, ldc, bias, mask, epi);
}

void mlp_colsum(int M, int N, const float* A, float* out, cudaStream_t st) {
    if (N <= 0) return;
    count_launch();
    k_colsum<<<(N + 127) / 128, 128, 0, st>>>(M, N, A, out);
}

void mlp_mse(int B, int N, const float* Y, const float* T, float* dY, float* rowloss, cudaStream_t st) {
    if (B <= 0) return;
    count_launch();
    k_mse<<<(B + 127) / 128, 128, 0, st>>>(B, N, Y, T, dY, rowloss);
}

void mlp_adam(int n, float* w, const float* g, float* m, float* v, void* wb, float lr, int step, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    count_launch();
    k_adam<<<(n + 255) / 256, 256, 0, st>>>(n, w, g, m, v, static_cast<__nv_bfloat16*>(wb), lr, b1, b2, 1e-8f,
                                            c1, c2);
}

void mlp_to_bf16(int n, const float* w, void* wb, cudaStream_t st) {
    count_launch();
    k_to_bf16<<<(n + 255) / 256, 256, 0, st>>>(n, w, static_cast<__nv_bfloat16*>(wb));
}

}  // namespace mpspt

// ----------------------------------------------------------------------
// Per-block features and initial-guess assembly of the learned
// preconditioner.  A block is one dense QN block of the two-site vector.
namespace mpspt {
namespace {

constexpr int NF = 16;   // features per block

__device__ double block_reduce_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    __syncthreads();
    return s;   // valid in thread 0
}

__device__ double block_reduce_min(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 1e300;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = fmin(s, sh[w]);
    __syncthreads();
    return s;
}

// feats[b][0..NF): statistics of diag(A), |g|, |x_warm| on block b plus the
// block's QN metadata meta[b][0..8) (already scaled by the host).
__global__ void k_block_features(const BlockRef* __restrict__ blocks, const double* __restrict__ diag,
                                 const double* __restrict__ g, const double* __restrict__ xw,
                                 const float* __restrict__ meta, float* __restrict__ feats) {
    __shared__ double sh[32];
    const BlockRef B = blocks[blockIdx.x];
    double s = 0, s2 = 0, mn = 1e300, mx = -1e300, gg = 0, xx = 0, gx = 0;
    for (int e = threadIdx.x; e < B.len; e += blockDim.x) {
        const double d = diag[B.off + e];
        s += d; s2 += d * d; mn = fmin(mn, d); mx = fmax(mx, d);
        const double gv = g[B.off + e], xv = xw[B.off + e];
        gg += gv * gv; xx += xv * xv; gx += gv * xv;
    }
    const double S = block_reduce_sum(s, sh), S2 = block_reduce_sum(s2, sh);
    const double MN = block_reduce_min(mn, sh), MX = -block_reduce_min(-mx, sh);
    const double GG = block_reduce_sum(gg, sh), XX = block_reduce_sum(xx, sh), GX = block_reduce_sum(gx, sh);
    if (threadIdx.x == 0) {
        float* f = feats + (size_t)blockIdx.x * NF;
        const double mean = S / B.len;
        const double var = fmax(S2 / B.len - mean * mean, 0.0);
        f[0] = (float)log10(fmax(mean, 1e-12));
        f[1] = (float)log10(fmax(MN, 1e-12));
        f[2] = (float)log10(fmax(MX, 1e-12));
        f[3] = (float)(sqrt(var) / fmax(fabs(mean), 1e-12));
        f[4] = (float)log10(sqrt(GG) + 1e-30);
        f[5] = (float)log10(sqrt(XX) + 1e-30);
        f[6] = (float)(GX / (sqrt(GG * XX) + 1e-300));
        f[7] = (float)log10(sqrt(GG) / (mean + 1e-12) + 1e-30);   // |P g| scale
        for (int q = 0; q < 8; ++q) f[8 + q] = meta[(size_t)blockIdx.x * 8 + q];
    }
}

// x0 = coef[b][0] * xw + coef[b][1] * (minv .* bvec) on block b
__global__ void k_block_combine(const BlockRef* __restrict__ blocks, const float* __restrict__ coef,
                                const double* __restrict__ xw, const double* __restrict__ minv,
                                const double* __restrict__ bvec, double* __restrict__ x0) {
    const BlockRef B = blocks[blockIdx.x];
    const double ga = coef[(size_t)blockIdx.x * 2], de = coef[(size_t)blockIdx.x * 2 + 1];
    for (int e = threadIdx.x; e < B.len; e += blockDim.x) {
        const size_t i = B.off + e;
        x0[i] = ga * xw[i] + de * minv[i] * bvec[i];
    }
}

// least-squares fit data per block: <w,w>, <w,p>, <p,p>, <w,x>, <p,x>
// with w = xw, p = minv .* bvec
__global__ void k_block_fit(const BlockRef* __restrict__ blocks, const double* __restrict__ xw,
                            const double* __restrict__ minv, const double* __restrict__ bvec,
                            const double* __restrict__ x, double* __restrict__ out) {
    __shared__ double sh[32];
    const BlockRef B = blocks[blockIdx.x];
    double ww = 0, wp = 0, pp = 0, wx = 0, px = 0;
    for (int e = threadIdx.x; e < B.len; e += blockDim.x) {
        const size_t i = B.off + e;
        const double w = xw[i], p = minv[i] * bvec[i], xv = x[i];
        ww += w * w; wp += w * p; pp += p * p; wx += w * xv; px += p * xv;
    }
    const double a = block_reduce_sum(ww, sh), b = block_reduce_sum(wp, sh), c = block_reduce_sum(pp, sh);
    const double d = block_reduce_sum(wx, sh), e2 = block_reduce_sum(px, sh);
    if (threadIdx.x == 0) {
        double* o = out + (size_t)blockIdx.x * 5;
        o[0] = a; o[1] = b; o[2] = c; o[3] = d; o[4] = e2;
    }
}

}  // namespace

void block_features(const BlockRef* blocks, int nb, const double* diag, const double* g, const double* xw,
                    const float* meta, float* feats, cudaStream_t st) {
    if (nb <= 0) return;
    count_launch();
    k_block_features<<<nb, 256, 0, st>>>(blocks, diag, g, xw, meta, feats);
}

void block_combine(const BlockRef* blocks, int nb, const float* coef, const double* xw, const double* minv,
                   const double* bvec, double* x0, cudaStream_t st) {
    if (nb <= 0) return;
    count_launch();
    k_block_combine<<<nb, 256, 0, st>>>(blocks, coef, xw, minv, bvec, x0);
}

void block_fit(const BlockRef* blocks, int nb, const double* xw, const double* minv, const double* bvec,
               const double* x, double* out, cudaStream_t st) {
    if (nb <= 0) return;
    count_launch();
    k_block_fit<<<nb, 256, 0, st>>>(blocks, xw, minv, bvec, x, out);
}

}  // namespace mpspt
