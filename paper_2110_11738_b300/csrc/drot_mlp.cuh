// Device code of the learned warm start for DROT.
//
// A small MLP maps per-point features of a source point (its position, its
// relative mass and a summary of both point clouds) to a predicted dual
// potential mu_i (in units of the unnormalised squared distance).  A warm start
// built from it follows the fixed-point relation of Lemma opt-rel (Appendix A.2):
// Y* = X* + rho (mu* 1^T + 1 nu*^T), i.e. phi_0 = rho mu, psi_0 = rho nu.  The
// target side is filled in by the c-transform nu_j = min_i (c_ij - mu_i) and the
// source side tightened by mu_i = min_j (c_ij - nu_j), so the seed is exactly dual
// feasible for the FP32 cost (mu_i + nu_j <= c_ij).
//
// Network: F (64) -> 256 -> 256 -> 256 -> 1, ReLU between layers.  Weights are
// kept in FP32 (Adam state) with BF16 copies for the matrix products; activations
// are stored in BF16; every product accumulates in FP32 in tensor memory (tcgen05.mma
// with TMA-staged operands, drot_tc.cuh).
#pragma once

#include <cuda_bf16.h>

#include <cstdint>
#include <type_traits>

#include "drot_kernels.cuh"
#include "drot_tc.cuh"

namespace drot {
namespace mlp {

constexpr int kIn = 64;      // feature width (multiple of 32)
constexpr int kWidth = 256;  // hidden width
constexpr int kRowPad = 64;  // row count granularity of the activation buffers

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------- features
//
// Layout of one feature row (source point i of a problem with m source and n
// target points, marginals p, q, points in the unit square):
//   0-1   x_i
//   2     m p_i
//   3-18  4x4 histogram of the source cloud weighted by p (cell (a,b) at 3 + 4a + b)
//   19-34 4x4 histogram of the target cloud weighted by q
//   35-36 p-weighted mean of the source cloud
//   37-38 q-weighted mean of the target cloud
//   39-41 q-weighted variances (x, y) and covariance of the target cloud
//   42    1
//   43-63 0
__device__ __forceinline__ int cell4(float v) {
    int c = (int)(v * 4.0f);
    return c < 0 ? 0 : (c > 3 ? 3 : c);
}

// One block per problem.  xs: m x 2, yt: n x 2 (FP32), p: m, q: n (FP64);
// out: rows [row0, row0 + m) of the BF16 feature matrix (kIn columns).
__global__ void __launch_bounds__(256) features_kernel(const float* xs, const float* yt, const double* p,
                                                       const double* q, long long m, long long n, bf16* out,
                                                       long long row0) {
    __shared__ float hist_s[16], hist_t[16];
    __shared__ float mom[8];  // mean_s (2), mean_t (2), E_t[x^2], E_t[y^2], E_t[xy]
    if (threadIdx.x < 16) {
        hist_s[threadIdx.x] = 0.f;
        hist_t[threadIdx.x] = 0.f;
    }
    if (threadIdx.x < 8) mom[threadIdx.x] = 0.f;
    __syncthreads();
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        const float x = xs[2 * i], y = xs[2 * i + 1], w = (float)p[i];
        atomicAdd(&hist_s[4 * cell4(x) + cell4(y)], w);
        atomicAdd(&mom[0], w * x);
        atomicAdd(&mom[1], w * y);
    }
    for (long long j = threadIdx.x; j < n; j += blockDim.x) {
        const float x = yt[2 * j], y = yt[2 * j + 1], w = (float)q[j];
        atomicAdd(&hist_t[4 * cell4(x) + cell4(y)], w);
        atomicAdd(&mom[2], w * x);
        atomicAdd(&mom[3], w * y);
        atomicAdd(&mom[4], w * x * x);
        atomicAdd(&mom[5], w * y * y);
        atomicAdd(&mom[6], w * x * y);
    }
    __syncthreads();
    const float vx = mom[4] - mom[2] * mom[2], vy = mom[5] - mom[3] * mom[3], cxy = mom[6] - mom[2] * mom[3];
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        bf16* r = out + (row0 + i) * kIn;
        float f[kIn];
        f[0] = xs[2 * i];
        f[1] = xs[2 * i + 1];
        f[2] = (float)((double)m * p[i]);
        for (int c = 0; c < 16; ++c) {
            f[3 + c] = hist_s[c];
            f[19 + c] = hist_t[c];
        }
        f[35] = mom[0];
        f[36] = mom[1];
        f[37] = mom[2];
        f[38] = mom[3];
        f[39] = vx;
        f[40] = vy;
        f[41] = cxy;
        f[42] = 1.f;
        for (int c = 43; c < kIn; ++c) f[c] = 0.f;
        for (int c = 0; c < kIn; ++c) r[c] = __float2bfloat16(f[c]);
    }
}

// ---------------------------------------------------------------- matrix products
//
// Every product of the network (forward layers, the backward pass into the hidden layers,
// the weight gradients) runs on the tcgen05 tensor cores through tc::gemm_tn (drot_tc.cuh):
// C = A B^T with both operands K-major.  The layouts that makes necessary are kept next to
// the natural ones: the training forward pass writes H1^T and H2^T beside H1 and H2, the
// backward pass D^T beside D, the features are transposed once per step, and the BF16
// weights W2, W3 have transposed copies (the backward pass multiplies by W, not W^T).
using Epilogue = tc::Epilogue;
constexpr int kStoreF32 = tc::kStoreF32, kReluBiasBf16 = tc::kReluBiasBf16, kMaskBf16 = tc::kMaskBf16,
              kAtomicF32 = tc::kAtomicF32;

// dst (cols x rows, pitch rows) = src^T (src: rows x cols, pitch cols), BF16; 32 x 32 tiles
// through shared memory.  rows and cols are multiples of 32.
__global__ void __launch_bounds__(256) transpose_bf16_kernel(const bf16* src, bf16* dst, int rows, int cols) {
    __shared__ bf16 t[32][34];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int i = ty; i < 32; i += 8) t[i][tx] = src[(size_t)(r0 + i) * cols + c0 + tx];
    __syncthreads();
    for (int i = ty; i < 32; i += 8) dst[(size_t)(c0 + i) * rows + r0 + tx] = t[tx][i];
}

// ---------------------------------------------------------------- output layer, loss

// out[r] = sum_k W4[k] H3[r, k] + b4 (one warp per row).
__global__ void output_kernel(const bf16* H3, const float* W4, const float* b4, float* out, long long rows) {
    const long long r = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    float s = 0.f;
    for (int k = lane; k < kWidth; k += 32) s += W4[k] * __bfloat162float(H3[r * kWidth + k]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[r] = s + b4[0];
}

// Gauge-invariant weighted loss per problem s (rows of s carry weights w_r = p_i
// with sum 1): with e_r = out_r - y_r and ebar_s = sum_{r in s} w_r e_r,
//   L = (1/S) sum_s sum_{r in s} w_r (e_r - ebar_s)^2,
//   dL/dout_r = (2/S) w_r (e_r - ebar_s).
// Pass 1 accumulates ebar_s and sum w per problem.
__global__ void loss_pass1_kernel(const float* out, const float* y, const float* w, const int* seg, long long rows,
                                  float* ebar, float* wsum) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
         r += (long long)gridDim.x * blockDim.x) {
        const int s = seg[r];
        if (s < 0) continue;
        atomicAdd(ebar + s, w[r] * (out[r] - y[r]));
        atomicAdd(wsum + s, w[r]);
    }
}

__global__ void loss_pass2_kernel(const float* out, const float* y, const float* w, const int* seg, long long rows,
                                  const float* ebar, const float* wsum, float inv_segments, float* g, float* loss) {
    float lsum = 0.f;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
         r += (long long)gridDim.x * blockDim.x) {
        const int s = seg[r];
        float gr = 0.f;
        if (s >= 0) {
            const float e = out[r] - y[r] - ebar[s] / wsum[s];
            lsum += w[r] * e * e;
            gr = 2.f * inv_segments * w[r] * e;
        }
        g[r] = gr;
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, lsum * inv_segments);
}

// Output-layer backward: dW4[k] += sum_r g_r H3[r,k]; db4 += sum_r g_r;
// D3[r,k] = bf16(g_r W4[k] (H3[r,k] > 0)) and its transpose.  One block per 64 rows, thread = k.
__global__ void __launch_bounds__(kWidth) output_backward_kernel(const float* g, const bf16* H3, const float* W4,
                                                                  long long rows, float* dW4, float* db4, bf16* D3,
                                                                  bf16* D3T) {
    const int k = threadIdx.x;
    const long long r0 = (long long)blockIdx.x * 64;
    float acc = 0.f, gs = 0.f;
    for (long long r = r0; r < min(rows, r0 + 64); ++r) {
        const float h = __bfloat162float(H3[r * kWidth + k]);
        acc += g[r] * h;
        gs += g[r];
        const bf16 d = __float2bfloat16(h > 0.f ? g[r] * W4[k] : 0.f);
        D3[r * kWidth + k] = d;
        D3T[(long long)k * rows + r] = d;  // D3^T (kWidth x rows) for the weight gradient of layer 3
    }
    atomicAdd(dW4 + k, acc);
    if (k == 0) atomicAdd(db4, gs);
}

// Column sums of a BF16 row-major matrix into FP32 (bias gradients): db[k] += sum_r D[r,k].
__global__ void __launch_bounds__(kWidth) column_sum_kernel(const bf16* D, long long rows, float* db) {
    const int k = threadIdx.x;
    const long long r0 = (long long)blockIdx.x * 64;
    float acc = 0.f;
    for (long long r = r0; r < min(rows, r0 + 64); ++r) acc += __bfloat162float(D[r * kWidth + k]);
    atomicAdd(db + k, acc);
}

// Adam (bias-corrected) on an FP32 parameter vector, refreshing its BF16 copy.
__global__ void adam_kernel(float* w, const float* grad, float* m1, float* m2, bf16* wb, long long count, float lr,
                            float beta1, float beta2, float eps, float corr1, float corr2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float a = beta1 * m1[i] + (1.f - beta1) * gi;
        const float b = beta2 * m2[i] + (1.f - beta2) * gi * gi;
        m1[i] = a;
        m2[i] = b;
        const float wi = w[i] - lr * (a / corr1) / (sqrtf(b / corr2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16(wi);
    }
}

__global__ void to_bf16_kernel(const float* src, bf16* dst, long long count) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16(src[i]);
}

// ---------------------------------------------------------------- warm-start seed

// mu_i = (pred_i - sum_k p_k pred_k) / scale (centred prediction in units of C).
// One block.
__global__ void __launch_bounds__(1024) centre_prediction_kernel(const float* pred, const double* p, long long m,
                                                                 double inv_scale, double* mu) {
    __shared__ double s_red[32][1];
    double v[1] = {0.0};
    for (long long i = threadIdx.x; i < m; i += blockDim.x) v[0] += p[i] * (double)pred[i];
    block_sum_f64<1, 1024>(v, s_red);
    __shared__ double mean;
    if (threadIdx.x == 0) mean = v[0];
    __syncthreads();
    for (long long i = threadIdx.x; i < m; i += blockDim.x) mu[i] = ((double)pred[i] - mean) * inv_scale;
}

// nu_j = min_i (c_ij - mu_i): one thread per column, rows streamed (coalesced across j).
__global__ void c_transform_cols_kernel(const float* C, long long m, long long n, long long ld, const double* mu,
                                        double* nu) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        double best = 1e300;
        for (long long i = 0; i < m; ++i) best = fmin(best, (double)C[i * ld + j] - mu[i]);
        nu[j] = best;
    }
}

// mu_i = min_j (c_ij - nu_j): one warp per row.
__global__ void c_transform_rows_kernel(const float* C, long long m, long long n, long long ld, const double* nu,
                                        double* mu) {
    const long long i = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= m) return;
    double best = 1e300;
    for (long long j = lane; j < n; j += 32) best = fmin(best, (double)C[i * ld + j] - nu[j]);
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) mu[i] = best;
}

}  // namespace mlp
}  // namespace drot
