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
// are stored in BF16; every product accumulates in FP32 (tensor-core MMA through
// the wmma interface: these products are a few hundred MFLOP per training step,
// far from any roofline, and not on the solver's hot path).
#pragma once

#include <cuda_bf16.h>
#include <mma.h>

#include <cstdint>
#include <type_traits>

#include "drot_kernels.cuh"

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
// C[M x N] = A[M x K] * B[K x N] with BF16 operands and FP32 accumulation.
// TA: A is stored as its transpose (K x M, row-major); TB: B is stored as its
// transpose (N x K, row-major).  M, N, K are multiples of 16 (32 for M, N).
// Each warp owns a 32 x 32 block of C; gridDim.z splits K (split-K products add
// into C with atomics).
enum Epilogue : int {
    kStoreF32 = 0,     // C = acc (FP32)
    kReluBiasBf16 = 1, // H = bf16(max(acc + bias[n], 0))
    kMaskBf16 = 2,     // D = bf16(acc * (mask[m, n] > 0))
    kAtomicF32 = 3     // C += acc (FP32 atomics; split-K)
};

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) gemm_kernel(const bf16* A, const bf16* B, int M, int N, int K, int lda,
                                                   int ldb, int epi, float* Cf, bf16* Cb, int ldc, const float* bias,
                                                   const bf16* mask) {
    using namespace nvcuda;
    __shared__ float stage[4][32 * 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_n = N / 32;
    const int tile = blockIdx.x * 4 + warp;
    if (tile >= (M / 32) * tiles_n) return;  // whole warp leaves together
    const int tm = (tile / tiles_n) * 32, tn = (tile % tiles_n) * 32;
    const int ksplit = gridDim.z;
    const int kchunk = ((K / 16 + ksplit - 1) / ksplit) * 16;
    const int k0 = blockIdx.z * kchunk, k1 = min(K, k0 + kchunk);

    using LayA = typename std::conditional<TA, wmma::col_major, wmma::row_major>::type;
    using LayB = typename std::conditional<TB, wmma::col_major, wmma::row_major>::type;
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) wmma::fill_fragment(acc[a][b], 0.f);
    for (int k = k0; k < k1; k += 16) {
        wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, LayA> fa[2];
        wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, LayB> fb[2];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const bf16* pa = TA ? A + (size_t)k * lda + (tm + 16 * a) : A + (size_t)(tm + 16 * a) * lda + k;
            wmma::load_matrix_sync(fa[a], pa, lda);
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const bf16* pb = TB ? B + (size_t)(tn + 16 * b) * ldb + k : B + (size_t)k * ldb + (tn + 16 * b);
            wmma::load_matrix_sync(fb[b], pb, ldb);
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) wmma::mma_sync(acc[a][b], fa[a], fb[b], acc[a][b]);
    }
    float* st = stage[warp];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
            wmma::store_matrix_sync(st + (16 * a) * 32 + 16 * b, acc[a][b], 32, wmma::mem_row_major);
    __syncwarp();
    for (int e = lane; e < 32 * 32; e += 32) {
        const int r = tm + e / 32, c = tn + e % 32;
        const float v = st[e];
        const size_t o = (size_t)r * ldc + c;
        if (epi == kStoreF32) Cf[o] = v;
        else if (epi == kReluBiasBf16) Cb[o] = __float2bfloat16(fmaxf(v + bias[c], 0.f));
        else if (epi == kMaskBf16) Cb[o] = __float2bfloat16(__bfloat162float(mask[o]) > 0.f ? v : 0.f);
        else atomicAdd(Cf + o, v);
    }
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
// D3[r,k] = bf16(g_r W4[k] (H3[r,k] > 0)).  One block per 64 rows, thread = k.
__global__ void __launch_bounds__(kWidth) output_backward_kernel(const float* g, const bf16* H3, const float* W4,
                                                                  long long rows, float* dW4, float* db4, bf16* D3) {
    const int k = threadIdx.x;
    const long long r0 = (long long)blockIdx.x * 64;
    float acc = 0.f, gs = 0.f;
    for (long long r = r0; r < min(rows, r0 + 64); ++r) {
        const float h = __bfloat162float(H3[r * kWidth + k]);
        acc += g[r] * h;
        gs += g[r];
        D3[r * kWidth + k] = __float2bfloat16(h > 0.f ? g[r] * W4[k] : 0.f);
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
