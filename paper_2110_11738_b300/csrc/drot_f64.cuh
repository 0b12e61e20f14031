// FP64 variant of the fused step (Algorithm 1, steps 4-5, Sec. 3.1) and of the set-up
// kernels that touch X.  Every quantity is FP64: the entries of X and C, phi_i, psi_j,
// the per-entry update and every sum.  The work split (row segments of one column tile
// per warp iteration, CTA ranges, slots), the partial-sum layout and the finish kernel
// are those of the FP32 path; only the tile width differs (256 columns: one warp reads
// 2 KB of X and 2 KB of C per row segment, as the FP32 path does with K = 4).
#pragma once

#include "drot_kernels.cuh"

namespace drot {

constexpr int kTileW64 = 256;  // columns per tile: 32 lanes x 4 chunks x 2 doubles

struct StepArgs64 {
    StepArgs base;      // work split, vectors, partials (base.X and base.C unused)
    const double* C;    // m x n, pitch ld, 16-byte aligned rows
    double* X;
};

// One pass over the CTA's row segments.  UPDATE = false: sums of the stored X only
// (the set-up pass that gives a_0, b_0 and alpha_0).
template <bool UPDATE>
__global__ void __launch_bounds__(kThreads, 2) drot_step_f64_kernel(StepArgs64 A64) {
    const StepArgs& A = A64.base;
    __shared__ double s_col[kWarps][kTileW64];
    __shared__ double s_red[kWarps][2];
    wait_for_predecessor();
    if (A.sc->done != kRunning) return;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long m = A.m, n = A.n, ld = A.ld;
    const long long w0 = A.wbound[blockIdx.x];
    const long long w1 = A.wbound[blockIdx.x + 1];
    const double rho = UPDATE ? A.sc->rho : 0.0;
    const double cs = __ldcg(&A.sc->c);
    int slot = A.slot_base[blockIdx.x];
    double scx = 0.0, sd = 0.0;

    long long w = w0;
    while (w < w1) {
        const long long t = w / m;
        const long long seg_end = min(w1, (t + 1) * m);
        const long long i0 = w - t * m, i1 = seg_end - t * m;
        const long long col0 = t * kTileW64;

        double psi[4][2], cacc[4][2];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const long long j = col0 + kk * 64 + lane * 2 + e;
                psi[kk][e] = (UPDATE && j < n) ? (__ldcg(A.h + j) + cs) * A.inv_m : 0.0;
                cacc[kk][e] = 0.0;
            }

        for (long long i = i0 + warp; i < i1; i += kWarps) {
            const double phi = UPDATE ? (__ldcg(A.g + i) + cs) * A.inv_n : 0.0;
            const long long rowoff = i * ld + col0 + lane * 2;
            double2 xv[4], cv[4];
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                if (col0 + kk * 64 + lane * 2 < n) {
                    xv[kk] = *reinterpret_cast<const double2*>(A64.X + rowoff + kk * 64);
                    if (UPDATE) cv[kk] = __ldcs(reinterpret_cast<const double2*>(A64.C + rowoff + kk * 64));
                }
            }
            double rs = 0.0;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const long long j = col0 + kk * 64 + lane * 2;
                if (j < n) {
                    double xs[2] = {xv[kk].x, xv[kk].y};
                    const double cc[2] = {UPDATE ? cv[kk].x : 0.0, UPDATE ? cv[kk].y : 0.0};
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        if (j + e < n) {
                            double xn = xs[e];
                            if (UPDATE) {
                                const double d = fma(-rho, cc[e], phi + psi[kk][e]);
                                xn = fmax(xs[e] + d, 0.0);
                                scx = fma(cc[e], xn, scx);
                                const double dp = fmax(d, 0.0);
                                sd = fma(dp, dp, sd);
                                xs[e] = xn;
                            }
                            rs += xn;
                            cacc[kk][e] += xn;
                        }
                    }
                    if (UPDATE) {
                        double* dst = A64.X + rowoff + kk * 64;
                        if (j + 1 < n) *reinterpret_cast<double2*>(dst) = make_double2(xs[0], xs[1]);
                        else dst[0] = xs[0];
                    }
                }
            }
            rs = warp_sum_f64(rs);
            if (lane == 0) {
                if (A.accumulate) atomicAdd(A.u + i, rs);
                else A.rowpart[t * m + i] = rs;
            }
        }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int e = 0; e < 2; ++e) s_col[warp][kk * 64 + lane * 2 + e] = cacc[kk][e];
        __syncthreads();
        double* out = A.colpart + (long long)slot * kTileW64;
        for (int x = threadIdx.x; x < kTileW64; x += kThreads) {
            double v = 0.0;
#pragma unroll
            for (int wv = 0; wv < kWarps; ++wv) v += s_col[wv][x];
            if (!A.accumulate) out[x] = v;
            else if (col0 + x < n) atomicAdd(A.v + col0 + x, v);
        }
        __syncthreads();
        ++slot;
        w = seg_end;
    }

    if (UPDATE) {
        double v[2] = {scx, sd};
        block_sum_f64<2, kThreads>(v, s_red);
        if (threadIdx.x == 0) {
            if (A.accumulate) {
                atomicAdd(acc_at(A.acc, 0), v[0]);
                atomicAdd(acc_at(A.acc, 1), v[1]);
            } else {
                A.ctapart[2 * blockIdx.x + 0] = v[0];
                A.ctapart[2 * blockIdx.x + 1] = v[1];
            }
        }
    }
}

// X_0 = p q^T (the paper's cold start, Sec. 4) in FP64.
__global__ void drot_init_plan_f64_kernel(double* X, const double* p, const double* q, long long m, long long n,
                                          long long ld) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx / n, j = idx - i * n;
        X[i * ld + j] = p[i] * q[j];
    }
}

__global__ void drot_count_nnz_f64_kernel(const double* X, long long m, long long n, long long ld, Scalars* sc) {
    unsigned long long cnt = 0;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx / n, j = idx - i * n;
        cnt += X[i * ld + j] > 0.0 ? 1ull : 0ull;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&sc->nnz, cnt);
}

}  // namespace drot
