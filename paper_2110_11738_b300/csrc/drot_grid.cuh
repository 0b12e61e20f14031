// Grid-resident DROT for mid-size problems (too large for one cluster, small enough that the
// whole plan and cost fit in the shared memory of one CTA per SM).
//
// One cooperative launch of G CTAs (at most one per SM) runs many iterations of Algorithm 1
// (Sec. 3.1).  CTA c keeps rows [c R, c R + R) of X and C in shared memory for the whole
// launch, so the step touches no global memory for the plan; it owns columns [c Q, c Q + Q)
// for steps 5-8 of the column side.  An iteration:
//   1. the step on the owned rows (row sums local), the column partials of all n columns
//      added into the FP64 column totals v with atomics, steps 5-8 of the owned rows and the
//      row-side sums (sum r, ||r||_1, ||r||^2, p.g', <C,X>, sum [d]_+^2) added into the
//      totals of this iteration's parity;
//   2. grid barrier #1; every CTA reads the row-side totals and forms beta and the new scalar
//      c = 2 beta - alpha (identically: the same values in the same order);
//   3. each owner reads v_j of its columns, resets it to 0, finishes steps 5-8 for them
//      (s_j, b_j, h_j), writes psi_j = (h_j + c) / m for the next pass and adds the
//      column-side sums; CTA 0 clears the other parity's totals;
//   4. grid barrier #2; every CTA reads the column-side totals, forms the dual objective, the
//      gap, the norms and the stopping decision (identically), and copies psi into shared
//      memory.
// The barriers are one monotonic arrival counter (grid_barrier_counter: barrier t of a launch
// waits for (t + 1) G arrivals); a CTA that waits longer than the spin limit, or sees another's fault, sets the
// fault flag and the launch ends (DROT_ERR_TIMEOUT on the host).  Buffer reuse is ordered by
// the barriers: v_j is reset by its only reader before barrier #2 and next added to after it;
// psi is written between the barriers and read after #2, before the next #1; the totals of
// parity k mod 2 are read until barrier #1 of iteration k + 1 and cleared after it.
#pragma once

#include "drot_cluster.cuh"
#include "drot_kernels.cuh"

namespace drot {

constexpr int kGridThreads = 256;
constexpr int kGridTotals = 16;  // per parity: 0-7 row side (layout below), 8-11 column side

struct GridArgs {
    ClusterArgs P;      // problem, state vectors and scalars; rows_per_cta R, cols_per_cta Q, npad
    double* v;          // [n] FP64 column totals (0 at launch; each owner resets its columns)
    float* psi_g;       // [n] psi of the next pass, written by the owners of the columns
    double* totals;     // [2][kGridTotals], 0 at launch
    unsigned int* bar;  // arrival counter, 0 at launch
};

struct GridSmem {
    float* Xs;      // [R][npad]
    float* Cs;      // [R][npad]
    float* psi;     // [npad]
    double* u;      // [R]
    double* arow;   // [R]
    double* grow;   // [R]
    double* prow;   // [R]
    double* bown;   // [Q] b_j of the owned columns
    double* qown;   // [Q]
    double* hown;   // [Q]
    double* red;    // [kGridThreads / 32][8]
};

__host__ __device__ inline size_t grid_smem_bytes(int R, int Q, int npad) {
    size_t b = 2 * (size_t)R * npad * sizeof(float) + (size_t)npad * sizeof(float);
    b = (b + 15) / 16 * 16;
    b += 4 * (size_t)R * sizeof(double) + 3 * (size_t)Q * sizeof(double);
    b += (kGridThreads / 32) * 8 * sizeof(double);
    return b;
}

__device__ inline GridSmem carve_grid_smem(unsigned char* base, int R, int Q, int npad) {
    GridSmem S;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = base + off;
        off += bytes;
        return p;
    };
    S.Xs = reinterpret_cast<float*>(take((size_t)R * npad * sizeof(float)));
    S.Cs = reinterpret_cast<float*>(take((size_t)R * npad * sizeof(float)));
    S.psi = reinterpret_cast<float*>(take((size_t)npad * sizeof(float)));
    off = (off + 15) / 16 * 16;
    S.u = reinterpret_cast<double*>(take((size_t)R * sizeof(double)));
    S.arow = reinterpret_cast<double*>(take((size_t)R * sizeof(double)));
    S.grow = reinterpret_cast<double*>(take((size_t)R * sizeof(double)));
    S.prow = reinterpret_cast<double*>(take((size_t)R * sizeof(double)));
    S.bown = reinterpret_cast<double*>(take((size_t)Q * sizeof(double)));
    S.qown = reinterpret_cast<double*>(take((size_t)Q * sizeof(double)));
    S.hown = reinterpret_cast<double*>(take((size_t)Q * sizeof(double)));
    S.red = reinterpret_cast<double*>(take((kGridThreads / 32) * 8 * sizeof(double)));
    return S;
}

__global__ void __launch_bounds__(kGridThreads, 1) drot_grid_kernel(GridArgs A) {
    const ClusterArgs& P = A.P;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int R = P.rows_per_cta, Q = P.cols_per_cta, npad = P.npad;
    const long long m = P.m, n = P.n;
    GridSmem S = carve_grid_smem(smem_raw, R, Q, npad);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = (int)gridDim.x;
    const long long r0 = (long long)blockIdx.x * R;
    const int nrows = (int)max(0LL, min((long long)R, m - r0));
    const long long c0 = (long long)blockIdx.x * Q;
    const int ncols = (int)max(0LL, min((long long)Q, n - c0));

    // ---- the owned rows of X and C with their state, the owned columns' state, psi of all columns
    for (long long e = tid; e < (long long)nrows * n; e += kGridThreads) {
        const long long i = e / n, j = e - i * n;
        S.Xs[i * npad + j] = P.X[(r0 + i) * P.ld + j];
        S.Cs[i * npad + j] = P.C[(r0 + i) * P.ld + j];
    }
    for (int i = tid; i < nrows; i += kGridThreads) {
        S.arow[i] = P.a[r0 + i];
        S.grow[i] = P.g[r0 + i];
        S.prow[i] = P.p[r0 + i];
    }
    for (int j = tid; j < ncols; j += kGridThreads) {
        S.bown[j] = P.b[c0 + j];
        S.qown[j] = P.q[c0 + j];
        S.hown[j] = P.h[c0 + j];
    }
    Scalars* sc = P.sc;
    const double rho = sc->rho, inv_rho = sc->inv_rho, tol = sc->tol;
    const double sum_p = sc->sum_p, sum_q = sc->sum_q;
    const long long max_iter = sc->max_iter;
    const int rule = sc->stop_rule;
    double alpha = sc->alpha, c = sc->c;
    long long k = sc->k;
    int done = sc->done;
    double primal = sc->primal, dual = sc->dual, gap = sc->gap, res_l1 = sc->res_l1;
    double res_l2_sq = sc->res_l2, dres_sq = sc->dual_res_prev, beta = sc->beta;
    const float rhof = (float)rho;
    for (long long j = tid; j < n; j += kGridThreads) S.psi[j] = (float)((P.h[j] + c) * P.inv_m);
    __syncthreads();

    __shared__ double s_row[8];
    __shared__ double s_bc[4];
    __shared__ int s_done;
    unsigned int target = 0;
    for (long long it = 0; it < P.budget && done == kRunning; ++it) {
        double* tot = A.totals + (size_t)(k & 1) * kGridTotals;
        double* tot_other = A.totals + (size_t)((k + 1) & 1) * kGridTotals;
        // ---- 1. step 4 on the owned rows, with row sums, <C,X> and sum [d]_+^2
        float scx = 0.f, sd = 0.f;
        for (int i = warp; i < nrows; i += kGridThreads / 32) {
            const float phi = (float)((S.grow[i] + c) * P.inv_n);
            float* xr = S.Xs + (size_t)i * npad;
            const float* cr = S.Cs + (size_t)i * npad;
            float rs = 0.f;
            for (int j4 = lane * 4; j4 < n; j4 += 128) {
                const float4 xv = *reinterpret_cast<const float4*>(xr + j4);
                const float4 cv = *reinterpret_cast<const float4*>(cr + j4);
                const float4 pv = *reinterpret_cast<const float4*>(S.psi + j4);
                float xs[4] = {xv.x, xv.y, xv.z, xv.w};
                const float cs4[4] = {cv.x, cv.y, cv.z, cv.w};
                const float ps4[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (j4 + e < n) {
                        const float d = fmaf(-rhof, cs4[e], phi + ps4[e]);
                        const float xn = fmaxf(xs[e] + d, 0.f);
                        xs[e] = xn;
                        rs += xn;
                        scx = fmaf(cs4[e], xn, scx);
                        const float dp = fmaxf(d, 0.f);
                        sd = fmaf(dp, dp, sd);
                    }
                }
                *reinterpret_cast<float4*>(xr + j4) = make_float4(xs[0], xs[1], xs[2], xs[3]);
            }
            rs = warp_sum_f32(rs);
            if (lane == 0) S.u[i] = (double)rs;
        }
        __syncthreads();
        // column partials of the owned rows (runs of 16 rows in FP32, then FP64) into v
        if (nrows > 0) {
            for (long long j = tid; j < n; j += kGridThreads) {
                double vp = 0.0;
                for (int i0 = 0; i0 < nrows; i0 += 16) {
                    float f = 0.f;
                    for (int i = i0; i < min(nrows, i0 + 16); ++i) f += S.Xs[(size_t)i * npad + j];
                    vp += (double)f;
                }
                atomicAdd(A.v + j, vp);
            }
        }
        // steps 5-8 of the owned rows; row-side sums
        // (layout: 0 sum r, 1 ||r||_1, 2 ||r||^2, 3 p.g', 6 <C,X>, 7 sum [d]_+^2)
        double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, (double)scx, (double)sd};
        for (int i = tid; i < nrows; i += kGridThreads) {
            const double pi = S.prow[i];
            const double r = S.u[i] - pi;
            const double gn = S.arow[i] - 2.0 * r;
            S.arow[i] -= r;
            S.grow[i] = gn;
            acc[0] += r;
            acc[1] += fabs(r);
            acc[2] += r * r;
            acc[3] += pi * gn;
        }
        {
            const double t = warp_sum8_scatter(acc);  // lane 4q holds the warp total of value q
            if ((lane & 3) == 0) S.red[warp * 8 + ((lane >> 2) & 7)] = t;
        }
        __syncthreads();
        if (tid < 8 && tid != 4 && tid != 5) {
            double s = 0.0;
            for (int w = 0; w < kGridThreads / 32; ++w) s += S.red[w * 8 + tid];
            atomicAdd(tot + tid, s);
        }
        target += (unsigned int)G;
        if (!grid_barrier_counter(A.bar, target, kBarrierSpins, sc)) break;  // #1: v and the row-side totals are complete

        // ---- 2. row-side totals and the new scalar c (every CTA identically)
        if (tid < 8) s_row[tid] = __ldcg(tot + tid);
        __syncthreads();
        beta = s_row[0] * P.inv_mn;
        const double c_new = 2.0 * beta - alpha;
        // ---- 3. steps 5-8 of the owned columns, psi of the next pass, column-side sums
        double cacc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // 0 sum s, 1 l1, 2 l2^2, 3 q.h'
        for (int jj = tid; jj < ncols; jj += kGridThreads) {
            const long long j = c0 + jj;
            const double vj = __ldcg(A.v + j);
            A.v[j] = 0.0;  // the next iteration's partials are added after barrier #2
            const double qj = S.qown[jj];
            const double sj = vj - qj;
            const double hn = S.bown[jj] - 2.0 * sj;
            S.bown[jj] -= sj;
            S.hown[jj] = hn;
            A.psi_g[j] = (float)((hn + c_new) * P.inv_m);
            cacc[0] += sj;
            cacc[1] += fabs(sj);
            cacc[2] += sj * sj;
            cacc[3] += qj * hn;
        }
        {
            const double t = warp_sum8_scatter(cacc);
            if ((lane & 3) == 0) S.red[warp * 8 + ((lane >> 2) & 7)] = t;
        }
        __syncthreads();
        if (tid < 4) {
            double s = 0.0;
            for (int w = 0; w < kGridThreads / 32; ++w) s += S.red[w * 8 + tid];
            atomicAdd(tot + 8 + tid, s);
        }
        // the other parity's totals were last read before barrier #1 of this iteration
        if (blockIdx.x == 0 && tid >= 32 && tid < 32 + kGridTotals) tot_other[tid - 32] = 0.0;
        target += (unsigned int)G;
        if (!grid_barrier_counter(A.bar, target, kBarrierSpins, sc)) break;  // #2: psi and the column-side totals are complete

        // ---- 4. totals, the stopping test (every CTA identically) and psi of the next pass
        if (tid == 0) {
            double t[8];
#pragma unroll
            for (int q2 = 0; q2 < 4; ++q2) t[q2] = __ldcg(tot + 8 + q2);
            const double sum_s = t[0], l1 = s_row[1] + t[1], l2 = s_row[2] + t[2];
            const double pphi = (s_row[3] + c_new * sum_p) * P.inv_n;
            const double qpsi = (t[3] + c_new * sum_q) * P.inv_m;
            primal = s_row[6];
            dual = (pphi + qpsi) * inv_rho;
            gap = fabs(primal - dual);
            res_l1 = l1;
            res_l2_sq = l2;
            dres_sq = s_row[7] * inv_rho * inv_rho;
            const bool finite = isfinite(primal) && isfinite(dual) && isfinite(res_l1) && isfinite(res_l2_sq) &&
                                isfinite(dres_sq) && isfinite(c_new) && isfinite(sum_s);
            const bool conv = tol >= 0.0 && (!(rule & 1) || gap <= tol) && (!(rule & 2) || res_l1 <= tol) &&
                              (!(rule & 4) || dres_sq <= tol * tol);
            int dn = kRunning;
            if (!finite) dn = kNonFinite;
            else if (conv) dn = kConverged;
            else if (k + 1 >= max_iter) dn = kIterCap;
            s_bc[0] = primal;
            s_bc[1] = dual;
            s_bc[2] = res_l1;
            s_bc[3] = res_l2_sq;
            s_done = dn;
        }
        for (long long j = tid; j < n; j += kGridThreads) S.psi[j] = __ldcg(A.psi_g + j);
        __syncthreads();
        alpha -= beta;
        c = c_new;
        primal = s_bc[0];
        dual = s_bc[1];
        res_l1 = s_bc[2];
        res_l2_sq = s_bc[3];
        gap = fabs(primal - dual);
        dres_sq = s_row[7] * inv_rho * inv_rho;
        done = s_done;
        k += 1;
        __syncthreads();  // s_row, s_bc and s_done are rewritten by the next iteration
    }

    // ---- write the iterate and the state back (each CTA its rows and its columns)
    for (long long e = tid; e < (long long)nrows * n; e += kGridThreads) {
        const long long i = e / n, j = e - i * n;
        P.X[(r0 + i) * P.ld + j] = S.Xs[i * npad + j];
    }
    for (int i = tid; i < nrows; i += kGridThreads) {
        P.a[r0 + i] = S.arow[i];
        P.g[r0 + i] = S.grow[i];
    }
    for (int j = tid; j < ncols; j += kGridThreads) {
        P.b[c0 + j] = S.bown[j];
        P.h[c0 + j] = S.hown[j];
    }
    if (blockIdx.x == 0 && tid == 0 && !*(volatile int*)&sc->fault) {
        sc->alpha = alpha;
        sc->c = c;
        sc->k = k;
        sc->beta = beta;
        sc->primal = primal;
        sc->dual = dual;
        sc->gap = gap;
        sc->res_l1 = res_l1;
        sc->res_l2 = res_l2_sq;
        sc->dual_res_prev = dres_sq;
        sc->done = done;
    }
}

}  // namespace drot
