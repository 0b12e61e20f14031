// Cluster-resident DROT for small problems.
//
// One thread-block cluster of CS CTAs keeps the whole problem on chip: CTA r holds a
// contiguous block of rows of X and C in its shared memory for the entire solve, so an
// iteration of Algorithm 1 (Sec. 3.1) touches no global memory at all.  The row sums
// are local to a CTA; column sums and the scalar totals are exchanged through
// distributed shared memory (each CTA owns a range of columns and finishes steps 5-8
// for its rows and its columns), and two hardware cluster barriers per iteration
// order the exchange.  Every CTA then forms the same scalar totals in the same order,
// so all CTAs take the same stopping decision and leave the loop together.
//
// Exchanges are pushed, not pulled: a CTA stores its column partials into the owners'
// shared memory, and its partial totals and its new h_j into every CTA's, before the
// cluster barrier that publishes them (barrier.cluster arrive has release and wait has
// acquire semantics), so every read on the critical path is local.  No double
// buffering is needed: each inbox is next written only after a barrier that every CTA
// reaches after its last read of it (column partials: written in phase 1, read in
// phase 2, rewritten after barrier #2; totals and h: written in phase 2, read in
// phase 3, rewritten after the next barrier #1).
#pragma once

#include <cooperative_groups.h>

#include "drot_kernels.cuh"

namespace drot {

constexpr int kClusterThreads = 256;
constexpr int kClusterParts = 8;  // sum r, ||.||_1, ||.||^2, p.g, q.h, sum s, <C,X>, sum [d]_+^2

struct ClusterArgs {
    const float* C;
    float* X;
    const double* p;
    const double* q;
    double *g, *h, *a, *b;  // state in global memory (read at entry, written at exit)
    Scalars* sc;
    long long m, n, ld;
    int rows_per_cta;       // R: CTA r owns rows [r R, min(m, (r + 1) R))
    int cols_per_cta;       // Q: CTA r owns columns [r Q, min(n, (r + 1) Q))
    int npad;               // shared-memory row pitch (floats), a multiple of 4 >= n
    long long budget;       // iterations this launch may run
    double inv_n, inv_m, inv_mn;
};

struct ClusterSmem {
    // carve of the dynamic shared memory of one CTA
    float* Xs;      // [R][npad]
    float* Cs;      // [R][npad]
    float* psi;     // [npad]   psi_j (FP32) for all columns
    double* colin;  // [CS][Q]  column partials of the owned columns, pushed by every CTA (rank-major)
    double* partin; // [CS][kClusterParts] scalar partials, pushed by every CTA (rank-major)
    double* u;      // [R]      row sums of the owned rows
    double* arow;   // [R]      a_i of the owned rows
    double* grow;   // [R]      g_i of the owned rows
    double* bcol;   // [Q]      b_j of the owned columns
    double* hall;   // [n]      h_j of all columns (pushed by their owners)
    double* red;    // [kClusterThreads / 32][kClusterParts] block reduction scratch
    double* prow;   // [R]      p_i of the owned rows
    double* qcol;   // [Q]      q_j of the owned columns
};

__host__ __device__ inline size_t cluster_smem_bytes(int R, int Q, int npad, long long n, int cs) {
    size_t b = 0;
    b += 2 * (size_t)R * npad * sizeof(float);
    b += (size_t)npad * sizeof(float);
    b = (b + 15) / 16 * 16;
    b += (size_t)cs * Q * sizeof(double) + (size_t)cs * kClusterParts * sizeof(double);
    b += 2 * (size_t)R * sizeof(double) + (size_t)R * sizeof(double) + (size_t)Q * sizeof(double);
    b += (size_t)n * sizeof(double) + (kClusterThreads / 32) * kClusterParts * sizeof(double);
    b += (size_t)R * sizeof(double) + (size_t)Q * sizeof(double);
    return b;
}

__device__ inline ClusterSmem carve_cluster_smem(unsigned char* base, int R, int Q, int npad, long long n, int cs) {
    ClusterSmem S;
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
    S.colin = reinterpret_cast<double*>(take((size_t)cs * Q * sizeof(double)));
    S.partin = reinterpret_cast<double*>(take((size_t)cs * kClusterParts * sizeof(double)));
    S.u = reinterpret_cast<double*>(take((size_t)R * sizeof(double)));
    S.arow = reinterpret_cast<double*>(take((size_t)R * sizeof(double)));
    S.grow = reinterpret_cast<double*>(take((size_t)R * sizeof(double)));
    S.bcol = reinterpret_cast<double*>(take((size_t)Q * sizeof(double)));
    S.hall = reinterpret_cast<double*>(take((size_t)n * sizeof(double)));
    S.red = reinterpret_cast<double*>(take((kClusterThreads / 32) * kClusterParts * sizeof(double)));
    S.prow = reinterpret_cast<double*>(take((size_t)R * sizeof(double)));
    S.qcol = reinterpret_cast<double*>(take((size_t)Q * sizeof(double)));
    return S;
}

template <int CS>
__global__ void __launch_bounds__(kClusterThreads, 1) drot_cluster_kernel(ClusterArgs P) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int R = P.rows_per_cta, Q = P.cols_per_cta, npad = P.npad;
    const long long m = P.m, n = P.n;
    ClusterSmem S = carve_cluster_smem(smem_raw, R, Q, npad, n, CS);
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long r0 = (long long)rank * R;
    const int nrows = (int)max(0LL, min((long long)R, m - r0));
    const long long c0 = (long long)rank * Q;
    const int ncols = (int)max(0LL, min((long long)Q, n - c0));

    // ---- load the owned rows of X and C, and the state, into shared memory
    for (long long e = tid; e < (long long)nrows * n; e += kClusterThreads) {
        const long long i = e / n, j = e - i * n;
        S.Xs[i * npad + j] = P.X[(r0 + i) * P.ld + j];
        S.Cs[i * npad + j] = P.C[(r0 + i) * P.ld + j];
    }
    for (int i = tid; i < nrows; i += kClusterThreads) {
        S.arow[i] = P.a[r0 + i];
        S.grow[i] = P.g[r0 + i];
        S.prow[i] = P.p[r0 + i];
    }
    for (int j = tid; j < ncols; j += kClusterThreads) {
        S.bcol[j] = P.b[c0 + j];
        S.qcol[j] = P.q[c0 + j];
    }
    for (long long j = tid; j < n; j += kClusterThreads) S.hall[j] = P.h[j];
    const double rho = P.sc->rho, inv_rho = P.sc->inv_rho, tol = P.sc->tol;
    const double sum_p = P.sc->sum_p, sum_q = P.sc->sum_q;
    const long long max_iter = P.sc->max_iter;
    const int rule = P.sc->stop_rule;
    double alpha = P.sc->alpha, c = P.sc->c;
    long long k = P.sc->k;
    int done = P.sc->done;
    double primal = P.sc->primal, dual = P.sc->dual, gap = P.sc->gap, res_l1 = P.sc->res_l1;
    double res_l2_sq = P.sc->res_l2, dres_sq = P.sc->dual_res_prev, beta = P.sc->beta;
    const float rhof = (float)rho;
    __syncthreads();
    for (long long j = tid; j < n; j += kClusterThreads) S.psi[j] = (float)((S.hall[j] + c) * P.inv_m);
    __syncthreads();

    for (long long it = 0; it < P.budget && done == kRunning; ++it) {
        // ---- phase 1: step 4 on the owned rows, with row sums, column partials, <C,X>, dual residual
        float scx = 0.f, sd = 0.f;
        for (int i = warp; i < nrows; i += kClusterThreads / 32) {
            const float phi = (float)((S.grow[i] + c) * P.inv_n);
            float* xr = S.Xs + (size_t)i * npad;
            const float* cr = S.Cs + (size_t)i * npad;
            float rs = 0.f;
            // four consecutive columns per lane per pass, 16-byte shared-memory accesses (rows and
            // psi start on 16-byte boundaries: npad is a multiple of 4); columns >= n are left alone
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
        // column partials: thread per column; runs of 16 rows in FP32, promoted to FP64
        // (FP64 has a long dependent latency on this GPU); pushed to the column's owner
        for (long long j = tid; j < n; j += kClusterThreads) {
            double v = 0.0;
            for (int i0 = 0; i0 < nrows; i0 += 16) {
                float f = 0.f;
                for (int i = i0; i < min(nrows, i0 + 16); ++i) f += S.Xs[(size_t)i * npad + j];
                v += (double)f;
            }
            const int owner = (int)(j / Q);
            cluster.map_shared_rank(S.colin, owner)[(size_t)rank * Q + (j - (long long)owner * Q)] = v;
        }
        // CTA totals of <C,X> and sum [d]_+^2 (warp sums in FP32, then FP64 across warps)
        scx = warp_sum_f32(scx);
        sd = warp_sum_f32(sd);
        if (lane == 0) {
            S.red[warp * kClusterParts + 0] = (double)scx;
            S.red[warp * kClusterParts + 1] = (double)sd;
        }
        cluster.sync();  // #1: every CTA's column partials are ready

        // ---- phase 2: steps 5-8 for the owned rows and columns, CTA partials of the totals
        double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // sum r, l1, l2^2, p.g, q.h, sum s
        for (int i = tid; i < nrows; i += kClusterThreads) {
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
        // columns: a group of CS lanes per column, lane g holding the partial pushed by
        // CTA g; a shuffle tree inside the group adds them (log2 CS dependent FP64 adds)
        // and the group's first lane finishes the column and pushes h_j to every CTA
        {
            constexpr int GPW = 32 / CS;  // columns per warp per pass
            const int g = lane % CS;
            for (int jj0 = warp * GPW; jj0 < ncols; jj0 += (kClusterThreads / 32) * GPW) {  // warp-uniform
                const int jj = jj0 + lane / CS;
                double v = jj < ncols ? S.colin[(size_t)g * Q + jj] : 0.0;
#pragma unroll
                for (int o = CS / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (g == 0 && jj < ncols) {
                    const long long j = c0 + jj;
                    const double qj = S.qcol[jj];
                    const double sj = v - qj;
                    const double hn = S.bcol[jj] - 2.0 * sj;
                    S.bcol[jj] -= sj;
#pragma unroll
                    for (int rr = 0; rr < CS; ++rr) cluster.map_shared_rank(S.hall, rr)[j] = hn;
                    acc[5] += sj;
                    acc[1] += fabs(sj);
                    acc[2] += sj * sj;
                    acc[4] += qj * hn;
                }
            }
        }
        {
            const double tot_l = warp_sum8_scatter(acc);  // lane 4q holds the warp total of value q
            const int qv = (lane >> 2) & 7;
            if ((lane & 3) == 0 && qv < 6) S.red[warp * kClusterParts + 2 + qv] = tot_l;
        }
        __syncthreads();
        if (tid < kClusterParts) {
            double v = 0.0;
            for (int w = 0; w < kClusterThreads / 32; ++w) v += S.red[w * kClusterParts + tid];
            // partial layout: 0 sum r, 1 l1, 2 l2^2, 3 p.g, 4 q.h, 5 sum s, 6 <C,X>, 7 sum [d]_+^2
            const int dst = tid < 2 ? 6 + tid : tid - 2;
#pragma unroll
            for (int rr = 0; rr < CS; ++rr) cluster.map_shared_rank(S.partin, rr)[rank * kClusterParts + dst] = v;
        }
        cluster.sync();  // #2: every CTA holds all partials and all h_j

        // ---- phase 3 (every CTA, identically): totals, scalars, stopping test, psi.
        // Warp 0 takes the CS partials (lane r those of CTA r), reduces them with a fixed
        // reduce-scatter pattern and lane 0 updates the scalars; the same code on the same data in
        // every CTA gives bitwise the same result everywhere.  Broadcast through shared memory.
        __shared__ double s_bc[4];
        __shared__ int s_done;
        if (warp == 0) {
            double t[kClusterParts];
            const double* rp = S.partin + (size_t)(lane < CS ? lane : 0) * kClusterParts;
#pragma unroll
            for (int q2 = 0; q2 < kClusterParts; ++q2) t[q2] = lane < CS ? rp[q2] : 0.0;
            const double tq = warp_sum8_scatter(t);  // lane 4q holds total q
#pragma unroll
            for (int q2 = 0; q2 < kClusterParts; ++q2) t[q2] = __shfl_sync(0xffffffffu, tq, 4 * q2);
            if (lane == 0) {
                beta = t[0] * P.inv_mn;
                const double c_new = 2.0 * beta - alpha;
                const double pphi = (t[3] + c_new * sum_p) * P.inv_n;
                const double qpsi = (t[4] + c_new * sum_q) * P.inv_m;
                primal = t[6];
                dual = (pphi + qpsi) * inv_rho;
                gap = fabs(primal - dual);
                res_l1 = t[1];
                res_l2_sq = t[2];
                dres_sq = t[7] * inv_rho * inv_rho;
                alpha -= beta;
                c = c_new;
                const bool finite = isfinite(primal) && isfinite(dual) && isfinite(res_l1) && isfinite(res_l2_sq) &&
                                    isfinite(dres_sq) && isfinite(c_new) && isfinite(t[5]);
                const bool conv = tol >= 0.0 && (!(rule & 1) || gap <= tol) && (!(rule & 2) || res_l1 <= tol) &&
                                  (!(rule & 4) || dres_sq <= tol * tol);
                int dn = kRunning;
                if (!finite) dn = kNonFinite;
                else if (conv) dn = kConverged;
                else if (k + 1 >= max_iter) dn = kIterCap;
                s_bc[0] = c;
                s_bc[1] = alpha;
                s_bc[2] = beta;
                s_done = dn;
            }
        }
        __syncthreads();
        c = s_bc[0];
        alpha = s_bc[1];
        beta = s_bc[2];
        done = s_done;
        k += 1;
        // psi for the next pass
        for (long long j = tid; j < n; j += kClusterThreads) S.psi[j] = (float)((S.hall[j] + c) * P.inv_m);
        __syncthreads();
    }

    // ---- write the iterate and the state back; no CTA leaves while others may read its memory
    for (long long e = tid; e < (long long)nrows * n; e += kClusterThreads) {
        const long long i = e / n, j = e - i * n;
        P.X[(r0 + i) * P.ld + j] = S.Xs[i * npad + j];
    }
    for (int i = tid; i < nrows; i += kClusterThreads) {
        P.a[r0 + i] = S.arow[i];
        P.g[r0 + i] = S.grow[i];
    }
    for (int j = tid; j < ncols; j += kClusterThreads) {
        P.b[c0 + j] = S.bcol[j];
        P.h[c0 + j] = S.hall[c0 + j];
    }
    if (rank == 0 && tid == 0) {
        Scalars* sc = P.sc;
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
    cluster.sync();
}

}  // namespace drot
