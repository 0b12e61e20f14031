// Device code of the batched DROT solver: many independent problems of uneven
// sizes advanced together, one fused-step launch and one finish launch per
// iteration for all problems that have not stopped yet.
//
// Each problem runs Algorithm 1 (Sec. 3.1) exactly as the single-problem solver
// does (same per-entry arithmetic, same FP64 totals in accumulation mode, its own
// scalar state, stopping test and flag).  What is shared is the launch: the row
// segments of all active problems form one list (problem-major, then tile-major,
// then row), the host cuts that list into one contiguous, cost-balanced range per
// CTA, and each CTA walks its range segment by segment, taking the tile width of
// the problem a segment belongs to.  Tiles with at most 256 valid columns (the narrow
// last tile of a 512-column tiling, or every tile of a narrower tiling) form a second
// list served by a second kernel, which packs four or eight rows into one warp iteration
// so that a narrow tile still moves up to 4 KB per array per memory round trip; it is a
// separate kernel so that neither loop takes registers from the other, and its CTAs
// start on the SMs the first kernel's CTAs leave.  Both kernels have a warp prefetch the
// rows of its next iteration into L2 while its current loads are in flight: a warp then
// keeps two iterations' bytes in flight with one iteration's registers, which is what a
// ragged or narrow tile (fewer bytes per round trip) and the start of every segment need.
// The finish launch gives each active problem
// its own group of blocks; the last block of a group closes that problem's
// iteration.  Converged problems are dropped from the lists between graph replays
// (and their segments skipped inside a replay), so the work of a launch shrinks as
// problems finish.
#pragma once

#include "drot_kernels.cuh"

namespace drot {

// Per-problem device descriptor (fixed for the whole batched call).
struct BatchProb {
    const float* C;
    float* X;
    const double* p;
    const double* q;
    double* mu;             // warm-start duals on entry, duals on exit
    double* nu;
    double *g, *h, *a, *b;  // phi/psi numerators and the a, b state vectors
    double *u, *v;          // row / column totals (FP64 atomics), reset by the finish pass
    double* acc;            // [8] <C,X>, sum [d]_+^2 and the finish totals (FP64 atomics)
    double* finpart;        // [fin_blocks][kFinishAcc]
    Scalars* sc;
    long long m, n, ld;
    double inv_n, inv_m;
    int K;                  // float4 chunks per lane (tile width 128 K)
    int T;                  // column tiles
    int Tw;                 // tiles [0, Tw) are wide (> 256 valid columns), [Tw, T) narrow
    int fin_blocks;         // blocks of the finish launch serving this problem
    int pad;
};

// Work lists of the current replay (rebuilt by the host between replays).
struct BatchArgs {
    const BatchProb* probs;
    const int* active;         // [nactive] problem indices, in segment-list order
    const long long* unit0;    // [nactive + 1] first segment of each active problem; unit0[nactive] = total
    const long long* wbound;   // [G + 1] segment range of each step CTA
    const int* fin_prob;       // [FB] problem served by each finish block (-1: idle)
    const int* fin_local;      // [FB] index of the block within its problem's group
    const int* nactive;        // number of active problems (device, updated between replays)
    const int* parity;         // parity of the iterations already run (device, updated between replays)
    // the narrow tiles' list, same layout (segments of tiles Tw .. T-1 of each problem that has any)
    const int* active_n;
    const long long* unit0_n;
    const long long* wbound_n;
    const int* nactive_n;
    int narrow_next;           // 1: the narrow-tile kernel follows this wide-tile launch
    int warm;
    int serp;                  // 1: alternate the direction of the passes (as SegWalk does)
    int odd;                   // parity of this pass in its graph; backwards when serp and parity + odd is odd
};

__device__ __forceinline__ FinishArgs batch_finish_args(const BatchProb& P) {
    FinishArgs F{};
    F.u = P.u;
    F.v = P.v;
    F.acc = P.acc;
    F.accumulate = 1;
    F.p = P.p;
    F.q = P.q;
    F.a = P.a;
    F.b = P.b;
    F.g = P.g;
    F.h = P.h;
    F.finpart = P.finpart;
    F.sc = P.sc;
    F.m = P.m;
    F.n = P.n;
    F.inv_n = P.inv_n;
    F.inv_m = P.inv_m;
    F.inv_mn = 1.0 / (double)(P.m + P.n);
    return F;
}

// Fused DR pass over the wide tiles of every active problem (UPDATE = false: row/column
// sums of X_0 only, used once at initialisation).
template <bool UPDATE>
__global__ void __launch_bounds__(kThreads, 2) drot_batched_step_kernel(BatchArgs B) {
    constexpr int KMAX = 4;
    __shared__ double s_col[kWarps][128 * KMAX];
    __shared__ double s_red[kWarps][2];
    __shared__ float s_psi[128 * KMAX];  // psi of the segment's tile and phi of a chunk of its rows,
    __shared__ float s_phi[kPhiChunk];   // formed once per CTA (FP64 is scarce: see StepSmem)

    wait_for_predecessor();
    // the narrow-tile kernel launched after this one may start its blocks now: it reads
    // only what the finish before this kernel wrote, and waits for this grid before it ends
    // (a finish launched next instead is not released early: its blocks would take the
    // SMs this kernel frees and hold them waiting)
    if (B.narrow_next) release_dependents();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long w0 = B.wbound[blockIdx.x];
    const long long w1 = B.wbound[blockIdx.x + 1];
    const int nactive = *B.nactive;
    if (w0 >= w1 || nactive <= 0) return;
    // Serpentine order (see SegWalk): every active problem has run the same number of
    // iterations, so one parity serves the whole launch.  Backwards, the problems, the
    // tiles of a problem and the rows of a tile are all walked in reverse.
    const bool rev = B.serp != 0 && ((*B.parity + B.odd) & 1) != 0;

    // the active problem holding the first segment walked: the last a with unit0[a] <= it
    const long long wfirst = rev ? w1 - 1 : w0;
    int lo = 0, hi = nactive - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.unit0[mid] <= wfirst) lo = mid;
        else hi = mid - 1;
    }
    int ai = lo;
    long long w = rev ? w1 : w0;
    while (rev ? w > w0 : w < w1) {
        if (rev) {
            while (ai > 0 && w - 1 < B.unit0[ai]) --ai;
        } else {
            while (ai + 1 < nactive && w >= B.unit0[ai + 1]) ++ai;
        }
        const BatchProb& P = B.probs[B.active[ai]];
        const long long base = B.unit0[ai];
        const long long m = P.m, n = P.n, ld = P.ld;
        const long long t = ((rev ? w - 1 : w) - base) / m;
        const long long seg_lo = rev ? max(w0, base + t * m) : w;
        const long long seg_hi = rev ? w : min(w1, base + (t + 1) * m);
        const long long i0 = seg_lo - base - t * m, i1 = seg_hi - base - t * m;
        w = rev ? seg_lo : seg_hi;
        if (P.sc->done != kRunning) continue;  // uniform: every thread reads the same flag

        const int K = P.K;
        const int TW = 128 * K;
        const long long col0 = t * TW;
        const double cs = P.sc->c;
        const float rho = UPDATE ? (float)P.sc->rho : 0.f;

        // every thread arrives here together (the previous segment ended with a barrier)
        if (UPDATE) {
            for (int x = threadIdx.x; x < TW; x += kThreads) {
                const long long j = col0 + x;
                s_psi[x] = j < n ? (float)((P.h[j] + cs) * P.inv_m) : 0.f;
            }
        }
        float psi[KMAX][4], cacc[KMAX][4];
        for (int x = lane; x < TW; x += 32) s_col[warp][x] = 0.0;

        float scx = 0.f, sd = 0.f;
        double scx64 = 0.0, sd64 = 0.0;
        int since_flush = 0;
        // chunks of kPhiChunk rows (a multiple of kWarps); the chunk edge c is the chunk's
        // first row forwards and one past its last row backwards
        const long long c_first = rev ? i1 : i0;
        for (long long c = c_first; rev ? c > i0 : c < i1; c += rev ? -kPhiChunk : kPhiChunk) {
        const long long r0 = rev ? max(i0, c - (long long)kPhiChunk) : c;
        const long long r1 = rev ? c : min(i1, c + (long long)kPhiChunk);
        if (UPDATE) {
            if (c != c_first) __syncthreads();  // every warp is done with the previous chunk's phi
            for (long long r = r0 + threadIdx.x; r < r1; r += kThreads)
                s_phi[r - r0] = (float)((P.g[r] + cs) * P.inv_n);
        }
        __syncthreads();
        if (c == c_first) {
#pragma unroll
            for (int kk = 0; kk < KMAX; ++kk)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    psi[kk][e] = (UPDATE && kk < K) ? s_psi[kk * 128 + lane * 4 + e] : 0.f;
                    cacc[kk][e] = 0.f;
                }
        }
        for (long long i = rev ? r1 - 1 - warp : r0 + warp; rev ? i >= r0 : i < r1; i += rev ? -kWarps : kWarps) {
            const float phi = UPDATE ? s_phi[i - r0] : 0.f;
            const long long rowoff = i * ld + col0 + lane * 4;
            float4 xv[KMAX], cv[KMAX];
#pragma unroll
            for (int kk = 0; kk < KMAX; ++kk) {
                if (kk < K && col0 + kk * 128 + lane * 4 < n) {
                    xv[kk] = *reinterpret_cast<const float4*>(P.X + rowoff + kk * 128);
                    if (UPDATE) cv[kk] = ld_stream_ro(P.C + rowoff + kk * 128);
                }
            }
            if (UPDATE) {
                // the warp's next row of this chunk into L2 (lanes 0-15: X, 16-31: C; one 128-byte
                // line each): its loads then find it there, so a warp has two rows in flight
                // without holding a second row's registers
                const long long inext = rev ? i - kWarps : i + kWarps;
                const int line = lane & 15;
                if (inext >= r0 && inext < r1 && line * 32 < TW && col0 + line * 32 < n) {
                    const float* pf = (lane < 16 ? P.X : P.C) + inext * ld + col0 + line * 32;
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(pf));
                }
            }
            float rs = 0.f;
#pragma unroll
            for (int kk = 0; kk < KMAX; ++kk) {
                const long long j = col0 + kk * 128 + lane * 4;
                if (kk < K && j < n) {
                    float xs[4] = {xv[kk].x, xv[kk].y, xv[kk].z, xv[kk].w};
                    float cc[4] = {0.f, 0.f, 0.f, 0.f};
                    if (UPDATE) { cc[0] = cv[kk].x; cc[1] = cv[kk].y; cc[2] = cv[kk].z; cc[3] = cv[kk].w; }
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (j + e < n) {
                            float xn = xs[e];
                            if (UPDATE) {
                                const float d = fmaf(-rho, cc[e], phi + psi[kk][e]);
                                xn = fmaxf(xs[e] + d, 0.f);
                                scx = fmaf(cc[e], xn, scx);
                                const float dp = fmaxf(d, 0.f);
                                sd = fmaf(dp, dp, sd);
                                xs[e] = xn;
                            }
                            rs += xn;
                            cacc[kk][e] += xn;
                        }
                    }
                    if (UPDATE) {
                        float* dst = P.X + rowoff + kk * 128;
                        if (j + 3 < n) {
                            *reinterpret_cast<float4*>(dst) = make_float4(xs[0], xs[1], xs[2], xs[3]);
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (j + e < n) dst[e] = xs[e];
                        }
                    }
                }
            }
            rs = warp_sum_f32(rs);
            if (lane == 0) atomicAdd(P.u + i, (double)rs);
            if (++since_flush == kFlushRows) {
#pragma unroll
                for (int kk = 0; kk < KMAX; ++kk)
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (kk < K) {
                            s_col[warp][kk * 128 + lane * 4 + e] += (double)cacc[kk][e];
                            cacc[kk][e] = 0.f;
                        }
                scx64 += (double)scx;
                sd64 += (double)sd;
                scx = 0.f;
                sd = 0.f;
                since_flush = 0;
            }
        }
        }  // row chunks
#pragma unroll
        for (int kk = 0; kk < KMAX; ++kk)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (kk < K) s_col[warp][kk * 128 + lane * 4 + e] += (double)cacc[kk][e];
        scx64 += (double)scx;
        sd64 += (double)sd;
        __syncthreads();
        for (int x = threadIdx.x; x < TW; x += kThreads) {
            double v = 0.0;
#pragma unroll
            for (int wv = 0; wv < kWarps; ++wv) v += s_col[wv][x];
            if (col0 + x < n) atomicAdd(P.v + col0 + x, v);
        }
        if (UPDATE) {
            double v2[2] = {scx64, sd64};
            block_sum_f64<2, kThreads>(v2, s_red);  // ends with a block barrier
            if (threadIdx.x == 0) {
                atomicAdd(acc_at(P.acc, 0), v2[0]);
                atomicAdd(acc_at(P.acc, 1), v2[1]);
            }
        } else {
            __syncthreads();
        }
    }
}

// Warp-wide sums of eight FP32 values per lane in a fixed order (a reduce-scatter
// butterfly, seven shuffles instead of eight five-level trees): lane l returns the warp
// total of value (l >> 2) & 7.
__device__ __forceinline__ float warp_sum8_scatter_f32(const float (&v)[8]) {
    const int lane = threadIdx.x & 31;
    const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
    float k4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float keep = b4 ? v[4 + i] : v[i];
        const float give = b4 ? v[i] : v[4 + i];
        k4[i] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
    float k2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float keep = b3 ? k4[2 + i] : k4[i];
        const float give = b3 ? k4[i] : k4[2 + i];
        k2[i] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
    float k1 = (b2 ? k2[1] : k2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? k2[0] : k2[1], 4);
    k1 += __shfl_xor_sync(0xffffffffu, k1, 2);
    k1 += __shfl_xor_sync(0xffffffffu, k1, 1);
    return k1;
}

// Rows of one narrow tile packed into warp iterations: a lane's kNarrowSlots float4 slots
// serve R = kNarrowSlots >> lg rows of the group (slot kk: row kk >> lg, column chunk
// kk & (2^lg - 1)), lg = 0 for at most 128 valid columns, 1 for at most 256.  A warp
// iteration thus moves up to 4 KB of X and as much of C (eight rows of 128 columns, or four
// of 256).  Slot kk touches the columns of chunk kk & 1 when
// lg = 1 and of chunk 0 when lg = 0, so a lane keeps psi and its FP32 column partials for
// two chunks (indexed kk & 1) whatever the number of slots; with lg = 0 both halves hold
// chunk 0 and are added together when they are promoted to FP64.
constexpr int kNarrowCols = 256;
constexpr int kNarrowSlots = 8;
// warp iterations between FP32 -> FP64 promotions: every column partial then holds
// kFlushRows rows, as in the wide-tile kernel (each half takes four rows per iteration)
constexpr int kNarrowFlushIters = kFlushRows / (kNarrowSlots / 2);
static_assert(kNarrowFlushIters * (kNarrowSlots / 2) == kFlushRows, "flush interval");

// Fused DR pass over the narrow tiles of every active problem (UPDATE = false: sums of X_0).
// Launched right after drot_batched_step_kernel as its programmatic dependent: it does not
// wait for that kernel to begin (it reads only what the finish before both wrote, through
// L2), and it waits for it before ending, so the finish launched after this kernel sees the
// totals of both.
template <bool UPDATE>
__global__ void __launch_bounds__(kThreads, 2) drot_batched_narrow_kernel(BatchArgs B) {
    constexpr int S = kNarrowSlots;
    __shared__ double s_col[kWarps][kNarrowCols];
    __shared__ double s_red[kWarps][2];
    __shared__ float s_psi[kNarrowCols];
    __shared__ float s_phi[kPhiChunk];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long w0 = B.wbound_n[blockIdx.x];
    const long long w1 = B.wbound_n[blockIdx.x + 1];
    const int nactive = __ldcg(B.nactive_n);
    if (w0 < w1 && nactive > 0) {
        const bool rev = B.serp != 0 && ((__ldcg(B.parity) + B.odd) & 1) != 0;
        const long long wfirst = rev ? w1 - 1 : w0;
        int lo = 0, hi = nactive - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B.unit0_n[mid] <= wfirst) lo = mid;
            else hi = mid - 1;
        }
        int ai = lo;
        long long w = rev ? w1 : w0;
        while (rev ? w > w0 : w < w1) {
            if (rev) {
                while (ai > 0 && w - 1 < B.unit0_n[ai]) --ai;
            } else {
                while (ai + 1 < nactive && w >= B.unit0_n[ai + 1]) ++ai;
            }
            const BatchProb& P = B.probs[B.active_n[ai]];
            const long long base = B.unit0_n[ai];
            const long long m = P.m, n = P.n, ld = P.ld;
            const long long tl = ((rev ? w - 1 : w) - base) / m;
            const long long seg_lo = rev ? max(w0, base + tl * m) : w;
            const long long seg_hi = rev ? w : min(w1, base + (tl + 1) * m);
            const long long i0 = seg_lo - base - tl * m, i1 = seg_hi - base - tl * m;
            w = rev ? seg_lo : seg_hi;
            if (__ldcg(&P.sc->done) != kRunning) continue;  // uniform: every thread reads the same flag

            const int TW = 128 * P.K;
            const long long col0 = (P.Tw + tl) * TW;
            const int wcols = (int)min((long long)TW, n - col0);  // <= kNarrowCols
            const int lg = wcols <= 128 ? 0 : 1;
            const int cmask = (1 << lg) - 1;
            const int R = S >> lg;
            const double cs = __ldcg(&P.sc->c);
            const float rho = UPDATE ? (float)P.sc->rho : 0.f;

            // every thread arrives here together (the previous segment ended with a barrier)
            if (UPDATE) {
                for (int x = threadIdx.x; x < wcols; x += kThreads)
                    s_psi[x] = (float)((__ldcg(P.h + col0 + x) + cs) * P.inv_m);
            }
            for (int x = lane; x < kNarrowCols; x += 32) s_col[warp][x] = 0.0;
            float psi[2][4], cacc[2][4];
            float scx = 0.f, sd = 0.f;
            double scx64 = 0.0, sd64 = 0.0;
            int since_flush = 0;
            const long long c_first = rev ? i1 : i0;
            for (long long c = c_first; rev ? c > i0 : c < i1; c += rev ? -kPhiChunk : kPhiChunk) {
            const long long r0 = rev ? max(i0, c - (long long)kPhiChunk) : c;
            const long long r1 = rev ? c : min(i1, c + (long long)kPhiChunk);
            if (UPDATE) {
                if (c != c_first) __syncthreads();  // every warp is done with the previous chunk's phi
                for (long long r = r0 + threadIdx.x; r < r1; r += kThreads)
                    s_phi[r - r0] = (float)((__ldcg(P.g + r) + cs) * P.inv_n);
            }
            __syncthreads();
            if (c == c_first) {
#pragma unroll
                for (int hh = 0; hh < 2; ++hh)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int x = (hh & cmask) * 128 + lane * 4 + e;
                        psi[hh][e] = (UPDATE && x < wcols) ? s_psi[x] : 0.f;
                        cacc[hh][e] = 0.f;
                    }
            }
            // slot kk holds the row at chunk offset q + dstep (kk >> lg), valid while in [0, nr)
            const int nr = (int)(r1 - r0);
            const int dstep = rev ? -kWarps : kWarps;
            float* const Xc = P.X + r0 * ld + col0;
            const float* const Cc = P.C + r0 * ld + col0;
            for (int q = rev ? nr - 1 - warp : warp; (unsigned)q < (unsigned)nr; q += R * dstep) {
                float4 xv[S], cv[S];
#pragma unroll
                for (int kk = 0; kk < S; ++kk) {
                    const int rq = q + dstep * (kk >> lg);
                    const int jl = (kk & cmask) * 128 + lane * 4;
                    if ((unsigned)rq < (unsigned)nr && jl < wcols) {
                        const long long off = (long long)rq * ld + jl;
                        xv[kk] = *reinterpret_cast<const float4*>(Xc + off);
                        if (UPDATE) cv[kk] = ld_stream_ro(Cc + off);
                    }
                }
                if (UPDATE) {
                    // the rows of the warp's next iteration into L2 (R rows x 2^(lg+2) lines x 2 arrays = 64)
                    const int qn = q + R * dstep;
                    const int lines = 4 << lg;
#pragma unroll
                    for (int t0 = 0; t0 < 64; t0 += 32) {
                        const int t = t0 + lane;
                        const int arr = t >> 5, rem = t & 31;
                        const int rq = qn + dstep * (rem >> (2 + lg));
                        const int line = rem & (lines - 1);
                        if ((unsigned)rq < (unsigned)nr && line * 32 < wcols) {
                            const float* pf = (arr ? Cc : Xc) + (long long)rq * ld + line * 32;
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(pf));
                        }
                    }
                }
                float rsk[S];
#pragma unroll
                for (int kk = 0; kk < S; ++kk) {
                    rsk[kk] = 0.f;
                    const int rq = q + dstep * (kk >> lg);
                    const int jl = (kk & cmask) * 128 + lane * 4;
                    if ((unsigned)rq < (unsigned)nr && jl < wcols) {
                        const float phi = UPDATE ? s_phi[rq] : 0.f;
                        float xs[4] = {xv[kk].x, xv[kk].y, xv[kk].z, xv[kk].w};
                        float cc[4] = {0.f, 0.f, 0.f, 0.f};
                        if (UPDATE) { cc[0] = cv[kk].x; cc[1] = cv[kk].y; cc[2] = cv[kk].z; cc[3] = cv[kk].w; }
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if (jl + e < wcols) {
                                float xn = xs[e];
                                if (UPDATE) {
                                    const float d = fmaf(-rho, cc[e], phi + psi[kk & 1][e]);
                                    xn = fmaxf(xs[e] + d, 0.f);
                                    scx = fmaf(cc[e], xn, scx);
                                    const float dp = fmaxf(d, 0.f);
                                    sd = fmaf(dp, dp, sd);
                                    xs[e] = xn;
                                }
                                rsk[kk] += xn;
                                cacc[kk & 1][e] += xn;
                            }
                        }
                        if (UPDATE) {
                            float* dst = Xc + (long long)rq * ld + jl;
                            if (jl + 3 < wcols) {
                                *reinterpret_cast<float4*>(dst) = make_float4(xs[0], xs[1], xs[2], xs[3]);
                            } else {
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    if (jl + e < wcols) dst[e] = xs[e];
                            }
                        }
                    }
                }
                // lanes 4g .. 4g+3 receive the warp total of slot g; a row owns 2^lg slots
                float tot = warp_sum8_scatter_f32(rsk);
                if (lg == 1) tot += __shfl_xor_sync(0xffffffffu, tot, 4);
                const int rq = q + dstep * (lane >> (2 + lg));
                if ((lane & ((4 << lg) - 1)) == 0 && (unsigned)rq < (unsigned)nr)
                    atomicAdd(P.u + r0 + rq, (double)tot);
                if (++since_flush == kNarrowFlushIters) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (lg == 0) {
                            s_col[warp][lane * 4 + e] += (double)cacc[0][e] + (double)cacc[1][e];
                        } else {
                            s_col[warp][lane * 4 + e] += (double)cacc[0][e];
                            s_col[warp][128 + lane * 4 + e] += (double)cacc[1][e];
                        }
                        cacc[0][e] = 0.f;
                        cacc[1][e] = 0.f;
                    }
                    scx64 += (double)scx;
                    sd64 += (double)sd;
                    scx = 0.f;
                    sd = 0.f;
                    since_flush = 0;
                }
            }
            }  // row chunks
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (lg == 0) {
                    s_col[warp][lane * 4 + e] += (double)cacc[0][e] + (double)cacc[1][e];
                } else {
                    s_col[warp][lane * 4 + e] += (double)cacc[0][e];
                    s_col[warp][128 + lane * 4 + e] += (double)cacc[1][e];
                }
            }
            scx64 += (double)scx;
            sd64 += (double)sd;
            __syncthreads();
            for (int x = threadIdx.x; x < wcols; x += kThreads) {
                double v = 0.0;
#pragma unroll
                for (int wv = 0; wv < kWarps; ++wv) v += s_col[wv][x];
                atomicAdd(P.v + col0 + x, v);
            }
            if (UPDATE) {
                double v2[2] = {scx64, sd64};
                block_sum_f64<2, kThreads>(v2, s_red);  // ends with a block barrier
                if (threadIdx.x == 0) {
                    atomicAdd(acc_at(P.acc, 0), v2[0]);
                    atomicAdd(acc_at(P.acc, 1), v2[1]);
                }
            } else {
                __syncthreads();
            }
        }
    }
    // end only after the wide-tile pass launched before this kernel (a no-op when this
    // kernel was not launched as a programmatic dependent)
    wait_for_predecessor();
}

// Steps 5-8 and the stopping test of every active problem (one block group each).
// Blocks of kBatchFinishThreads threads, one per kBatchFinishElems elements of a
// problem (four per thread): a batch of hundreds of problems would otherwise launch
// tens of thousands of small blocks per iteration, and the block launch rate, not the
// work, would set the finish's length (117 us per iteration for 512 problems).
constexpr int kBatchFinishThreads = 256;
constexpr int kBatchFinishElems = 4 * kBatchFinishThreads;
__global__ void __launch_bounds__(kBatchFinishThreads) drot_batched_finish_kernel(BatchArgs B) {
    wait_for_predecessor();
    const int pi = B.fin_prob[blockIdx.x];
    if (pi < 0) return;
    const BatchProb& P = B.probs[pi];
    if (P.sc->done != kRunning) return;
    finish_body<kBatchFinishThreads>(batch_finish_args(P), B.fin_local[blockIdx.x], P.fin_blocks);
}

// a_0, b_0, alpha_0 and the numerators of phi_0, psi_0 of every active problem.
__global__ void __launch_bounds__(kFinishThreads) drot_batched_init_state_kernel(BatchArgs B) {
    const int pi = B.fin_prob[blockIdx.x];
    if (pi < 0) return;
    const BatchProb& P = B.probs[pi];
    init_state_body(batch_finish_args(P), B.warm ? P.mu : nullptr, B.warm ? P.nu : nullptr,
                    B.fin_local[blockIdx.x], P.fin_blocks);
}

// Marginal (and warm-dual) sums: one block per problem of the batch.
__global__ void __launch_bounds__(1024) drot_batched_vector_sums_kernel(const BatchProb* probs, int warm) {
    const BatchProb& P = probs[blockIdx.x];
    __shared__ double s_red[32][6];
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long i = threadIdx.x; i < P.m; i += blockDim.x) {
        v[0] += P.p[i];
        if (!(P.p[i] >= 0.0) || !isfinite(P.p[i])) v[4] += 1.0;
        if (warm) v[2] += P.mu[i];
    }
    for (long long j = threadIdx.x; j < P.n; j += blockDim.x) {
        v[1] += P.q[j];
        if (!(P.q[j] >= 0.0) || !isfinite(P.q[j])) v[5] += 1.0;
        if (warm) v[3] += P.nu[j];
    }
    block_sum_f64<6, 1024>(v, s_red);
    if (threadIdx.x == 0) {
        Scalars* sc = P.sc;
        sc->sum_p = v[0];
        sc->sum_q = v[1];
        sc->sum_phi0 = sc->rho * v[2];
        sc->sum_psi0 = sc->rho * v[3];
        sc->nonfinite_input = (v[4] > 0.0 ? 1 : 0) | (v[5] > 0.0 ? 2 : 0) |
                              ((isfinite(v[2]) && isfinite(v[3])) ? 0 : 4);
    }
}

// X_0 = p q^T for every problem flagged in `cold` (blockIdx.y = problem).
__global__ void drot_batched_init_plan_kernel(const BatchProb* probs, const int* cold) {
    const BatchProb& P = probs[blockIdx.y];
    if (!cold[blockIdx.y]) return;
    const long long m = P.m, n = P.n, ld = P.ld;
    const long long nv = (n + 3) / 4;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < m * nv;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx / nv;
        const long long j = (idx - i * nv) * 4;
        const double pi = P.p[i];
        float* dst = P.X + i * ld + j;
        if (j + 3 < n) {
            *reinterpret_cast<float4*>(dst) = make_float4((float)(pi * P.q[j]), (float)(pi * P.q[j + 1]),
                                                          (float)(pi * P.q[j + 2]), (float)(pi * P.q[j + 3]));
        } else {
            for (int e = 0; e < 4; ++e)
                if (j + e < n) dst[e] = (float)(pi * P.q[j + e]);
        }
    }
}

// mu = phi / rho, nu = psi / rho and nnz(X) of every problem (blockIdx.y = problem).
__global__ void drot_batched_export_kernel(const BatchProb* probs, const int* live) {
    const BatchProb& P = probs[blockIdx.y];
    if (!live[blockIdx.y]) return;
    const Scalars* sc = P.sc;
    const double c = sc->c, rho = sc->rho;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < P.m + P.n;
         idx += (long long)gridDim.x * blockDim.x) {
        if (idx < P.m) P.mu[idx] = (P.g[idx] + c) * P.inv_n / rho;
        else P.nu[idx - P.m] = (P.h[idx - P.m] + c) * P.inv_m / rho;
    }
    unsigned long long cnt = 0;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < P.m * P.n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx / P.n, j = idx - i * P.n;
        cnt += P.X[i * P.ld + j] > 0.f ? 1ull : 0ull;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&P.sc->nnz, cnt);
}

}  // namespace drot
