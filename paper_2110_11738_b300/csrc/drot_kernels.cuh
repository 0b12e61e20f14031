// Device code of the DROT solver for sm_103a.
//
// One DROT iteration (Algorithm 1, Sec. 3.1) is two launches:
//
//   drot_step_kernel    the fused pass over the dense plan: step 4
//                         x <- max(x + phi_i + psi_j - rho c_ij, 0)
//                       in place, with the partial reductions the rest of the
//                       iteration needs taken on the fly (row sums, column sums,
//                       <C, X_{k+1}>, and ||[phi_k + psi_j - rho C]_+||_F^2 for the
//                       dual residual of the stopping test, Sec. 3.1).  Each entry
//                       of X and C is read once and X written once: 12 bytes per
//                       entry, the whole HBM cost of the iteration.
//   drot_finish_kernel  the O(m + n) vector work: finishes the row and column sums
//                       from the per-tile partials, forms r, s, beta and the updates
//                       of steps 6-8, the stopping quantities, and the convergence
//                       flag.  The last block to finish (a ticket counter, no
//                       waiting) does the scalar part.
//
// The vectors are carried as FP64 numerators so that the step reads one double
// per row and per column:  phi_k = (g + c_k) / n,  psi_k = (h + c_k) / m,  with
// g = a_{k-1} - 2 r_k, h = b_{k-1} - 2 s_k and the scalar c_k = 2 beta_k - alpha_{k-1}
// (steps 6-7 rewritten).  All cross-thread sums are FP64 and taken in a fixed
// order, so a solve is bitwise reproducible for a fixed launch plan.
//
// Work decomposition of the fused step.  Columns are cut into tiles of
// TW = 128*K floats (K float4 per lane); a "row segment" is one row of one tile.
// Segments are numbered tile-major (w = t*m + i) and each CTA takes one
// contiguous range of segments whose boundaries the host balances by bytes.  Inside
// a CTA the 8 warps take interleaved rows, so at any time a CTA streams 8
// neighbouring row segments of X and C with 128-bit coalesced loads.  Consecutive
// passes walk the ranges in opposite directions (SegWalk), so that each pass starts on
// what the previous one left in L2.  Row sums
// are reduced with warp shuffles and written once per segment (rowpart[t][i]);
// column sums accumulate in registers, are promoted to FP64 in shared memory every
// few rows, reduced across warps and written once per (CTA, tile) ("slot").
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace drot {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kFlushRows = 16;   // rows per warp between FP32 -> FP64 promotions
constexpr int kPhiChunk = 4096;  // rows whose phi a CTA forms at once (a multiple of kWarps)
// Finish blocks are small so that the O(m + n) FP64 work (B300's FP64 rate is a
// small fraction of its FP32 rate) spreads over every SM.
constexpr int kFinishThreads = 64;
constexpr int kFinishAcc = 6;
// The FP64 totals of accumulation mode (<C,X>, sum [d]_+^2 and the six finish totals)
// sit one per 128-byte line, so that the atomics aimed at different totals are spread
// over L2 slices instead of queueing on one.
constexpr int kAccSlots = 8;
constexpr int kAccStride = 16;
__device__ __forceinline__ double* acc_at(double* acc, int c) { return acc + c * kAccStride; }

enum DoneCode : int { kRunning = 0, kConverged = 1, kIterCap = 2, kNonFinite = 3, kFault = 4 };

// Device-resident scalar state of one solve.
struct Scalars {
    double c;              // scalar term of phi_k, psi_k (see above)
    double alpha;          // alpha_k
    double rho;
    double inv_rho;        // 1 / rho (set with rho; avoids FP64 divisions on the device)
    double tol;
    double sum_p, sum_q;
    double min_p, min_q;
    double sum_phi0, sum_psi0;
    double primal, dual, gap, res_l1, res_l2, dual_res_prev, beta;
    long long k;           // iterations completed
    long long max_iter;
    int done;              // DoneCode
    int stop_rule;         // DROT_STOP_* bitmask (never 0)
    int nonfinite_input;   // set by the marginal check
    unsigned int counter;  // finish-kernel ticket counter, reset by the last block
    int fault;             // set when a bounded device-side wait gave up
    unsigned long long nnz;
};

struct StepArgs {
    const float* C;
    float* X;
    const double* g;            // phi numerators (m)
    const double* h;            // psi numerators (n)
    const Scalars* sc;
    double* rowpart;            // [T][m]
    double* colpart;            // [slots][TW]
    double* ctapart;            // [G][2]: <C,X> and sum [d]_+^2 per CTA
    double* u;                  // accumulation mode: row totals (m), added with FP64 atomics
    double* v;                  // accumulation mode: column totals (n)
    double* acc;                // accumulation mode: [8] <C,X>, sum [d]_+^2 (added here), finish totals
    int accumulate;             // 1: atomics into u, v, acc; 0: fixed-order partials
    int serp;                   // 1: alternate the direction of the passes (see SegWalk)
    int odd;                    // parity of this pass in its launch sequence; backwards when serp && odd
    const long long* wbound;    // [G+1] segment range of each CTA
    const int* slot_base;       // [G]   first slot of each CTA
    long long m, n, ld;
    double inv_n, inv_m;
};

// Programmatic dependent launch: wait until the preceding kernel of the stream has
// completed and its writes are visible (returns at once when the kernel was not
// launched as a programmatic dependent).
__device__ __forceinline__ void wait_for_predecessor() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next kernel of the stream (launched as a programmatic dependent) start its
// blocks now; it still waits in griddepcontrol.wait for this whole grid to finish.
__device__ __forceinline__ void release_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp-wide sums of eight FP64 values per lane with nine FP64 additions per lane, in a
// fixed order (a reduce-scatter butterfly): at offsets 16, 8 and 4 a lane keeps half
// of its running values, receives its partner's copies of them and adds; offsets 2
// and 1 finish the one value left.  Lane l returns the warp total of value
// (l >> 2) & 7.  A plain shuffle tree would take 8 x 5 = 40 additions; a dependent
// FP64 add is slow on this GPU, so the tree sat on the critical path of every finish.
__device__ __forceinline__ double warp_sum8_scatter(const double (&v)[8]) {
    const int lane = threadIdx.x & 31;
    const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
    double k4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const double keep = b4 ? v[4 + i] : v[i];
        const double give = b4 ? v[i] : v[4 + i];
        k4[i] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
    double k2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const double keep = b3 ? k4[2 + i] : k4[i];
        const double give = b3 ? k4[i] : k4[2 + i];
        k2[i] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
    double k1 = (b2 ? k2[1] : k2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? k2[0] : k2[1], 4);
    k1 += __shfl_xor_sync(0xffffffffu, k1, 2);
    k1 += __shfl_xor_sync(0xffffffffu, k1, 1);
    return k1;
}

// Partial-sum sinks of the fused step.  Fixed-order mode writes one partial per
// (column tile, row), per (CTA, tile) and per CTA, each with a single writer, for
// the finish kernel to add in a fixed order (bitwise reproducible).  Accumulation
// mode adds them into the totals with FP64 atomic adds as they are produced, so
// the finish kernel reads one value per row and column.
struct StepArgs;

// Block-wide sum of NV doubles in a fixed order; result valid in thread 0.
template <int NV, int NT>
__device__ __forceinline__ void block_sum_f64(double (&v)[NV], double (*scratch)[NV]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = warp_sum_f64(v[c]);
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < NV; ++c) scratch[warp][c] = v[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w) s += scratch[w][c];
            v[c] = s;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ float4 ld_stream_ro(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}

// The row segments of one CTA, [w0, w1) in tile-major numbering, walked forwards or
// backwards.  Serpentine order: a pass that walks backwards (tiles, and rows within a
// tile, in reverse) starts on the lines of X and C that the forward pass before it
// touched last, which are still in L2 when the plan is a few times larger than L2.
// Forwards, the k-th row of a segment visited is i0 + k; backwards it is i1 - 1 - k,
// and warp w takes the k = w + kWarps j in both cases.  Column-partial slots keep
// their tile: a backward walk starts at the CTA's last slot.
struct SegWalk {
    long long w0, w1, m;
    bool rev;
    __device__ __forceinline__ long long start() const { return rev ? w1 : w0; }
    __device__ __forceinline__ bool more(long long w) const { return rev ? w > w0 : w < w1; }
    // tile t and rows [i0, i1) of the segment at position w of the walk
    __device__ __forceinline__ void seg(long long w, long long& t, long long& i0, long long& i1) const {
        t = (rev ? w - 1 : w) / m;
        const long long lo = rev ? max(w0, t * m) : w;
        const long long hi = rev ? w : min(w1, (t + 1) * m);
        i0 = lo - t * m;
        i1 = hi - t * m;
    }
    __device__ __forceinline__ long long next(long long t, long long i0, long long i1) const {
        return t * m + (rev ? i0 : i1);
    }
    __device__ __forceinline__ int first_slot(int base) const {
        return base + ((rev && w1 > w0) ? (int)((w1 - 1) / m - w0 / m) : 0);
    }
    __device__ __forceinline__ long long row(long long i0, long long i1, long long k) const {
        return rev ? i1 - 1 - k : i0 + k;
    }
};

// The fused DR pass (UPDATE = true) or a plain row/column-sum pass over X
// (UPDATE = false, used once to initialise a_0 and b_0 from the stored X_0).
// C-load skipping (Claim 1, Sec. 3.3): CM = 0 is the plain pass; CM = 1 reads X and C
// and stores W = x+ - rho c instead of x+; CM = 2 reads W (no C) and forms
// x+ = [W + phi + psi]_+.  A CM = 1 / CM = 2 pair moves 12 + 8 bytes per entry;
// <C,X> and the dual residual need C and are only produced by CM = 0 / 1 passes.
// Shared memory of the register-fed pass, declared by the kernel that runs it.
template <int K>
struct StepSmem {
    double col[kWarps][128 * K];
    double red[kWarps][2];
    // psi of the tile's columns and phi of a chunk of rows, formed once per CTA: a warp
    // would otherwise compute its own copy of all of them in FP64, whose throughput on
    // this GPU (a warp-wide FP64 instruction holds a sub-partition's pipe ~80 cycles)
    // made the per-warp copies a burst of ~5 us at every tile start
    float psi[128 * K];
    float phi[kPhiChunk];
};

template <int K, bool UPDATE, int CM>
__device__ __forceinline__ void step_pass(const StepArgs& A, int cta, StepSmem<K>& sm, const bool rev) {
    constexpr int TW = 128 * K;
    auto& s_col = sm.col;
    auto& s_red = sm.red;
    float* s_psi = sm.psi;
    float* s_phi = sm.phi;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long m = A.m, n = A.n, ld = A.ld;
    const long long w0 = A.wbound[cta];
    const long long w1 = A.wbound[cta + 1];
    const float rho = UPDATE ? (float)A.sc->rho : 0.f;
    const double cs = __ldcg(&A.sc->c);
    const SegWalk walk{w0, w1, m, rev};
    int slot = walk.first_slot(A.slot_base[cta]);
    double scx64 = 0.0, sd64 = 0.0;

    for (long long w = walk.start(); walk.more(w);) {
        long long t, i0, i1;
        walk.seg(w, t, i0, i1);
        const long long col0 = t * TW;

        // every thread arrives here together (the previous segment ended with a barrier)
        if (UPDATE) {
            for (int x = threadIdx.x; x < TW; x += kThreads) {
                const long long j = col0 + x;
                s_psi[x] = j < n ? (float)((__ldcg(A.h + j) + cs) * A.inv_m) : 0.f;
            }
        }
        float psi[K][4], cacc[K][4];
        for (int x = lane; x < TW; x += 32) s_col[warp][x] = 0.0;

        float scx = 0.f, sd = 0.f;
        int since_flush = 0;
        // rows in chunks of kPhiChunk (a multiple of kWarps, so warp w keeps the rows
        // k = w + kWarps j of the whole segment, in the same order); the chunk edge c
        // is the chunk's first row forwards and one past its last row backwards
        const long long c_first = rev ? i1 : i0;
        for (long long c = c_first; rev ? c > i0 : c < i1; c += rev ? -kPhiChunk : kPhiChunk) {
        const long long r0 = rev ? max(i0, c - (long long)kPhiChunk) : c;
        const long long r1 = rev ? c : min(i1, c + (long long)kPhiChunk);
        if (UPDATE) {
            if (c != c_first) __syncthreads();  // every warp is done with the previous chunk's phi
            for (long long r = r0 + threadIdx.x; r < r1; r += kThreads)
                s_phi[r - r0] = (float)((__ldcg(A.g + r) + cs) * A.inv_n);
        }
        __syncthreads();
        if (c == c_first) {
#pragma unroll
            for (int kk = 0; kk < K; ++kk)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    psi[kk][e] = UPDATE ? s_psi[kk * 128 + lane * 4 + e] : 0.f;
                    cacc[kk][e] = 0.f;
                }
        }
        for (long long i = rev ? r1 - 1 - warp : r0 + warp; rev ? i >= r0 : i < r1; i += rev ? -kWarps : kWarps) {
            const float phi = UPDATE ? s_phi[i - r0] : 0.f;
            const long long rowoff = i * ld + col0 + lane * 4;
            float4 xv[K], cv[K];
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                if (col0 + kk * 128 + lane * 4 < n) {
                    xv[kk] = *reinterpret_cast<const float4*>(A.X + rowoff + kk * 128);
                    if (UPDATE && CM != 2) cv[kk] = ld_stream_ro(A.C + rowoff + kk * 128);
                }
            }
            float rs = 0.f;
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                const long long j = col0 + kk * 128 + lane * 4;
                if (j < n) {
                    float xs[4] = {xv[kk].x, xv[kk].y, xv[kk].z, xv[kk].w};
                    float cc[4] = {0.f, 0.f, 0.f, 0.f};
                    if (UPDATE && CM != 2) { cc[0] = cv[kk].x; cc[1] = cv[kk].y; cc[2] = cv[kk].z; cc[3] = cv[kk].w; }
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (j + e < n) {
                            float xn = xs[e];
                            if (UPDATE && CM == 2) {
                                xn = fmaxf(xs[e] + (phi + psi[kk][e]), 0.f);  // xs holds W = X - rho C
                                xs[e] = xn;
                            } else if (UPDATE) {
                                const float d = fmaf(-rho, cc[e], phi + psi[kk][e]);
                                xn = fmaxf(xs[e] + d, 0.f);
                                scx = fmaf(cc[e], xn, scx);
                                const float dp = fmaxf(d, 0.f);
                                sd = fmaf(dp, dp, sd);
                                xs[e] = CM == 1 ? fmaf(-rho, cc[e], xn) : xn;  // CM 1 stores W
                            }
                            rs += xn;
                            cacc[kk][e] += xn;
                        }
                    }
                    if (UPDATE) {
                        float* dst = A.X + rowoff + kk * 128;
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
            if (lane == 0) {
                if (A.accumulate) atomicAdd(A.u + i, (double)rs);
                else A.rowpart[t * m + i] = (double)rs;
            }
            if (++since_flush == kFlushRows) {
#pragma unroll
                for (int kk = 0; kk < K; ++kk)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
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
        for (int kk = 0; kk < K; ++kk)
#pragma unroll
            for (int e = 0; e < 4; ++e) s_col[warp][kk * 128 + lane * 4 + e] += (double)cacc[kk][e];
        scx64 += (double)scx;
        sd64 += (double)sd;
        __syncthreads();
        double* out = A.colpart + (long long)slot * TW;
        for (int x = threadIdx.x; x < TW; x += kThreads) {
            double v = 0.0;
#pragma unroll
            for (int wv = 0; wv < kWarps; ++wv) v += s_col[wv][x];
            if (!A.accumulate) out[x] = v;
            else if (col0 + x < n) atomicAdd(A.v + col0 + x, v);
        }
        __syncthreads();
        slot += rev ? -1 : 1;
        w = walk.next(t, i0, i1);
    }

    if (UPDATE) {
        double v[2] = {scx64, sd64};
        block_sum_f64<2, kThreads>(v, s_red);
        if (threadIdx.x == 0) {
            if (A.accumulate) {
                atomicAdd(acc_at(A.acc, 0), v[0]);
                atomicAdd(acc_at(A.acc, 1), v[1]);
            } else {
                A.ctapart[2 * cta + 0] = v[0];
                A.ctapart[2 * cta + 1] = v[1];
            }
        }
    }
}

template <int K, bool UPDATE, int CM = 0>
__device__ __forceinline__ void step_body(const StepArgs& A, int cta, bool rev) {
    __shared__ StepSmem<K> sm;
    step_pass<K, UPDATE, CM>(A, cta, sm, rev);
}

template <int K, bool UPDATE, int CM = 0>
__global__ void __launch_bounds__(kThreads, 2) drot_step_kernel(StepArgs A) {
    wait_for_predecessor();
    if (A.sc->done != kRunning) return;
    step_body<K, UPDATE, CM>(A, blockIdx.x, A.serp != 0 && A.odd != 0);
}

// X = W + rho C: restores the plan after a solve that stopped on a C-reading pass of
// the C-skipping schedule (the array then holds W = X - rho C, rounded to FP32).  An
// entry that was 0 comes back as the rounding error of rho c, at most 2^-24 rho c in
// magnitude; results at or below 2^-22 rho c are therefore set to 0, so X stays
// nonnegative and keeps its zeros.
__global__ void drot_restore_plan_kernel(float* X, const float* C, long long m, long long n, long long ld,
                                         const Scalars* sc) {
    const float rho = (float)sc->rho;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx / n, j = idx - i * n;
        const float rc = rho * C[i * ld + j];
        const float x = fmaf(rho, C[i * ld + j], X[i * ld + j]);
        X[i * ld + j] = x > rc * 2.384185791015625e-07f ? x : 0.f;  // 2^-22
    }
}


// ------------------------------------------------------------------ TMA-fed variant
//
// Same arithmetic, partials and work split as drot_step_kernel<K, true>, but the
// row segments of X and C reach shared memory through 1-D bulk copies
// (cp.async.bulk, the TMA engine) into an S-stage ring, so the bytes in flight per
// SM do not depend on registers or occupancy.  One producer warp (one elected
// lane) issues the copies of 8 row segments per stage and signals a "full"
// mbarrier with the byte count; the 8 consumer warps each take one row of the
// stage, compute x+ from shared memory, store it to global memory with 128-bit
// stores, and arrive on the stage's "empty" mbarrier.  Every wait is bounded:
// after kWaitLimit polls the kernel records a fault in Scalars and returns.

constexpr uint32_t kWaitLimit = 1u << 20;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity to complete; false on timeout
// or when another warp of the block has already given up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 1023u) == 1023u && *abort_flag) return false;
    }
    return false;
}

__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void consumer_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
}

template <int K, int S>
struct TmaLayout {
    static constexpr int TW = 128 * K;
    static constexpr size_t stage_floats = (size_t)kWarps * TW;
    static constexpr size_t bytes = 2 * S * stage_floats * sizeof(float)   // X and C rings
                                    + (size_t)kWarps * TW * sizeof(double)  // column accumulators
                                    + 2 * S * sizeof(uint64_t);             // full / empty barriers
};

template <int K, int S>
__global__ void __launch_bounds__(kThreads + 32, 1) drot_step_tma_kernel(StepArgs A) {
    constexpr int TW = 128 * K;
    constexpr int R = kWarps;  // rows per stage, one per consumer warp
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* sX = reinterpret_cast<float*>(smem_raw);
    float* sC = sX + (size_t)S * R * TW;
    double* s_col = reinterpret_cast<double*>(sC + (size_t)S * R * TW);
    uint64_t* full = reinterpret_cast<uint64_t*>(s_col + kWarps * TW);
    uint64_t* empty = full + S;
    __shared__ double s_red[kWarps + 1][2];
    __shared__ int s_abort;
    __shared__ uint32_t s_issued;

    wait_for_predecessor();
    if (A.sc->done != kRunning) return;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long m = A.m, n = A.n, ld = A.ld;
    const long long w0 = A.wbound[blockIdx.x];
    const long long w1 = A.wbound[blockIdx.x + 1];
    const SegWalk walk{w0, w1, m, A.serp != 0 && A.odd != 0};
    if (threadIdx.x == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], kWarps);
        }
        s_abort = 0;
        s_issued = 0;
        fence_mbar_init();
    }
    __syncthreads();

    double scx64 = 0.0, sd64 = 0.0;
    bool ok = true;

    if (warp == kWarps) {
        // ---------------- producer: one lane issues every bulk copy
        if (lane == 0) {
            uint32_t g = 0;
            for (long long w = walk.start(); walk.more(w) && ok;) {
                long long t, i0, i1;
                walk.seg(w, t, i0, i1);
                const long long col0 = t * TW;
                const long long cols = min((long long)TW, n - col0);
                const uint32_t bytes = (uint32_t)(((cols + 3) / 4) * 16);
                // stage g holds the segment's rows k0 .. k0 + R - 1 in walk order
                for (long long k0 = 0; k0 < i1 - i0; k0 += R, ++g) {
                    const int st = (int)(g % S);
                    const uint32_t use = g / S;
                    if (!mbar_wait(&empty[st], (use & 1u) ^ 1u, &s_abort)) {
                        ok = false;
                        break;
                    }
                    const int rows = (int)min((long long)R, i1 - i0 - k0);
                    mbar_arrive_expect_tx(&full[st], (uint32_t)rows * 2u * bytes);
                    for (int rr = 0; rr < rows; ++rr) {
                        const long long off = walk.row(i0, i1, k0 + rr) * ld + col0;
                        bulk_load(sX + ((size_t)st * R + rr) * TW, A.X + off, bytes, &full[st]);
                        bulk_load(sC + ((size_t)st * R + rr) * TW, A.C + off, bytes, &full[st]);
                    }
                }
                w = walk.next(t, i0, i1);
            }
            s_issued = g;
            if (!ok) {
                s_abort = 1;
                atomicExch(const_cast<int*>(&A.sc->fault), 1);
            }
        }
        __syncwarp();
    } else {
        // ---------------- consumers
        const double cs = A.sc->c;
        const float rho = (float)A.sc->rho;
        int slot = walk.first_slot(A.slot_base[blockIdx.x]);
        uint32_t g = 0;
        for (long long w = walk.start(); walk.more(w);) {
            long long t, i0, i1;
            walk.seg(w, t, i0, i1);
            const long long col0 = t * TW;

            float psi[K][4], cacc[K][4];
#pragma unroll
            for (int kk = 0; kk < K; ++kk)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const long long j = col0 + kk * 128 + lane * 4 + e;
                    psi[kk][e] = j < n ? (float)((A.h[j] + cs) * A.inv_m) : 0.f;
                    cacc[kk][e] = 0.f;
                }
            for (int x = lane; x < TW; x += 32) s_col[warp * TW + x] = 0.0;
            __syncwarp();

            float scx = 0.f, sd = 0.f;
            int since_flush = 0;
            for (long long k0 = 0; k0 < i1 - i0; k0 += R, ++g) {
                const int st = (int)(g % S);
                const uint32_t use = g / S;
                if (ok && !mbar_wait(&full[st], use & 1u, &s_abort)) {
                    ok = false;
                    if (lane == 0) {
                        s_abort = 1;
                        atomicExch(const_cast<int*>(&A.sc->fault), 1);
                    }
                }
                const long long i = walk.row(i0, i1, k0 + warp);
                if (ok && k0 + warp < i1 - i0) {
                    const float phi = (float)((A.g[i] + cs) * A.inv_n);
                    const float* xs_row = sX + ((size_t)st * R + warp) * TW;
                    const float* cs_row = sC + ((size_t)st * R + warp) * TW;
                    float* dst_row = A.X + i * ld + col0;
                    float rs = 0.f;
#pragma unroll
                    for (int kk = 0; kk < K; ++kk) {
                        const int jl = kk * 128 + lane * 4;
                        const long long j = col0 + jl;
                        if (j < n) {
                            const float4 xv = *reinterpret_cast<const float4*>(xs_row + jl);
                            const float4 cv = *reinterpret_cast<const float4*>(cs_row + jl);
                            float xs[4] = {xv.x, xv.y, xv.z, xv.w};
                            const float cc[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                if (j + e < n) {
                                    const float d = fmaf(-rho, cc[e], phi + psi[kk][e]);
                                    const float xn = fmaxf(xs[e] + d, 0.f);
                                    scx = fmaf(cc[e], xn, scx);
                                    const float dp = fmaxf(d, 0.f);
                                    sd = fmaf(dp, dp, sd);
                                    xs[e] = xn;
                                    rs += xn;
                                    cacc[kk][e] += xn;
                                }
                            }
                            if (j + 3 < n) {
                                *reinterpret_cast<float4*>(dst_row + jl) = make_float4(xs[0], xs[1], xs[2], xs[3]);
                            } else {
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    if (j + e < n) dst_row[jl + e] = xs[e];
                            }
                        }
                    }
                    rs = warp_sum_f32(rs);
                    if (lane == 0) {
                        if (A.accumulate) atomicAdd(A.u + i, (double)rs);
                        else A.rowpart[t * m + i] = (double)rs;
                    }
                    if (++since_flush == kFlushRows) {
#pragma unroll
                        for (int kk = 0; kk < K; ++kk)
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                s_col[warp * TW + kk * 128 + lane * 4 + e] += (double)cacc[kk][e];
                                cacc[kk][e] = 0.f;
                            }
                        scx64 += (double)scx;
                        sd64 += (double)sd;
                        scx = 0.f;
                        sd = 0.f;
                        since_flush = 0;
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[st]);
            }
#pragma unroll
            for (int kk = 0; kk < K; ++kk)
#pragma unroll
                for (int e = 0; e < 4; ++e) s_col[warp * TW + kk * 128 + lane * 4 + e] += (double)cacc[kk][e];
            scx64 += (double)scx;
            sd64 += (double)sd;
            consumer_sync();
            double* out = A.colpart + (long long)slot * TW;
            for (int x = threadIdx.x; x < TW; x += kThreads) {
                double v = 0.0;
#pragma unroll
                for (int wv = 0; wv < kWarps; ++wv) v += s_col[wv * TW + x];
                if (!A.accumulate) out[x] = v;
                else if (col0 + x < n) atomicAdd(A.v + col0 + x, v);
            }
            consumer_sync();
            slot += walk.rev ? -1 : 1;
            w = walk.next(t, i0, i1);
        }
    }

    double v[2] = {scx64, sd64};
    block_sum_f64<2, kThreads + 32>(v, s_red);
    if (threadIdx.x == 0) {
        if (A.accumulate) {
            atomicAdd(acc_at(A.acc, 0), v[0]);
            atomicAdd(acc_at(A.acc, 1), v[1]);
        } else {
            A.ctapart[2 * blockIdx.x + 0] = v[0];
            A.ctapart[2 * blockIdx.x + 1] = v[1];
        }
        if (s_abort) {
            // after a give-up, let the copies already issued land before the
            // block's shared memory is released (each wait bounded as well)
            const uint32_t last = s_issued;
            for (uint32_t u = last > (uint32_t)S ? last - S : 0u; u < last; ++u)
                for (uint32_t it = 0; it < kWaitLimit; ++it)
                    if (mbar_try_wait(&full[u % S], (u / S) & 1u)) break;
        }
    }
}


// ------------------------------------------------------------ async-copy-fed variant
//
// Same arithmetic, partials and work split as drot_step_kernel<K, true>.  Each warp
// streams its own rows through a private S-stage ring in shared memory filled with
// 16-byte cp.async copies: while a warp computes row r, the copies of its next S-1
// rows are in flight, and they occupy shared memory, not registers.  Every lane
// reads back only the 16-byte chunks it copied itself, so a lane's own
// cp.async.wait_group is the only synchronisation the ring needs.  Column partials
// are promoted to FP64 in registers; the ring is reused as the cross-warp
// reduction buffer at the end of each column tile.

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int K, int S>
struct AsyncLayout {
    static constexpr int TW = 128 * K;
    static constexpr size_t ring_floats = (size_t)kWarps * S * 2 * TW;  // X and C per stage
    static constexpr size_t bytes = ring_floats * sizeof(float) > (size_t)kWarps * TW * sizeof(double)
                                        ? ring_floats * sizeof(float)
                                        : (size_t)kWarps * TW * sizeof(double);
};

// Copies row r of this warp's rows in the tile (row first + stride r, if r < nr; the
// stride is kWarps forwards, -kWarps backwards) of X and C into ring stage r mod S, and
// commits a group (empty past the last row, which keeps the group count in step).
template <int K, int S>
__device__ __forceinline__ void async_issue_row(const StepArgs& A, float* ring, long long first, long long stride,
                                                int nr, long long col0, int lane, int r) {
    constexpr int TW = 128 * K;
    if (r < nr) {
        const long long i = first + stride * r;
        float* xs = ring + (size_t)(r % S) * 2 * TW;
        float* cs_ = xs + TW;
        const long long rowoff = i * A.ld + col0 + lane * 4;
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            if (col0 + kk * 128 + lane * 4 < A.n) {
                cp_async16(xs + kk * 128 + lane * 4, A.X + rowoff + kk * 128);
                cp_async16(cs_ + kk * 128 + lane * 4, A.C + rowoff + kk * 128);
            }
        }
    }
    cp_async_commit();
}

template <int K, int S>
__global__ void __launch_bounds__(kThreads, 2) drot_step_async_kernel(StepArgs A) {
    constexpr int TW = 128 * K;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* ring = reinterpret_cast<float*>(smem_raw) + (size_t)(threadIdx.x >> 5) * S * 2 * TW;
    double* s_col = reinterpret_cast<double*>(smem_raw);  // reused at the end of each tile
    __shared__ double s_red[kWarps][2];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long m = A.m, n = A.n, ld = A.ld;
    const long long w0 = A.wbound[blockIdx.x];
    const long long w1 = A.wbound[blockIdx.x + 1];
    const SegWalk walk{w0, w1, m, A.serp != 0 && A.odd != 0};
    const long long stride = walk.rev ? -kWarps : kWarps;

    // The copies of the first S - 1 rows go out before the wait for the preceding
    // finish kernel: X and C are final once that kernel runs (it waited for the step
    // before it), and what it writes (g, h, the scalars, the zeroed totals) is read or
    // accumulated only after the wait.  A solve that has already stopped skips them.
    bool primed = false;
    if (w0 < w1 && __ldcg(&A.sc->done) == kRunning) {
        long long t, i0, i1;
        walk.seg(walk.start(), t, i0, i1);
        const long long first = walk.row(i0, i1, warp);
        const int nr = warp < i1 - i0 ? (int)((i1 - i0 - 1 - warp) / kWarps + 1) : 0;
#pragma unroll
        for (int r = 0; r < S - 1; ++r) async_issue_row<K, S>(A, ring, first, stride, nr, t * TW, lane, r);
        primed = true;
    }
    wait_for_predecessor();
    if (A.sc->done != kRunning) {
        cp_async_wait<0>();  // let the early copies land before the block's shared memory is released
        return;
    }

    const float rho = (float)A.sc->rho;
    const double cs = A.sc->c;
    int slot = walk.first_slot(A.slot_base[blockIdx.x]);
    double scx64 = 0.0, sd64 = 0.0;

    for (long long w = walk.start(); walk.more(w);) {
        long long t, i0, i1;
        walk.seg(w, t, i0, i1);
        const long long col0 = t * TW;

        float psi[K][4], cacc[K][4];
        double cacc64[K][4];
#pragma unroll
        for (int kk = 0; kk < K; ++kk)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const long long j = col0 + kk * 128 + lane * 4 + e;
                psi[kk][e] = j < n ? (float)((A.h[j] + cs) * A.inv_m) : 0.f;
                cacc[kk][e] = 0.f;
                cacc64[kk][e] = 0.0;
            }
        // rows of this warp in the tile: the segment's rows k = warp + kWarps r in walk
        // order, r = 0 .. nr-1
        const long long first = walk.row(i0, i1, warp);
        const int nr = warp < i1 - i0 ? (int)((i1 - i0 - 1 - warp) / kWarps + 1) : 0;
        auto issue = [&](int r) { async_issue_row<K, S>(A, ring, first, stride, nr, col0, lane, r); };
        if (!primed) {
#pragma unroll
            for (int r = 0; r < S - 1; ++r) issue(r);
        }
        primed = false;

        float scx = 0.f, sd = 0.f;
        int since_flush = 0;
        for (int r = 0; r < nr; ++r) {
            issue(r + S - 1);
            cp_async_wait<S - 1>();
            const long long i = first + stride * r;
            const float* xs = ring + (size_t)(r % S) * 2 * TW;
            const float* csr = xs + TW;
            const float phi = (float)((A.g[i] + cs) * A.inv_n);
            float* dst_row = A.X + i * ld + col0;
            float rs = 0.f;
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                const int jl = kk * 128 + lane * 4;
                const long long j = col0 + jl;
                if (j < n) {
                    const float4 xv = *reinterpret_cast<const float4*>(xs + jl);
                    const float4 cv = *reinterpret_cast<const float4*>(csr + jl);
                    float x4[4] = {xv.x, xv.y, xv.z, xv.w};
                    const float cc[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (j + e < n) {
                            const float d = fmaf(-rho, cc[e], phi + psi[kk][e]);
                            const float xn = fmaxf(x4[e] + d, 0.f);
                            scx = fmaf(cc[e], xn, scx);
                            const float dp = fmaxf(d, 0.f);
                            sd = fmaf(dp, dp, sd);
                            x4[e] = xn;
                            rs += xn;
                            cacc[kk][e] += xn;
                        }
                    }
                    if (j + 3 < n) {
                        *reinterpret_cast<float4*>(dst_row + jl) = make_float4(x4[0], x4[1], x4[2], x4[3]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (j + e < n) dst_row[jl + e] = x4[e];
                    }
                }
            }
            rs = warp_sum_f32(rs);
            if (lane == 0) {
                if (A.accumulate) atomicAdd(A.u + i, (double)rs);
                else A.rowpart[t * m + i] = (double)rs;
            }
            if (++since_flush == kFlushRows) {
#pragma unroll
                for (int kk = 0; kk < K; ++kk)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        cacc64[kk][e] += (double)cacc[kk][e];
                        cacc[kk][e] = 0.f;
                    }
                scx64 += (double)scx;
                sd64 += (double)sd;
                scx = 0.f;
                sd = 0.f;
                since_flush = 0;
            }
        }
        cp_async_wait<0>();
#pragma unroll
        for (int kk = 0; kk < K; ++kk)
#pragma unroll
            for (int e = 0; e < 4; ++e) cacc64[kk][e] += (double)cacc[kk][e];
        scx64 += (double)scx;
        sd64 += (double)sd;
        __syncthreads();  // every warp is done with its ring: reuse it for the column reduction
#pragma unroll
        for (int kk = 0; kk < K; ++kk)
#pragma unroll
            for (int e = 0; e < 4; ++e) s_col[(size_t)warp * TW + kk * 128 + lane * 4 + e] = cacc64[kk][e];
        __syncthreads();
        double* out = A.colpart + (long long)slot * TW;
        for (int x = threadIdx.x; x < TW; x += kThreads) {
            double v = 0.0;
#pragma unroll
            for (int wv = 0; wv < kWarps; ++wv) v += s_col[(size_t)wv * TW + x];
            if (!A.accumulate) out[x] = v;
            else if (col0 + x < n) atomicAdd(A.v + col0 + x, v);
        }
        __syncthreads();
        slot += walk.rev ? -1 : 1;
        w = walk.next(t, i0, i1);
    }

    double v[2] = {scx64, sd64};
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

struct FinishArgs {
    const double* rowpart;
    const double* colpart;
    const double* ctapart;
    double* u;              // accumulation mode: row totals, read and reset to 0
    double* v;              // accumulation mode: column totals, read and reset to 0
    double* acc;            // accumulation mode: kAccSlots totals (acc_at): <C,X>, sum [d]_+^2, the six finish totals,
                            // read and reset by the last block
    int accumulate;
    const int* tile_slot;   // [T+1] first slot of each column tile
    const double* p;
    const double* q;
    double* a;
    double* b;
    double* g;
    double* h;
    double* finpart;        // [gridDim.x][kFinishAcc]
    Scalars* sc;
    long long m, n;
    int T, TW, G;
    double inv_n, inv_m;
    double inv_mn;          // 1 / (m + n)
    int no_test;            // 1: the preceding pass had no C (C-skipping): <C,X> unknown, no stopping test
    double* trace;          // optional: [2 * trace_len] <C, X_k> and ||r||_1 + ||s||_1 of iterate k at 2(k-1)
    long long trace_len;
};

// Sum of `count` partials spaced `stride` apart, in a fixed order: four
// interleaved accumulators (so that up to eight loads are in flight), combined
// as (a0 + a1) + (a2 + a3).
__device__ __forceinline__ double strided_total(const double* base, long long stride, int count) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int t = 0;
    for (; t + 8 <= count; t += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(base + (long long)(t + u) * stride);
        a0 += v[0]; a1 += v[1]; a2 += v[2]; a3 += v[3];
        a0 += v[4]; a1 += v[5]; a2 += v[6]; a3 += v[7];
    }
    for (; t < count; ++t) {
        const double v = __ldcg(base + (long long)t * stride);
        switch (t & 3) {
            case 0: a0 += v; break;
            case 1: a1 += v; break;
            case 2: a2 += v; break;
            default: a3 += v; break;
        }
    }
    return (a0 + a1) + (a2 + a3);
}

__device__ __forceinline__ double row_total(const FinishArgs& A, long long i) {
    if (A.accumulate) {
        const double u = __ldcg(A.u + i);
        A.u[i] = 0.0;
        return u;
    }
    return strided_total(A.rowpart + i, A.m, A.T);
}

__device__ __forceinline__ double col_total(const FinishArgs& A, long long j) {
    if (A.accumulate) {
        const double v = __ldcg(A.v + j);
        A.v[j] = 0.0;
        return v;
    }
    const long long t = j / A.TW;
    const long long jj = j - t * A.TW;
    const int s0 = A.tile_slot[t];
    return strided_total(A.colpart + (long long)s0 * A.TW + jj, A.TW, A.tile_slot[t + 1] - s0);
}

// Returns true in every thread of the block that arrived last (all blocks'
// finpart rows are then visible).  No block waits for another.
__device__ __forceinline__ bool arrive_last(Scalars* sc, int nblk) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int ticket = atomicAdd(&sc->counter, 1u);
        s_last = (ticket == (unsigned int)nblk - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// Scalars the finish reads that the step before it does not write: the solve's
// constants, and alpha, k and the last primal value, which only the previous finish
// writes.  The single-problem finish kernel loads them before it waits for the step.
struct FinishConsts {
    double alpha, sum_p, sum_q, inv_rho, tol, primal;
    long long k, max_iter;
    int stop_rule;
};

__device__ __forceinline__ FinishConsts load_finish_consts(const Scalars* sc) {
    FinishConsts K;
    K.alpha = __ldcg(&sc->alpha);
    K.sum_p = __ldcg(&sc->sum_p);
    K.sum_q = __ldcg(&sc->sum_q);
    K.inv_rho = __ldcg(&sc->inv_rho);
    K.tol = __ldcg(&sc->tol);
    K.primal = __ldcg(&sc->primal);
    K.k = __ldcg(&sc->k);
    K.max_iter = __ldcg(&sc->max_iter);
    K.stop_rule = __ldcg(&sc->stop_rule);
    return K;
}

// Scalar part of the finish (one thread): steps 5-8's scalars and the stopping test
// (Sec. 3.1) from the totals tot[0..5] (sum r, ||r||_1 + ||s||_1, ||r||^2 + ||s||^2,
// p.g', q.h', sum s), <C,X> and sum [phi + psi - rho C]_+^2.  Norms are kept squared on
// the device (the host takes the square roots it reports), so the test needs no FP64
// sqrt.  No fence before `done`: it is read by later kernels (after their wait for
// this one or after a grid barrier, both of which order it) and by the host after the
// stream's work has completed.
__device__ __forceinline__ void finish_scalars(const FinishArgs& A, const double* tot, double scx, double sdx,
                                               const FinishConsts& K) {
    Scalars* sc = A.sc;
    const double beta = tot[0] * A.inv_mn;             // step 5
    const double c_new = 2.0 * beta - K.alpha;         // steps 6-7 scalar term
    const double pphi = (tot[3] + c_new * K.sum_p) * A.inv_n;
    const double qpsi = (tot[4] + c_new * K.sum_q) * A.inv_m;
    const double primal = A.no_test ? K.primal : scx;
    const double dual = (pphi + qpsi) * K.inv_rho;
    const double gap = fabs(primal - dual);
    const double res_l1 = tot[1];
    const double res_l2_sq = tot[2];
    const double dres_sq = sdx * K.inv_rho * K.inv_rho;
    sc->alpha = K.alpha - beta;                        // step 8
    sc->c = c_new;
    sc->beta = beta;
    if (!A.no_test) {
        sc->primal = primal;
        sc->dual = dual;
        sc->gap = gap;
        sc->res_l1 = res_l1;
        sc->res_l2 = res_l2_sq;          // squared (see above)
        sc->dual_res_prev = dres_sq;     // squared
    }
    const long long k = K.k + 1;
    sc->k = k;
    if (A.trace && !A.no_test && k <= A.trace_len) {
        A.trace[2 * (k - 1)] = primal;
        A.trace[2 * (k - 1) + 1] = res_l1;
    }
    const bool finite = isfinite(primal) && isfinite(dual) && isfinite(res_l1) && isfinite(res_l2_sq) &&
                        isfinite(dres_sq) && isfinite(c_new) && isfinite(tot[5]);
    const int rule = K.stop_rule;
    const double tol = K.tol;
    const bool conv = !A.no_test && tol >= 0.0 && (!(rule & 1) || gap <= tol) && (!(rule & 2) || res_l1 <= tol) &&
                      (!(rule & 4) || dres_sq <= tol * tol);
    int done = kRunning;
    if (__ldcg(&sc->fault)) done = kFault;
    else if (!finite) done = kNonFinite;
    else if (conv) done = kConverged;
    else if (k >= K.max_iter) done = kIterCap;
    sc->counter = 0u;
    sc->done = done;
}

// The first element of a finish thread, loaded before the wait for the step: p_i and
// a_i (row) or q_j and b_j (column); the previous finish wrote a and b.
struct FinishPre {
    bool valid;
    double pq, ab;
};

__device__ __forceinline__ FinishPre load_finish_pre(const FinishArgs& A, long long idx) {
    FinishPre F{false, 0.0, 0.0};
    if (idx < A.m) {
        F = FinishPre{true, __ldcg(A.p + idx), __ldcg(A.a + idx)};
    } else if (idx < A.m + A.n) {
        F = FinishPre{true, __ldcg(A.q + idx - A.m), __ldcg(A.b + idx - A.m)};
    }
    return F;
}

// Steps 5-8 of Algorithm 1 and the stopping test (Sec. 3.1), executed by block
// `blk` of the `nblk` blocks (of NT threads) that serve this problem.
//
// Accumulation mode: the block reduces its six partial sums (warp shuffles, then
// shared memory) and thread 0 adds them into the FP64 totals with atomics and takes
// a ticket; in the block that arrived last, thread 0 reads the totals once and
// forms the scalars.  Fixed-order mode: per-block partials (finpart) summed by the
// last block in block order.  FP64 has a long dependent latency on this GPU, so the
// accumulation path keeps the chain after the element work to one block reduction,
// one fence, one ticket and one read of the totals.  `pre` (optional) holds this
// thread's first element and `kc` (optional) the scalars, both loaded earlier.
template <int NT = kFinishThreads>
__device__ __forceinline__ void finish_body(const FinishArgs& A, int blk, int nblk, FinishPre pre = FinishPre{},
                                            const FinishConsts* kc = nullptr) {
    __shared__ double s_red[NT / 32][kFinishAcc];
    Scalars* sc = A.sc;

    // acc: 0 sum r, 1 ||r||_1 + ||s||_1, 2 ||r||^2 + ||s||^2, 3 p.g', 4 q.h', 5 sum s
    double acc[kFinishAcc] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const long long mn = A.m + A.n;
    // E elements per thread per pass, all their loads issued before any store (a store
    // to a, g, u could alias a later load as far as the compiler knows, which would
    // otherwise serialise one memory round trip per element)
    constexpr int E = 4;
    const long long stride = (long long)nblk * NT;
    for (long long base = (long long)blk * NT + threadIdx.x; base < mn; base += E * stride) {
        double tot[E], pq[E], ab[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const long long idx = base + e * stride;
            tot[e] = pq[e] = ab[e] = 0.0;
            if (idx < A.m) {
                tot[e] = A.accumulate ? __ldcg(A.u + idx) : row_total(A, idx);
                pq[e] = (e == 0 && pre.valid) ? pre.pq : A.p[idx];
                ab[e] = (e == 0 && pre.valid) ? pre.ab : __ldcg(A.a + idx);
            } else if (idx < mn) {
                const long long j = idx - A.m;
                tot[e] = A.accumulate ? __ldcg(A.v + j) : col_total(A, j);
                pq[e] = (e == 0 && pre.valid) ? pre.pq : A.q[j];
                ab[e] = (e == 0 && pre.valid) ? pre.ab : __ldcg(A.b + j);
            }
        }
        pre.valid = false;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const long long idx = base + e * stride;
            if (idx < A.m) {
                const long long i = idx;
                if (A.accumulate) A.u[i] = 0.0;  // the totals start from zero in the next step
                const double r = tot[e] - pq[e];
                const double gn = ab[e] - 2.0 * r;
                A.a[i] = ab[e] - r;
                A.g[i] = gn;
                acc[0] += r;
                acc[1] += fabs(r);
                acc[2] += r * r;
                acc[3] += pq[e] * gn;
            } else if (idx < mn) {
                const long long j = idx - A.m;
                if (A.accumulate) A.v[j] = 0.0;
                const double sj = tot[e] - pq[e];
                const double hn = ab[e] - 2.0 * sj;
                A.b[j] = ab[e] - sj;
                A.h[j] = hn;
                acc[5] += sj;
                acc[1] += fabs(sj);
                acc[2] += sj * sj;
                acc[4] += pq[e] * hn;
            }
        }
    }
    if (A.accumulate) {
        const double v8[8] = {acc[0], acc[1], acc[2], acc[3], acc[4], acc[5], 0.0, 0.0};
        const double tot_l = warp_sum8_scatter(v8);  // lane 4q holds the warp total of value q
        const int q = (threadIdx.x >> 2) & 7;
        if ((threadIdx.x & 3) == 0 && q < kFinishAcc) s_red[threadIdx.x >> 5][q] = tot_l;
        __syncthreads();
        if (threadIdx.x != 0) return;
#pragma unroll
        for (int c = 0; c < kFinishAcc; ++c) acc[c] = s_red[0][c];
#pragma unroll
        for (int w = 1; w < NT / 32; ++w)
#pragma unroll
            for (int c = 0; c < kFinishAcc; ++c) acc[c] += s_red[w][c];
#pragma unroll
        for (int c = 0; c < kFinishAcc; ++c) atomicAdd(acc_at(A.acc, 2 + c), acc[c]);
        __threadfence();
        if (atomicAdd(&sc->counter, 1u) != (unsigned int)nblk - 1u) return;
        __threadfence();
        double tot[kFinishAcc];
#pragma unroll
        for (int c = 0; c < kFinishAcc; ++c) tot[c] = __ldcg(acc_at(A.acc, 2 + c));
        const double scx = __ldcg(acc_at(A.acc, 0)), sdx = __ldcg(acc_at(A.acc, 1));
#pragma unroll
        for (int c = 0; c < kAccSlots; ++c) *acc_at(A.acc, c) = 0.0;
        finish_scalars(A, tot, scx, sdx, kc ? *kc : load_finish_consts(sc));
        return;
    }

    block_sum_f64<kFinishAcc, NT>(acc, s_red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < kFinishAcc; ++c) A.finpart[blk * kFinishAcc + c] = acc[c];
    }
    if (!arrive_last(sc, nblk)) return;

    // Last block: fixed-order totals over the blocks of this launch and the
    // CTAs of the step launch.
    double tot[kFinishAcc + 2];
    for (int c = 0; c < kFinishAcc + 2; ++c) tot[c] = 0.0;
    for (int bidx = threadIdx.x; bidx < nblk; bidx += NT)
        for (int c = 0; c < kFinishAcc; ++c) tot[c] += __ldcg(A.finpart + bidx * kFinishAcc + c);
    for (int bidx = threadIdx.x; bidx < A.G; bidx += NT) {
        tot[kFinishAcc + 0] += __ldcg(A.ctapart + 2 * bidx + 0);
        tot[kFinishAcc + 1] += __ldcg(A.ctapart + 2 * bidx + 1);
    }
    __shared__ double s_red2[NT / 32][kFinishAcc + 2];
    block_sum_f64<kFinishAcc + 2, NT>(tot, s_red2);
    if (threadIdx.x == 0)
        finish_scalars(A, tot, tot[kFinishAcc + 0], tot[kFinishAcc + 1], kc ? *kc : load_finish_consts(sc));
}

// The finish of the single-problem graph.  It is launched as a programmatic dependent
// of the step, so the loads that do not depend on the step (this thread's first
// element of p, a / q, b and the scalars of FinishConsts) are issued before the wait.
__global__ void __launch_bounds__(kFinishThreads) drot_finish_kernel(FinishArgs A) {
    const FinishPre pre = load_finish_pre(A, (long long)blockIdx.x * kFinishThreads + threadIdx.x);
    const FinishConsts kc = load_finish_consts(A.sc);
    wait_for_predecessor();
    release_dependents();  // the next step may start its blocks and its first copies of X and C
    if (A.sc->done != kRunning) return;
    finish_body<kFinishThreads>(A, blockIdx.x, gridDim.x, pre, &kc);
}

// ------------------------------------------------------------------ persistent solve
//
// One cooperative launch (every CTA resident) runs up to `budget` iterations:
// fused step -> grid barrier -> finish (elements spread over all CTAs, scalar part
// in the last CTA to arrive) -> grid barrier.  The grid barrier is a counter and a
// generation word; a CTA that waits longer than kBarrierSpins polls (or the solve's
// configured limit, GridSync::spin_limit) records a
// fault in Scalars and leaves, and every other CTA then leaves at its next wait,
// so a broken launch ends instead of hanging.

constexpr unsigned long long kBarrierSpins = 1ull << 24;

struct GridSync {
    unsigned int count;             // barrier arrivals of the current launch (cleared before each launch)
    unsigned int pad;
    unsigned long long step_ns;     // time from each step's start to the end of its barrier (CTA 0)
    unsigned long long iters;       // iterations timed
    unsigned long long spin_limit;  // polls before a barrier wait gives up (0: kBarrierSpins)
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier on a monotonic arrival counter (cleared by the host before each launch):
// barrier t of a launch waits until (t + 1) G CTAs have arrived, `target` holding (t + 1) G.
// One atomic per CTA and a spin on one word (1.27 us per barrier on B300 with 148 CTAs, against
// 2.39 us for a generation flip with back-off).  Returns false in every thread of the CTA if the
// wait gave up: after `limit` polls, or on seeing another CTA's fault, it sets the fault flag.
__device__ __forceinline__ bool grid_barrier_counter(unsigned int* count, unsigned int target,
                                                     unsigned long long limit, Scalars* sc) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        int ok = 1;
        unsigned long long spins = 0;
        while (ld_acquire_u32(count) < target) {
            if (++spins > limit || ((spins & 255ull) == 0 && *(volatile int*)&sc->fault)) {
                atomicExch(&sc->fault, 1);
                ok = 0;
                break;
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The persistent solve's barrier (GridSync::spin_limit polls, or kBarrierSpins).
__device__ __forceinline__ bool grid_barrier(GridSync* gs, Scalars* sc, unsigned int& target) {
    target += gridDim.x;
    return grid_barrier_counter(&gs->count, target, gs->spin_limit ? gs->spin_limit : kBarrierSpins, sc);
}

template <int K>
__global__ void __launch_bounds__(kThreads, 2) drot_persistent_kernel(StepArgs A, FinishArgs F, GridSync* gs,
                                                                      long long budget) {
    __shared__ StepSmem<K> sm;
    Scalars* sc = F.sc;
    unsigned int target = 0;  // arrivals the next barrier waits for (the counter is 0 at launch)
    for (long long it = 0; it < budget; ++it) {
        if (*(volatile int*)&sc->done != kRunning) break;  // uniform: read after a barrier
        const unsigned long long t0 = (blockIdx.x == 0 && threadIdx.x == 0) ? global_ns() : 0ull;
        step_pass<K, true, 0>(A, blockIdx.x, sm, A.serp != 0 && (it & 1) != 0);
        if (!grid_barrier(gs, sc, target)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            gs->step_ns += global_ns() - t0;
            gs->iters += 1;
        }
        finish_body<kThreads>(F, blockIdx.x, gridDim.x);
        if (!grid_barrier(gs, sc, target)) return;
    }
}

// ---------------------------------------------------------------- set-up / tear-down

// X_0 = p q^T (the paper's cold start, Sec. 4), rounded to FP32.
__global__ void drot_init_plan_kernel(float* X, const double* p, const double* q, long long m, long long n,
                                      long long ld) {
    const long long nv = (n + 3) / 4;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < m * nv;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx / nv;
        const long long j = (idx - i * nv) * 4;
        const double pi = p[i];
        float* dst = X + i * ld + j;
        if (j + 3 < n) {
            *reinterpret_cast<float4*>(dst) = make_float4((float)(pi * q[j]), (float)(pi * q[j + 1]),
                                                          (float)(pi * q[j + 2]), (float)(pi * q[j + 3]));
        } else {
            for (int e = 0; e < 4; ++e)
                if (j + e < n) dst[e] = (float)(pi * q[j + e]);
        }
    }
}

// Sums and minima of the marginals and of the warm-start duals (one block).
__global__ void __launch_bounds__(1024) drot_vector_sums_kernel(const double* p, const double* q, const double* mu0,
                                                                const double* nu0, long long m, long long n,
                                                                Scalars* sc) {
    __shared__ double s_red[32][6];
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // sum p, sum q, sum mu0, sum nu0, bad p, bad q
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        v[0] += p[i];
        if (!(p[i] >= 0.0) || !isfinite(p[i])) v[4] += 1.0;
        if (mu0) v[2] += mu0[i];
    }
    for (long long j = threadIdx.x; j < n; j += blockDim.x) {
        v[1] += q[j];
        if (!(q[j] >= 0.0) || !isfinite(q[j])) v[5] += 1.0;
        if (nu0) v[3] += nu0[j];
    }
    block_sum_f64<6, 1024>(v, s_red);
    if (threadIdx.x == 0) {
        sc->sum_p = v[0];
        sc->sum_q = v[1];
        sc->sum_phi0 = sc->rho * v[2];
        sc->sum_psi0 = sc->rho * v[3];
        sc->nonfinite_input = (v[4] > 0.0 ? 1 : 0) | (v[5] > 0.0 ? 2 : 0) |
                              ((isfinite(v[2]) && isfinite(v[3])) ? 0 : 4);
    }
}

// a_0 = Y_0 e - p, b_0 = Y_0^T f - q with Y_0 = X_0 + phi_0 e^T + f psi_0^T
// (Algorithm 1's initialisation, with a warm start phi_0 = rho mu_0,
// psi_0 = rho nu_0), the numerators g = n phi_0, h = m psi_0, c_0 = 0 and
// alpha_0 = f^T a_0 / (m + n).  Row and column sums of X_0 come from a
// preceding UPDATE = false pass of the step kernel.
__device__ __forceinline__ void init_state_body(const FinishArgs& A, const double* mu0, const double* nu0, int blk,
                                                int nblk) {
    __shared__ double s_red[kFinishThreads / 32][1];
    Scalars* sc = A.sc;
    const double rho = sc->rho;
    const double nd = (double)A.n, md = (double)A.m;
    double acc[1] = {0.0};
    const long long mn = A.m + A.n;
    for (long long idx = (long long)blk * kFinishThreads + threadIdx.x; idx < mn;
         idx += (long long)nblk * kFinishThreads) {
        if (idx < A.m) {
            const long long i = idx;
            const double phi0 = mu0 ? rho * mu0[i] : 0.0;
            const double ai = row_total(A, i) - A.p[i] + nd * phi0 + sc->sum_psi0;
            A.a[i] = ai;
            A.g[i] = nd * phi0;
            acc[0] += ai;
        } else {
            const long long j = idx - A.m;
            const double psi0 = nu0 ? rho * nu0[j] : 0.0;
            A.b[j] = col_total(A, j) - A.q[j] + md * psi0 + sc->sum_phi0;
            A.h[j] = md * psi0;
        }
    }
    block_sum_f64<1, kFinishThreads>(acc, s_red);
    if (threadIdx.x == 0) A.finpart[blk * kFinishAcc] = acc[0];
    if (!arrive_last(sc, nblk)) return;
    double tot[1] = {0.0};
    for (int bidx = threadIdx.x; bidx < nblk; bidx += kFinishThreads)
        tot[0] += __ldcg(A.finpart + bidx * kFinishAcc);
    __shared__ double s_red2[kFinishThreads / 32][1];
    block_sum_f64<1, kFinishThreads>(tot, s_red2);
    if (threadIdx.x == 0) {
        sc->alpha = tot[0] * A.inv_mn;
        sc->c = 0.0;
        sc->k = 0;
        sc->counter = 0u;
        sc->done = kRunning;
    }
}

__global__ void __launch_bounds__(kFinishThreads) drot_init_state_kernel(FinishArgs A, const double* mu0,
                                                                         const double* nu0) {
    init_state_body(A, mu0, nu0, blockIdx.x, gridDim.x);
}

// mu = phi / rho, nu = psi / rho (Appendix A.2, eq. dual:var).
__global__ void drot_export_duals_kernel(const double* g, const double* h, const Scalars* sc, double* mu, double* nu,
                                         long long m, long long n, double inv_n, double inv_m) {
    const double c = sc->c, rho = sc->rho;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < m + n;
         idx += (long long)gridDim.x * blockDim.x) {
        if (idx < m) mu[idx] = (g[idx] + c) * inv_n / rho;
        else nu[idx - m] = (h[idx - m] + c) * inv_m / rho;
    }
}

// Number of strictly positive entries of the plan.
__global__ void drot_count_nnz_kernel(const float* X, long long m, long long n, long long ld, Scalars* sc) {
    unsigned long long cnt = 0;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx / n, j = idx - i * n;
        cnt += X[i * ld + j] > 0.f ? 1ull : 0ull;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&sc->nnz, cnt);
}

}  // namespace drot
