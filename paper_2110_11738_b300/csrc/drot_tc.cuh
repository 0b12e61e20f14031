// Tensor-core matrix products of the warm-start network on the fifth-generation tensor
// cores (tcgen05): C = A B^T with BF16 operands and an FP32 accumulator.
//
// Both operands are K-major (row-major with the reduced index contiguous): A is M x K,
// B is N x K.  One CTA computes a 128-row block of C over a K range of at most 256:
//   * one thread issues TMA tensor copies (cp.async.bulk.tensor, 128-byte swizzle) of the
//     K range of its A rows and of all N rows of B into shared memory, in chunks of 64
//     K elements (one 128-byte swizzle row), and arrives on an mbarrier with their byte
//     count;
//   * once they have landed, the same thread issues tcgen05.mma (kind::f16, M = 128,
//     N = the product's width, K = 16 per instruction) into an FP32 accumulator in tensor
//     memory (TMEM, allocated by warp 0) and commits them to a second mbarrier;
//   * the four warps then read the accumulator back with tcgen05.ld (warp w owns TMEM
//     lanes 32w .. 32w + 31, i.e. rows 32w .. 32w + 31 of the block) and apply the
//     layer's epilogue (bias and ReLU, ReLU-derivative mask, or an atomic add for split-K
//     weight gradients), optionally also writing the transpose of a BF16 result for the
//     weight-gradient products of the backward pass.
// A K range longer than 256 is split over gridDim.y, the partial products added with
// atomics.  Rows of A beyond M and K beyond the operands' extent are read as zeros (TMA
// out-of-bounds fill), so M and K need no padding to the block sizes.  Products of one
// K range with N = 256 (every layer of the network against its weight matrix) use the
// persistent variant below instead: B stays resident, A streams through a ring, and two
// tensor-memory accumulators let one block's epilogue overlap the next block's products.
//
// Every wait is bounded: a CTA whose copies or products do not complete within the limit
// records a fault in *err, waits (bounded again) for what it has issued, frees its tensor
// memory and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "drot_kernels.cuh"

namespace drot {
namespace tc {

using bf16 = __nv_bfloat16;

constexpr int kBM = 128;          // rows of C per CTA (the MMA's M)
constexpr int kBK = 64;           // K elements per chunk: one 128-byte swizzle row of BF16
constexpr int kMaxChunks = 4;     // K chunks per CTA: a K range of at most 256
constexpr int kThreads = 128;     // four warps, one per 32 TMEM lanes in the epilogue
constexpr uint32_t kPollLimit = 1u << 24;  // polls (with back-off) before a wait gives up

// Epilogues (same numbering as the warp-level product they replace).
enum Epilogue : int {
    kStoreF32 = 0,      // C = acc (FP32)
    kReluBiasBf16 = 1,  // H = bf16(max(acc + bias[n], 0))
    kMaskBf16 = 2,      // D = bf16(acc * (mask[m, n] > 0))
    kAtomicF32 = 3      // C += acc (FP32 atomics; split-K)
};

struct EpiArgs {
    int kind;
    float* Cf;              // FP32 result (kStoreF32, kAtomicF32)
    bf16* Cb;               // BF16 result (kReluBiasBf16, kMaskBf16)
    bf16* CbT;              // optional: its transpose, N x M with pitch ldt
    int ldc, ldt;
    const float* bias;      // kReluBiasBf16: N
    const bf16* mask;       // kMaskBf16: M x N with pitch ldc
    int* err;               // set to 1 when a wait gives up
};

// Shared-memory bytes of a CTA computing an N-wide block (1024 bytes of slack to align
// the swizzled tiles, plus the two mbarriers).
__host__ __device__ constexpr int smem_bytes(int N) { return kMaxChunks * (kBM + N) * 128 + 1024 + 64; }

// Shared-memory matrix descriptor of a K-major operand tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, groups of 8 rows 1024 bytes apart (stride byte
// offset), leading byte offset unused for this layout (1), descriptor version 1 (bit 46),
// layout type 2 = 128-byte swizzle (bits 61-63).  The tile must start 1024-byte aligned;
// the K-th group of 16 elements inside a 64-element chunk starts 32 K bytes further.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t smem_addr) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < kPollLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it >= 64) __nanosleep(128);
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once every tcgen05.mma this thread issued before has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// C[m0 .. m0+127, 0 .. N-1] (+)= A[m0.., k0 .. k0+kchunks*64) B[.., same]^T, k0 = blockIdx.y * kchunks * 64.
template <int N>
__global__ void __launch_bounds__(kThreads, 1) gemm_tn_kernel(const __grid_constant__ CUtensorMap mapA,
                                                              const __grid_constant__ CUtensorMap mapB, int M,
                                                              int kchunks, EpiArgs E) {
    static_assert(N == 64 || N == 128 || N == 256, "N: a TMEM column count and a valid MMA width");
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    // 1024-byte aligned tiles: A chunks (128 rows x 128 B each), then B chunks (N rows x 128 B)
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint8_t* sA = base;
    uint8_t* sB = base + kMaxChunks * kBM * 128;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kMaxChunks * N * 128);  // [0] loads, [1] products
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM;
    const int k0 = blockIdx.y * kchunks * kBK;

    if (threadIdx.x == 0) {
        s_fail = 0;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&s_tmem, (uint32_t)N);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = s_tmem;

    bool issued = false;
    if (threadIdx.x == 0) {
        const uint32_t bytes = (uint32_t)kchunks * (kBM + N) * 128u;
        mbar_arrive_expect_tx(&bars[0], bytes);
        for (int c = 0; c < kchunks; ++c) {
            tma_load_2d(sA + c * kBM * 128, &mapA, k0 + c * kBK, m0, &bars[0]);
            tma_load_2d(sB + c * N * 128, &mapB, k0 + c * kBK, 0, &bars[0]);
        }
        if (wait_bounded(&bars[0], 0)) {
            fence_after_sync();
            constexpr uint32_t idesc = mma_idesc(kBM, N);
            for (int c = 0; c < kchunks; ++c) {
                const uint32_t a0 = smem_u32(sA + c * kBM * 128), b0 = smem_u32(sB + c * N * 128);
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk)
                    mma_bf16(tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                             (c > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(&bars[1]);
            issued = true;
        } else {
            s_fail = 1;
            wait_bounded(&bars[0], 0);  // the copies already issued, before the block leaves
        }
    }
    __syncthreads();
    bool ok = s_fail == 0;
    if (ok) {
        // every thread waits for the products (the commit arrives once they have completed)
        ok = wait_bounded(&bars[1], 0);
        if (!ok) s_fail = 1;
    }
    fence_after_sync();
    __syncthreads();
    ok = s_fail == 0;
    if (ok) {
        const int r = m0 + warp * 32 + lane;  // this thread's row of C (TMEM lane 32w + l)
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (r >= M) continue;
            if (E.kind == kAtomicF32 || E.kind == kStoreF32) {
                float* dst = E.Cf + (size_t)r * E.ldc + c0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    if (E.kind == kAtomicF32) atomicAdd(dst + j, v[j]);
                    else dst[j] = v[j];
                }
            } else {
                __align__(16) bf16 o[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float x;
                    if (E.kind == kReluBiasBf16) x = fmaxf(v[j] + E.bias[c0 + j], 0.f);
                    else x = __bfloat162float(E.mask[(size_t)r * E.ldc + c0 + j]) > 0.f ? v[j] : 0.f;
                    o[j] = __float2bfloat16(x);
                }
                uint4* dst = reinterpret_cast<uint4*>(E.Cb + (size_t)r * E.ldc + c0);
                const uint4* src = reinterpret_cast<const uint4*>(o);
#pragma unroll
                for (int j = 0; j < 4; ++j) dst[j] = src[j];
                if (E.CbT) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) E.CbT[(size_t)(c0 + j) * E.ldt + r] = o[j];
                }
            }
        }
    } else if (threadIdx.x == 0 && E.err) {
        atomicExch(E.err, 1);
        if (issued) wait_bounded(&bars[1], 0);  // products in flight still write tensor memory
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, (uint32_t)N);
}

// ------------------------------------------------------------------ persistent variant
//
// For products whose B is one weight matrix (K <= 256) shared by every row block: each CTA
// loads B once and keeps it in shared memory, then walks row blocks blockIdx.x,
// blockIdx.x + gridDim.x, ...  Warp 0 (one lane) streams the blocks' A chunks through a ring
// of kRing slots; warp 1 (one lane) issues the products into one of two TMEM accumulators and
// commits each slot back to the producer once its products are done; warps 2-9 drain the
// other accumulator (warp w reads TMEM lanes 32 (w mod 4) .. and one half of the columns)
// while the next block's products run, and hand it back.  Copies, products and epilogues of
// consecutive blocks overlap.  BF16 results leave through shared memory: each epilogue warp
// stages a 32 x 32 tile (and, when asked, its transpose) and one lane writes it with a TMA
// tensor store, so the stores are whole 64-byte rows instead of one thread's 16-byte pieces.
constexpr int kRing = 4;               // A chunk slots of 16 KB
constexpr int kEpiWarps = 8;           // two per group of 32 TMEM lanes, one per column half
constexpr int kResThreads = 64 + 32 * kEpiWarps;  // producer warp, MMA warp, epilogue warps
constexpr int kStageBytes = 2 * 32 * 32 * 2;       // per epilogue warp: a 32 x 32 BF16 tile and its transpose

__host__ __device__ constexpr int resident_smem_bytes(int N) {
    return kMaxChunks * N * 128 + kRing * kBM * 128 + kEpiWarps * kStageBytes + 1024 + 256;
}

// TMA tensor store of a 32 x 32 BF16 box from shared memory (bulk async-group of this thread).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of this thread's stores have been read
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// this thread's stores have completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy writes to shared memory visible to the TMA (async proxy)
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait that also gives up as soon as another role of the block has (*abort).
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort) {
    for (uint32_t it = 0; it < kPollLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (it >= 64) __nanosleep(64);
    }
    *abort = 1;
    return false;
}

template <int N>
__device__ __forceinline__ void epilogue_row(const EpiArgs& E, const float (&v)[32], int r, int c0) {
    if (E.kind == kAtomicF32 || E.kind == kStoreF32) {
        float* dst = E.Cf + (size_t)r * E.ldc + c0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (E.kind == kAtomicF32) atomicAdd(dst + j, v[j]);
            else dst[j] = v[j];
        }
        return;
    }
    __align__(16) bf16 o[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        float x;
        if (E.kind == kReluBiasBf16) x = fmaxf(v[j] + E.bias[c0 + j], 0.f);
        else x = __bfloat162float(E.mask[(size_t)r * E.ldc + c0 + j]) > 0.f ? v[j] : 0.f;
        o[j] = __float2bfloat16(x);
    }
    uint4* dst = reinterpret_cast<uint4*>(E.Cb + (size_t)r * E.ldc + c0);
    const uint4* src = reinterpret_cast<const uint4*>(o);
#pragma unroll
    for (int j = 0; j < 4; ++j) dst[j] = src[j];
    if (E.CbT) {
#pragma unroll
        for (int j = 0; j < 32; ++j) E.CbT[(size_t)(c0 + j) * E.ldt + r] = o[j];
    }
}

template <int N>
__global__ void __launch_bounds__(kResThreads, 1) gemm_tn_resident_kernel(const __grid_constant__ CUtensorMap mapA,
                                                                          const __grid_constant__ CUtensorMap mapB,
                                                                          const __grid_constant__ CUtensorMap mapC,
                                                                          const __grid_constant__ CUtensorMap mapCT,
                                                                          int M, int kchunks, int tma_out, EpiArgs E) {
    // tma_out: bit 0 = the BF16 result Cb is stored by TMA through mapC (32 x 32 boxes), bit 1 = its
    // transpose CbT through mapCT; otherwise each thread stores its row directly
    static_assert(N == 128 || N == 256, "two accumulators of N columns fit the 512 TMEM columns");
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ volatile int s_consumed;  // A slots the MMA warp has taken (for the drain after an abort)
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint8_t* sB = base;                               // kchunks x N rows x 128 B, resident
    uint8_t* sA = base + kMaxChunks * N * 128;        // kRing x 128 rows x 128 B
    uint8_t* sStage = sA + kRing * kBM * 128;      // kEpiWarps x (32 x 32 tile, its transpose), BF16
    uint64_t* b_full = reinterpret_cast<uint64_t*>(sStage + kEpiWarps * kStageBytes);
    uint64_t* a_full = b_full + 1;
    uint64_t* a_empty = a_full + kRing;
    uint64_t* acc_full = a_empty + kRing;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* drain = acc_empty + 2;     // after an abort: every product issued has completed
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = (M + kBM - 1) / kBM;
    const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (threadIdx.x == 0) {
        s_abort = 0;
        s_consumed = 0;
        mbar_init(b_full, 1);
        for (int s = 0; s < kRing; ++s) {
            mbar_init(&a_full[s], 1);
            mbar_init(&a_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kEpiWarps);  // one arrival per epilogue warp
        }
        mbar_init(drain, 1);
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(&s_tmem, 2u * N);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = s_tmem;

    if (warp == 0 && lane == 0) {
        // ---- producer: B once, then the A chunks of every block through the ring
        mbar_arrive_expect_tx(b_full, (uint32_t)kchunks * N * 128u);
        for (int c = 0; c < kchunks; ++c) tma_load_2d(sB + c * N * 128, &mapB, c * kBK, 0, b_full);
        int issued = 0;
        for (int i = 0; i < my_tiles && !s_abort; ++i) {
            const int m0 = ((int)blockIdx.x + i * (int)gridDim.x) * kBM;
            for (int c = 0; c < kchunks; ++c, ++issued) {
                const int slot = issued % kRing;
                const uint32_t ph = (uint32_t)(issued / kRing) & 1u;
                if (!wait_or_abort(&a_empty[slot], ph ^ 1u, &s_abort)) break;
                mbar_arrive_expect_tx(&a_full[slot], kBM * 128u);
                tma_load_2d(sA + slot * kBM * 128, &mapA, c * kBK, m0, &a_full[slot]);
            }
        }
        if (s_abort) {
            // copies still in flight land before the block leaves
            wait_bounded(b_full, 0);
            for (int j = s_consumed; j < issued; ++j) wait_bounded(&a_full[j % kRing], (uint32_t)(j / kRing) & 1u);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        constexpr uint32_t idesc = mma_idesc(kBM, N);
        bool ok = wait_or_abort(b_full, 0, &s_abort);
        fence_after_sync();
        int taken = 0;
        for (int i = 0; ok && i < my_tiles; ++i) {
            const int b = i & 1;
            ok = wait_or_abort(&acc_empty[b], ((uint32_t)(i >> 1) & 1u) ^ 1u, &s_abort);
            if (!ok) break;
            fence_after_sync();
            const uint32_t d = tmem + (uint32_t)(b * N);
            for (int c = 0; c < kchunks; ++c, ++taken) {
                const int slot = taken % kRing;
                ok = wait_or_abort(&a_full[slot], (uint32_t)(taken / kRing) & 1u, &s_abort);
                if (!ok) break;
                s_consumed = taken + 1;
                fence_after_sync();
                const uint32_t a0 = smem_u32(sA + slot * kBM * 128), b0 = smem_u32(sB + c * N * 128);
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk)
                    mma_bf16(d, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                             (c > 0 || kk > 0) ? 1u : 0u);
                mma_commit(&a_empty[slot]);  // the slot is free once these products are done
            }
            if (!ok) break;
            mma_commit(&acc_full[b]);
        }
        if (!ok) {
            // products already issued still write tensor memory: wait for all of them
            mma_commit(drain);
            wait_bounded(drain, 0);
        }
    } else if (warp >= 2) {
        // ---- epilogue warps: TMEM lanes 32 g .. 32 g + 31 are rows 32 g .. of the block;
        // columns [h N / 2, (h + 1) N / 2)
        const int g = warp & 3;
        const int h = (warp - 2) >> 2;
        bf16* stC = reinterpret_cast<bf16*>(sStage + (warp - 2) * kStageBytes);  // [32 rows][32 cols]
        bf16* stT = stC + 32 * 32;                                                // [32 cols][32 rows]
        for (int i = 0; i < my_tiles; ++i) {
            const int b = i & 1;
            if (!wait_or_abort(&acc_full[b], (uint32_t)(i >> 1) & 1u, &s_abort)) break;
            fence_after_sync();
            const int rg = ((int)blockIdx.x + i * (int)gridDim.x) * kBM + g * 32;  // first row of the group
            const int r = rg + lane;
#pragma unroll 1
            for (int c0 = h * (N / 2); c0 < (h + 1) * (N / 2); c0 += 32) {
                float v[32];
                tmem_ld32(tmem + (uint32_t)(b * N) + ((uint32_t)(g * 32) << 16) + (uint32_t)c0, v);
                if (!tma_out) {
                    if (r < M) epilogue_row<N>(E, v, r, c0);
                    continue;
                }
                // BF16 epilogue staged in shared memory and written by TMA stores (rows >= M are
                // computed but clipped by the store)
                __align__(16) bf16 o[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float x;
                    if (E.kind == kReluBiasBf16) x = fmaxf(v[j] + E.bias[c0 + j], 0.f);
                    else x = (r < M && __bfloat162float(E.mask[(size_t)r * E.ldc + c0 + j]) > 0.f) ? v[j] : 0.f;
                    o[j] = __float2bfloat16(x);
                }
                if (lane == 0) bulk_wait_read_all();  // the previous chunk's stores have read the stage
                __syncwarp();
                if (tma_out & 1) {
                    uint4* dst = reinterpret_cast<uint4*>(stC + lane * 32);
                    const uint4* src = reinterpret_cast<const uint4*>(o);
#pragma unroll
                    for (int j = 0; j < 4; ++j) dst[j] = src[j];
                } else if (r < M) {
                    uint4* dst = reinterpret_cast<uint4*>(E.Cb + (size_t)r * E.ldc + c0);
                    const uint4* src = reinterpret_cast<const uint4*>(o);
#pragma unroll
                    for (int j = 0; j < 4; ++j) dst[j] = src[j];
                }
                if (tma_out & 2) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) stT[j * 32 + lane] = o[j];
                } else if (E.CbT && r < M) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) E.CbT[(size_t)(c0 + j) * E.ldt + r] = o[j];
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    if (rg < M) {  // a group wholly beyond the last row stores nothing
                        if (tma_out & 1) tma_store_2d(&mapC, c0, rg, stC);
                        if (tma_out & 2) tma_store_2d(&mapCT, rg, c0, stT);
                    }
                    bulk_commit();
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
        if (lane == 0) bulk_wait_all();  // every store of this warp has completed
    }
    fence_before_sync();
    __syncthreads();
    if (s_abort && threadIdx.x == 0 && E.err) atomicExch(E.err, 1);
    if (warp == 1) tmem_dealloc(tmem, 2u * N);
}

// ------------------------------------------------------------------ host side

// cuTensorMapEncodeTiled, looked up once through the runtime (the library does not link the
// driver library itself).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return static_cast<EncodeTiledFn>(nullptr);
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// Tensor map of a row-major rows x cols BF16 matrix with pitch ld (elements) read in boxes of
// 64 columns x box_rows rows with the 128-byte swizzle; out-of-range elements read as 0.
inline bool make_map(CUtensorMap* map, const bf16* ptr, long long rows, long long cols, long long ld, int box_rows,
                     int box_cols = kBK, bool swizzle = true) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn || (reinterpret_cast<uintptr_t>(ptr) & 15u) || (ld * 2) % 16 != 0 || rows < 1 || cols < 1) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    const cuuint32_t elem[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(ptr), dims, strides, box, elem,
              CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C = A B^T with A: M x K (pitch lda), B: N x K (pitch ldb), both BF16 row-major.  K ranges
// longer than 256 are split over gridDim.y, which needs the atomic epilogue.
template <int N>
cudaError_t gemm_tn(cudaStream_t s, const bf16* A, int M, int K, int lda, const bf16* B, int ldb,
                    const EpiArgs& E) {
    if (M < 1 || K < 1) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, M, K, lda, kBM) || !make_map(&mb, B, N, K, ldb, N)) return cudaErrorInvalidValue;
    const int chunks = (K + kBK - 1) / kBK;
    const int kc = chunks < kMaxChunks ? chunks : kMaxChunks;
    const int splits = (chunks + kc - 1) / kc;
    if (splits > 1 && E.kind != kAtomicF32) return cudaErrorInvalidValue;
    cudaError_t e;
    if constexpr (N == 256) {
        if (splits == 1) {
            // one weight matrix shared by every row block: the persistent kernel keeps it resident
            int dev = 0, sms = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            e = cudaFuncSetAttribute(gemm_tn_resident_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     resident_smem_bytes(N));
            if (e != cudaSuccess) return e;
            // BF16 results (and their transposes) leave through TMA stores of 32 x 32 boxes
            CUtensorMap mc{}, mct{};
            int tma_out = 0;
            if ((E.kind == kReluBiasBf16 || E.kind == kMaskBf16) && E.Cb) {
                if (make_map(&mc, E.Cb, M, N, E.ldc, 32, 32, false)) tma_out |= 1;
                if (E.CbT && make_map(&mct, E.CbT, N, M, E.ldt, 32, 32, false)) tma_out |= 2;
            }
            const int tiles = (M + kBM - 1) / kBM;
            gemm_tn_resident_kernel<N><<<tiles < sms ? tiles : sms, kResThreads, resident_smem_bytes(N), s>>>(
                ma, mb, mc, mct, M, kc, tma_out, E);
            return cudaGetLastError();
        }
    }
    e = cudaFuncSetAttribute(gemm_tn_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(N));
    if (e != cudaSuccess) return e;
    gemm_tn_kernel<N><<<dim3((M + kBM - 1) / kBM, splits), kThreads, smem_bytes(N), s>>>(ma, mb, M, kc, E);
    return cudaGetLastError();
}

}  // namespace tc
}  // namespace drot
