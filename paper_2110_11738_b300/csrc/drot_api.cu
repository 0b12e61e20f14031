// Host driver and C ABI of the DROT solver (declarations and contracts in include/drot.h).
//
// A solve is: argument checks -> marginal sums (one small kernel, read back once) ->
// X_0 = p q^T (cold start) -> a_0, b_0, alpha_0 from the stored X_0 -> repeated
// replays of a CUDA graph that holds `graph_iters` iterations of
// [fused step kernel -> finish kernel] -> duals and nnz export.  The finish kernel
// raises a device flag when the stopping test fires or the iteration cap is reached;
// every later kernel of the graph returns at once, and the host, which keeps two
// replays in flight, stops issuing replays when it reads the flag.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/drot.h"
#include "drot_kernels.cuh"
#include "drot_batched.cuh"
#include "drot_mlp.cuh"
#include "drot_cluster.cuh"
#include "drot_f64.cuh"
#include "drot_grid.cuh"

using drot::Scalars;

namespace {

struct Plan {
    int K = 4, TW = 512, T = 1, G = 1, slots = 1, fin_blocks = 1, graph_iters = 1;
    int variant = 1, S = 0;  // fused-step variant (1 register-fed, 2 TMA-fed) and ring stages
    int accumulate = 1;      // 1: FP64 atomics into row/column totals; 0: fixed-order partials
    std::vector<long long> wbound;  // G+1
    std::vector<int> slot_base;     // G
    std::vector<int> tile_slot;     // T+1
};

struct GraphKey {
    long long m = -1, n = -1, ld = -1;
    const void *C = nullptr, *X = nullptr, *p = nullptr, *q = nullptr;
    const void *arena = nullptr;
    int K = 0, G = 0, graph_iters = 0, profile = 0, variant = 0, accumulate = 0, c_skip = 0, f64 = 0;
    const void *trace = nullptr;
    bool operator==(const GraphKey &o) const {
        return m == o.m && n == o.n && ld == o.ld && C == o.C && X == o.X && p == o.p && q == o.q &&
               arena == o.arena && K == o.K && G == o.G && graph_iters == o.graph_iters && profile == o.profile &&
               variant == o.variant && accumulate == o.accumulate && c_skip == o.c_skip && f64 == o.f64 &&
               trace == o.trace;
    }
};

struct Arena {
    void *ptr = nullptr;
    size_t cap = 0;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Cost model of the CTA work split over row segments (one row of one column tile).
// A warp takes one row segment per memory round trip whatever the segment's width (a
// lane issues all its 16-byte loads of the row at once), so a segment of w columns
// costs w + kRowTripCols column-equivalents: its bytes plus a fixed charge for the
// round trip, the same for every tile width.  Balancing by columns alone would hand
// the m rows of a ragged last tile of a few columns (n = 20000 leaves 32 after 39
// tiles of 512) to one CTA, whose m / 8 round trips per warp would then set the
// step's length (measured on B300: 1.7 TB/s at 20000 x 20000); in a batch it would
// load the CTAs that hold narrow problems with several times too many rows (their
// SMs were busy for the whole launch while the average SM idled a third of it).
// 1536 (three 512-column rows) was the best of 0.25 .. 8 rows and pure row counting
// over square, wide, tall and ragged shapes (6.1 TB/s at 20000 x 20000).  Entering a
// tile costs kTileSwitchCols more, 64 full rows: the column partials of the tile a CTA
// leaves are reduced and flushed and its copy pipeline drains and refills (CTAs whose
// range crossed a tile boundary were the last to finish, by about 5 us, before this
// charge; 64 rows beat 32 in a batch of 512 small problems, 3.77 vs 3.66 TB/s).
constexpr double kRowTripCols = 1536.0;
constexpr double kTileSwitchCols = 64.0 * (512.0 + kRowTripCols);

// Rows the batched narrow-tile kernel packs into one warp iteration for a tile of w valid
// columns (w <= 256): eight up to 128 columns, four up to 256.
inline int packed_rows(long long w) { return w <= 128 ? 8 : (w <= 256 ? 4 : 1); }

struct SegCost {
    long long m, T, TW, last_w;
    double full, last, sw;  // cost of a row segment of a full tile / of the last tile; of a tile start
    // pack: segments of the narrow-tile kernel, whose round-trip charge is shared by the rows
    // one warp iteration packs
    SegCost(long long m_, long long T_, long long TW_, long long n, bool pack = false)
        : m(m_), T(T_), TW(TW_), last_w(n - (T_ - 1) * TW_),
          full((double)TW_ + kRowTripCols / (pack ? packed_rows(TW_) : 1)),
          last((double)last_w + kRowTripCols / (pack ? packed_rows(last_w) : 1)), sw(kTileSwitchCols) {}
    // Cost of the first u segments (tile-major order).
    double before(long long u) const {
        const long long full_units = (T - 1) * m;
        const double rows = u <= full_units ? (double)u * full
                                            : (double)full_units * full + (double)(u - full_units) * last;
        return rows + (double)((u + m - 1) / m) * sw;
    }
    double total() const { return before(T * m); }
    // The number of leading segments whose cost is closest to `cost`.
    long long units_for(double cost) const {
        long long lo = 0, hi = T * m;  // before() is increasing: find the first u with before(u) >= cost
        while (lo < hi) {
            const long long mid = lo + (hi - lo) / 2;
            if (before(mid) < cost) lo = mid + 1;
            else hi = mid;
        }
        if (lo > 0 && cost - before(lo - 1) < before(lo) - cost) --lo;
        return lo;
    }
};

// Ring depth of the TMA-fed step for a tile width (each stage holds 8 rows of X and C).
// K = 4 rings take 160 KB (one CTA per SM); K = 2 and K = 1 rings fit two CTAs per SM.
int tma_stages(int K) { return K == 4 ? 4 : (K == 2 ? 4 : 8); }

// Launch `kernel`; with pdl, as a programmatic dependent of the previous kernel in the
// stream (its launch and set-up overlap that kernel's tail; the kernel itself waits in
// griddepcontrol.wait before reading anything the previous kernel wrote).
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                     Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int K, int S>
cudaError_t set_tma_attr() {
    return cudaFuncSetAttribute(drot::drot_step_tma_kernel<K, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)drot::TmaLayout<K, S>::bytes);
}

template <int K, int S>
cudaError_t set_async_attr() {
    return cudaFuncSetAttribute(drot::drot_step_async_kernel<K, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)drot::AsyncLayout<K, S>::bytes);
}

// Ring depth of the async-copy-fed step per tile width: 96 KB of ring per CTA, two CTAs per SM.
int async_stages(int K) { return K == 4 ? 3 : (K == 2 ? 6 : 12); }

// Cluster-resident solve: cluster size and per-CTA shared memory for a problem, or 0
// if it does not fit on one cluster.
constexpr size_t kClusterSmemMax = 200 * 1024;

struct ClusterPlan {
    int cs = 0, R = 0, Q = 0, npad = 0;
    size_t smem = 0;
};

ClusterPlan cluster_plan(long long m, long long n) {
    ClusterPlan cp;
    for (int cs : {16, 8}) {
        if (m < cs || n < cs) continue;
        const int R = (int)((m + cs - 1) / cs), Q = (int)((n + cs - 1) / cs);
        const int npad = (int)((n + 3) / 4 * 4);
        const size_t bytes = drot::cluster_smem_bytes(R, Q, npad, n, cs);
        if (bytes <= kClusterSmemMax) {
            cp.cs = cs;
            cp.R = R;
            cp.Q = Q;
            cp.npad = npad;
            cp.smem = bytes;
            return cp;
        }
    }
    return cp;
}

// Grid-resident solve: one CTA per SM (at most), rows and columns split evenly, X and C of a
// CTA's rows in its shared memory; 0 CTAs if the rows do not fit.  Chosen automatically from
// kGridMinEntries on: per iteration (µs, streaming graph / grid-resident, B300) 800^2 12.1 / 13.3,
// 1000^2 12.5 / 14.2, 1200^2 14.3 / 16.0, 1400^2 15.3 / 16.2, 1500^2 19.8 / 16.3, 1600^2 20.1 / 17.7,
// 1800^2 21.2 / 18.3: its two grid barriers and FP64 reduction chains cost more than the graph's
// launch chain until the plan is large enough for the streaming step to leave L2-latency territory.
constexpr long long kGridMinEntries = 2000000;
struct GridPlan {
    int G = 0, R = 0, Q = 0, npad = 0;
    size_t smem = 0;
};

GridPlan grid_plan(long long m, long long n, int sms) {
    GridPlan gp;
    if (sms < 1 || m < 1 || n < 1) return gp;
    const long long G0 = std::min<long long>(sms, m);
    const int R = (int)((m + G0 - 1) / G0);
    const int G = (int)((m + R - 1) / R);
    const int Q = (int)((n + G - 1) / G);
    const int npad = (int)((n + 3) / 4 * 4);
    const size_t bytes = drot::grid_smem_bytes(R, Q, npad);
    if (bytes > kClusterSmemMax) return gp;
    gp.G = G;
    gp.R = R;
    gp.Q = Q;
    gp.npad = npad;
    gp.smem = bytes;
    return gp;
}

template <int CS>
cudaError_t launch_cluster(const ClusterPlan &cp, const drot::ClusterArgs &args, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(CS);
    cfg.blockDim = dim3(drot::kClusterThreads);
    cfg.dynamicSmemBytes = cp.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, drot::drot_cluster_kernel<CS>, args);
}

// Opt the ring-fed kernels into their shared-memory size on the current device
// (done once per handle, outside any stream capture).
cudaError_t set_kernel_attributes() {
    cudaError_t e = set_tma_attr<1, 8>();
    if (e == cudaSuccess) e = set_tma_attr<2, 4>();
    if (e == cudaSuccess) e = set_tma_attr<4, 4>();
    if (e == cudaSuccess) e = set_async_attr<1, 12>();
    if (e == cudaSuccess) e = set_async_attr<2, 6>();
    if (e == cudaSuccess) e = set_async_attr<4, 3>();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(drot::drot_cluster_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kClusterSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(drot::drot_cluster_kernel<16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(drot::drot_cluster_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kClusterSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(drot::drot_grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kClusterSmemMax);
    return e;
}

template <int K, int S>
int tma_occupancy() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, drot::drot_step_tma_kernel<K, S>, drot::kThreads + 32,
                                                      drot::TmaLayout<K, S>::bytes) != cudaSuccess)
        return -1;
    return nb;
}

template <int K, int S>
int async_occupancy() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, drot::drot_step_async_kernel<K, S>, drot::kThreads,
                                                      drot::AsyncLayout<K, S>::bytes) != cudaSuccess)
        return -1;
    return nb;
}

template <int K>
int persistent_occupancy() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, drot::drot_persistent_kernel<K>, drot::kThreads, 0) !=
        cudaSuccess)
        return -1;
    return nb;
}

template <int K>
cudaError_t launch_persistent(int G, drot::StepArgs A, drot::FinishArgs F, drot::GridSync *gs, long long budget,
                              cudaStream_t s) {
    void *args[] = {&A, &F, &gs, &budget};
    return cudaLaunchCooperativeKernel(reinterpret_cast<void *>(drot::drot_persistent_kernel<K>), dim3(G),
                                       dim3(drot::kThreads), args, 0, s);
}

template <int K>
int ldg_occupancy() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, drot::drot_step_kernel<K, true>, drot::kThreads, 0) !=
        cudaSuccess)
        return -1;
    return nb;
}

template <int K, int S>
cudaError_t launch_async(int G, const drot::StepArgs &A, cudaStream_t s, bool pdl = false) {
    return launch_k(drot::drot_step_async_kernel<K, S>, dim3(G), dim3(drot::kThreads), drot::AsyncLayout<K, S>::bytes,
                    s, pdl, A);
}

template <int K, int S>
cudaError_t launch_tma(int G, const drot::StepArgs &A, cudaStream_t s, bool pdl = false) {
    return launch_k(drot::drot_step_tma_kernel<K, S>, dim3(G), dim3(drot::kThreads + 32), drot::TmaLayout<K, S>::bytes,
                    s, pdl, A);
}

}  // namespace

struct drot_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    drot_config cfg{};
    int num_sms = 148;

    Arena work;     // solver workspace
    Arena staging;  // device copies for host-pointer calls
    Scalars *d_sc = nullptr;
    Scalars *h_sc = nullptr;      // pinned: upload source
    Scalars *h_status = nullptr;  // pinned: two read-back slots

    // graph cache: two instances (alternating replays keep their profile events apart)
    GraphKey key;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> ev[2];

    // per-solve carved pointers
    double *g = nullptr, *h = nullptr, *a = nullptr, *b = nullptr;
    double *rowpart = nullptr, *colpart = nullptr, *ctapart = nullptr, *finpart = nullptr;
    double *u = nullptr, *v = nullptr, *acc = nullptr;
    drot::GridSync *gsync = nullptr;
    long long *wbound = nullptr;
    int *slot_base = nullptr, *tile_slot = nullptr;

    drot_profile prof{};
    std::string last_error;

    int occ[4][5] = {};  // resident CTAs per SM of the fused step [variant][K]
    int occ_persistent[5] = {};  // resident CTAs per SM of the persistent solve kernel [K]
    struct Tuned {
        long long m, n;
        int variant, K;
    };
    std::vector<Tuned> tuned;  // autotuner choices per problem shape
    Arena tune_x;              // scratch plan the autotuner streams over

    // batched solver state
    Arena batch;                        // per-problem vectors, scalars and work lists
    Scalars *h_bstat = nullptr;         // pinned read-back of every problem's scalars
    size_t h_bstat_cap = 0;
    int batch_k_thresholds[2] = {-1, -1};  // tile policy of the last tuned batch: K = 1 below t0, 2 below t1, else 4
    unsigned long long batch_tuned_sig = 0;  // shape signature of that batch (0: none)
};

namespace {
cudaError_t fill_occupancy(drot_handle *h) {
    const int v[4][5] = {{0, 0, 0, 0, 0},
                         {0, ldg_occupancy<1>(), ldg_occupancy<2>(), 0, ldg_occupancy<4>()},
                         {0, tma_occupancy<1, 8>(), tma_occupancy<2, 4>(), 0, tma_occupancy<4, 4>()},
                         {0, async_occupancy<1, 12>(), async_occupancy<2, 6>(), 0, async_occupancy<4, 3>()}};
    for (int a = 0; a < 4; ++a)
        for (int k = 0; k < 5; ++k) {
            if (v[a][k] < 0) return cudaErrorUnknown;
            h->occ[a][k] = v[a][k];
        }
    const int pk[3] = {persistent_occupancy<1>(), persistent_occupancy<2>(), persistent_occupancy<4>()};
    if (pk[0] < 0 || pk[1] < 0 || pk[2] < 0) return cudaErrorUnknown;
    h->occ_persistent[1] = pk[0];
    h->occ_persistent[2] = pk[1];
    h->occ_persistent[4] = pk[2];
    return cudaSuccess;
}

}  // namespace

namespace {

drot_status fail(drot_handle *h, drot_status s, const char *fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->last_error = buf;
    }
    return s;
}

#define DROT_CUDA(h, call)                                                                          \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            return fail((h), e_ == cudaErrorMemoryAllocation ? DROT_ERR_OOM : DROT_ERR_CUDA,        \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
        }                                                                                           \
    } while (0)

drot_status arena_reserve(drot_handle *h, Arena &ar, size_t bytes) {
    if (ar.cap >= bytes) return DROT_OK;
    if (ar.ptr) {
        DROT_CUDA(h, cudaStreamSynchronize(h->stream));
        DROT_CUDA(h, cudaFree(ar.ptr));
        ar.ptr = nullptr;
        ar.cap = 0;
    }
    size_t cap = align_up(bytes + bytes / 4, 1 << 20);
    DROT_CUDA(h, cudaMalloc(&ar.ptr, cap));
    ar.cap = cap;
    return DROT_OK;
}

bool is_device_ptr(const void *p, int device) {
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) && attr.device == device;
}

// Choose the tile width, the grid and the per-CTA segment ranges.  Segment
// ranges are balanced by SegCost (a row of a ragged last tile costs less than a
// full one, but not in proportion to its width), and slots are numbered in CTA
// order, which is also column-tile order.
void make_plan(const drot_handle *h, long long m, long long n, Plan &P, int force_variant = 0, int force_k = 0) {
    int K = force_k ? force_k : h->cfg.tile_k;
    int variant = force_variant ? force_variant : h->cfg.step_variant;
    if (!force_k && !force_variant && h->cfg.autotune) {
        for (const auto &t : h->tuned)
            if (t.m == m && t.n == n) {
                if (K != 1 && K != 2 && K != 4) K = t.K;
                if (variant < 1 || variant > 3) variant = t.variant;
            }
    }
    if (K != 1 && K != 2 && K != 4) {
        // the widest tile the rows fill ...
        if (n >= 1536) K = 4;
        else if (n >= 384) K = 2;
        else K = 1;
        // ... but a plan of a few million entries sits in L2, where a pass is bound by the
        // latency of each warp's row round trips rather than by bandwidth, and narrower tiles
        // put more row segments in flight.  Measured per iteration on B300 (128- / 256- /
        // 512-column tiles): 1024^2 14.7 / 15.8 / 20.0 µs, 1536^2 17.7 / 17.6 / 21.5,
        // 2048^2 20.6 / 20.0 / 22.8, 700 x 5000 20.4 / 19.9 / 22.7; 3072^2 34.2 / 30.0 / 28.6
        const double entries = (double)m * (double)n;
        if (entries <= 1.5e6) K = 1;
        else if (entries <= 6.0e6) K = std::min(K, 2);
    }
    P.K = K;
    P.TW = 128 * K;
    P.T = (int)((n + P.TW - 1) / P.TW);
    const long long units = (long long)P.T * m;
    if (variant < 1 || variant > 3) variant = 1;
    P.variant = variant;
    P.S = variant == 2 ? tma_stages(K) : (variant == 3 ? async_stages(K) : 0);
    P.accumulate = h->cfg.deterministic ? 0 : 1;
    if (h->cfg.persistent || h->cfg.c_skip) {
        P.variant = variant = 1;
        P.S = 0;
    }
    if (h->cfg.persistent) P.accumulate = 1;
    int G = h->cfg.grid_ctas;
    if (G <= 0) {
        // as many CTAs as fit on the SMs at once (one wave); small problems use fewer
        // CTAs so that each warp has rows
        const long long want = (units + drot::kWarps - 1) / drot::kWarps;
        const long long per_sm = std::max(1, h->cfg.persistent ? h->occ_persistent[K] : h->occ[variant][K]);
        G = (int)std::min<long long>(per_sm * h->num_sms, std::max<long long>(1, want));
    }
    G = (int)std::min<long long>(G, std::max<long long>(1, units));
    // a cooperative launch needs every CTA resident at once
    if (h->cfg.persistent) G = std::min(G, std::max(1, h->occ_persistent[K]) * h->num_sms);
    P.G = G;

    const SegCost cost(m, P.T, P.TW, n);
    const double total_cost = cost.total();
    P.wbound.assign(G + 1, 0);
    for (int g = 1; g < G; ++g) P.wbound[g] = std::max(P.wbound[g - 1], cost.units_for(total_cost * g / G));
    P.wbound[G] = units;

    P.slot_base.assign(G, 0);
    std::vector<int> slot_tile;
    for (int g = 0; g < G; ++g) {
        P.slot_base[g] = (int)slot_tile.size();
        const long long w0 = P.wbound[g], w1 = P.wbound[g + 1];
        if (w1 <= w0) continue;
        for (long long t = w0 / m; t <= (w1 - 1) / m; ++t) slot_tile.push_back((int)t);
    }
    P.slots = std::max<int>(1, (int)slot_tile.size());
    P.tile_slot.assign(P.T + 1, (int)slot_tile.size());
    for (int t = P.T - 1; t >= 0; --t) {
        int first = P.tile_slot[t + 1];
        for (int s = (int)slot_tile.size() - 1; s >= 0; --s)
            if (slot_tile[s] >= t) first = std::min(first, s);
        P.tile_slot[t] = first;
    }
    const long long mn = m + n;
    P.fin_blocks = (int)std::min<long long>(2LL * h->num_sms,
                                            std::max<long long>(1, (mn + drot::kFinishThreads - 1) / drot::kFinishThreads));
    if (h->cfg.persistent) P.fin_blocks = G;  // the finish phase runs on the same CTAs

    int gi = h->cfg.graph_iters;
    if (gi <= 0) {
        const double t_iter = 12.0 * (double)m * (double)n / 6.0e12 + 6.0e-6;
        gi = (int)std::lround(2.0e-3 / t_iter);
        gi = std::max(1, std::min(gi, 256));
        // serpentine passes alternate by their position in the replay: an even count
        // keeps the alternation across replay boundaries
        if (h->cfg.serpentine >= 0) gi = std::max(2, gi + (gi & 1));
    }
    if (h->cfg.c_skip) gi = std::max(2, gi + (gi & 1));  // whole (C-reading, C-free) pairs per replay
    P.graph_iters = gi;
}

template <typename T>
T *carve(char *&cur, size_t count) {
    T *p = reinterpret_cast<T *>(cur);
    cur += align_up(count * sizeof(T), 256);
    return p;
}

drot_status setup_workspace(drot_handle *h, long long m, long long n, const Plan &P) {
    const size_t bytes = align_up(sizeof(double) * m, 256) * 3 + align_up(sizeof(double) * n, 256) * 2 +
                         align_up(sizeof(double) * (size_t)P.T * m, 256) +
                         align_up(sizeof(double) * (size_t)P.slots * P.TW, 256) +
                         align_up(sizeof(double) * 2 * P.G, 256) +
                         align_up(sizeof(double) * drot::kFinishAcc * P.fin_blocks, 256) +
                         align_up(sizeof(long long) * (P.G + 1), 256) + align_up(sizeof(int) * P.G, 256) +
                         align_up(sizeof(int) * (P.T + 1), 256) + align_up(sizeof(double) * m, 256) +
                         align_up(sizeof(double) * n, 256) +
                         align_up(sizeof(double) * drot::kAccSlots * drot::kAccStride, 256) +
                         align_up(sizeof(drot::GridSync), 256) + 4096;
    drot_status st = arena_reserve(h, h->work, bytes);
    if (st != DROT_OK) return st;
    char *cur = static_cast<char *>(h->work.ptr);
    h->g = carve<double>(cur, m);
    h->a = carve<double>(cur, m);
    carve<double>(cur, m);  // spare row vector (keeps the layout stable)
    h->h = carve<double>(cur, n);
    h->b = carve<double>(cur, n);
    h->rowpart = carve<double>(cur, (size_t)P.T * m);
    h->colpart = carve<double>(cur, (size_t)P.slots * P.TW);
    h->ctapart = carve<double>(cur, 2 * (size_t)P.G);
    h->finpart = carve<double>(cur, (size_t)drot::kFinishAcc * P.fin_blocks);
    h->wbound = carve<long long>(cur, P.G + 1);
    h->slot_base = carve<int>(cur, P.G);
    h->tile_slot = carve<int>(cur, P.T + 1);
    h->u = carve<double>(cur, m);
    h->v = carve<double>(cur, n);
    h->acc = carve<double>(cur, (size_t)drot::kAccSlots * drot::kAccStride);
    h->gsync = carve<drot::GridSync>(cur, 1);
    DROT_CUDA(h, cudaMemsetAsync(h->gsync, 0, sizeof(drot::GridSync), h->stream));
    if (h->cfg.wait_limit > 0) {
        const unsigned long long lim = (unsigned long long)h->cfg.wait_limit;
        DROT_CUDA(h, cudaMemcpyAsync(&h->gsync->spin_limit, &lim, sizeof lim, cudaMemcpyHostToDevice, h->stream));
        DROT_CUDA(h, cudaStreamSynchronize(h->stream));  // lim lives on this stack frame
    }
    if (P.accumulate) {
        // totals start at zero; every finish pass resets what it reads
        DROT_CUDA(h, cudaMemsetAsync(h->u, 0, sizeof(double) * m, h->stream));
        DROT_CUDA(h, cudaMemsetAsync(h->v, 0, sizeof(double) * n, h->stream));
        DROT_CUDA(h, cudaMemsetAsync(h->acc, 0, sizeof(double) * drot::kAccSlots * drot::kAccStride, h->stream));
    }
    DROT_CUDA(h, cudaMemcpyAsync(h->wbound, P.wbound.data(), sizeof(long long) * (P.G + 1), cudaMemcpyHostToDevice,
                                 h->stream));
    DROT_CUDA(h, cudaMemcpyAsync(h->slot_base, P.slot_base.data(), sizeof(int) * P.G, cudaMemcpyHostToDevice,
                                 h->stream));
    DROT_CUDA(h, cudaMemcpyAsync(h->tile_slot, P.tile_slot.data(), sizeof(int) * (P.T + 1), cudaMemcpyHostToDevice,
                                 h->stream));
    return DROT_OK;
}

drot::StepArgs step_args(const drot_handle *h, const Plan &P, long long m, long long n, long long ld, const float *C,
                         float *X) {
    drot::StepArgs A{};
    A.u = h->u;
    A.v = h->v;
    A.acc = h->acc;
    A.accumulate = P.accumulate;
    A.serp = h->cfg.serpentine >= 0 ? 1 : 0;
    A.odd = 0;  // set per launch by the launcher
    A.C = C;
    A.X = X;
    A.g = h->g;
    A.h = h->h;
    A.sc = h->d_sc;
    A.rowpart = h->rowpart;
    A.colpart = h->colpart;
    A.ctapart = h->ctapart;
    A.wbound = h->wbound;
    A.slot_base = h->slot_base;
    A.m = m;
    A.n = n;
    A.ld = ld;
    A.inv_n = 1.0 / (double)n;
    A.inv_m = 1.0 / (double)m;
    return A;
}

drot::FinishArgs finish_args(const drot_handle *h, long long m, long long n, const Plan &P, const double *p,
                             const double *q) {
    drot::FinishArgs F{};
    F.u = h->u;
    F.v = h->v;
    F.acc = h->acc;
    F.accumulate = P.accumulate;
    F.rowpart = h->rowpart;
    F.colpart = h->colpart;
    F.ctapart = h->ctapart;
    F.tile_slot = h->tile_slot;
    F.p = p;
    F.q = q;
    F.a = h->a;
    F.b = h->b;
    F.g = h->g;
    F.h = h->h;
    F.finpart = h->finpart;
    F.sc = h->d_sc;
    F.m = m;
    F.n = n;
    F.T = P.T;
    F.TW = P.TW;
    F.G = P.G;
    F.inv_n = 1.0 / (double)n;
    F.inv_m = 1.0 / (double)m;
    F.inv_mn = 1.0 / (double)(m + n);
    F.trace = h->cfg.trace;
    F.trace_len = h->cfg.trace ? h->cfg.trace_len : 0;
    return F;
}

// Register-fed step in a C-skipping mode (1: read X and C, store X - rho C; 2: read that array only).
cudaError_t launch_step_cskip(const Plan &P, const drot::StepArgs &A, int cm, cudaStream_t s, bool pdl = false) {
    const dim3 g(P.G), b(drot::kThreads);
    if (cm == 1) {
        switch (P.K) {
            case 1: return launch_k(drot::drot_step_kernel<1, true, 1>, g, b, 0, s, pdl, A);
            case 2: return launch_k(drot::drot_step_kernel<2, true, 1>, g, b, 0, s, pdl, A);
            default: return launch_k(drot::drot_step_kernel<4, true, 1>, g, b, 0, s, pdl, A);
        }
    }
    switch (P.K) {
        case 1: return launch_k(drot::drot_step_kernel<1, true, 2>, g, b, 0, s, pdl, A);
        case 2: return launch_k(drot::drot_step_kernel<2, true, 2>, g, b, 0, s, pdl, A);
        default: return launch_k(drot::drot_step_kernel<4, true, 2>, g, b, 0, s, pdl, A);
    }
}

template <bool UPDATE>
cudaError_t launch_step(const Plan &P, const drot::StepArgs &A, cudaStream_t s, bool pdl = false) {
    if (UPDATE && P.variant == 3) {
        switch (P.K) {
            case 1: return launch_async<1, 12>(P.G, A, s, pdl);
            case 2: return launch_async<2, 6>(P.G, A, s, pdl);
            default: return launch_async<4, 3>(P.G, A, s, pdl);
        }
    }
    if (UPDATE && P.variant == 2) {
        switch (P.K) {
            case 1: return launch_tma<1, 8>(P.G, A, s, pdl);
            case 2: return launch_tma<2, 4>(P.G, A, s, pdl);
            default: return launch_tma<4, 4>(P.G, A, s, pdl);
        }
    }
    const dim3 g(P.G), b(drot::kThreads);
    switch (P.K) {
        case 1: return launch_k(drot::drot_step_kernel<1, UPDATE>, g, b, 0, s, pdl, A);
        case 2: return launch_k(drot::drot_step_kernel<2, UPDATE>, g, b, 0, s, pdl, A);
        default: return launch_k(drot::drot_step_kernel<4, UPDATE>, g, b, 0, s, pdl, A);
    }
}

// The FP64 fused step (one variant; tiles of drot::kTileW64 columns, i.e. K = 2).
template <bool UPDATE>
cudaError_t launch_step64(const Plan &P, const drot::StepArgs64 &A, cudaStream_t s, bool pdl = false) {
    return launch_k(drot::drot_step_f64_kernel<UPDATE>, dim3(P.G), dim3(drot::kThreads), 0, s, pdl, A);
}

void destroy_graphs(drot_handle *h) {
    for (int i = 0; i < 2; ++i) {
        if (h->exec[i]) cudaGraphExecDestroy(h->exec[i]);
        h->exec[i] = nullptr;
        for (cudaEvent_t e : h->ev[i]) cudaEventDestroy(e);
        h->ev[i].clear();
    }
    h->key = GraphKey{};
}

// Capture `graph_iters` iterations of [step -> finish] into two executable graphs.
drot_status build_graphs(drot_handle *h, const GraphKey &key, const Plan &P, const drot::StepArgs &A,
                         const drot::FinishArgs &F, const drot::StepArgs64 *A64 = nullptr) {
    destroy_graphs(h);
    const bool prof = key.profile != 0;
    for (int inst = 0; inst < 2; ++inst) {
        if (prof) {
            h->ev[inst].resize(3 * P.graph_iters + 1);
            for (auto &e : h->ev[inst]) DROT_CUDA(h, cudaEventCreate(&e));
        }
        cudaGraph_t graph = nullptr;
        DROT_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t err = cudaSuccess;
        // profile events per iteration: [3 it] before the step, [3 it + 1] between step and
        // finish, [3 it + 2] after the finish; [3 G] closes the last iteration
        for (int it = 0; it < P.graph_iters && err == cudaSuccess; ++it) {
            const bool cskip = key.c_skip != 0;
            if (prof) err = cudaEventRecordWithFlags(h->ev[inst][3 * it], h->stream, cudaEventRecordExternal);
            const bool pdl = !prof;  // an event record between kernels would break the programmatic edge
            drot::StepArgs Ai = A;
            Ai.odd = it & 1;  // odd positions walk backwards when A.serp is set
            if (err == cudaSuccess)
                err = A64     ? launch_step64<true>(P, *A64, h->stream, pdl)
                      : cskip ? launch_step_cskip(P, Ai, (it & 1) ? 2 : 1, h->stream, pdl)
                              : launch_step<true>(P, Ai, h->stream, pdl);
            if (prof && err == cudaSuccess)
                err = cudaEventRecordWithFlags(h->ev[inst][3 * it + 1], h->stream, cudaEventRecordExternal);
            if (err == cudaSuccess) {
                drot::FinishArgs Fi = F;
                Fi.no_test = (cskip && (it & 1)) ? 1 : 0;
                err = launch_k(drot::drot_finish_kernel, dim3(P.fin_blocks), dim3(drot::kFinishThreads), 0, h->stream,
                               pdl, Fi);
            }
            if (prof && err == cudaSuccess)
                err = cudaEventRecordWithFlags(h->ev[inst][3 * it + 2], h->stream, cudaEventRecordExternal);
        }
        cudaError_t end = cudaStreamEndCapture(h->stream, &graph);
        if (err != cudaSuccess || end != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(h, DROT_ERR_CUDA, "graph capture failed: %s",
                        cudaGetErrorString(err != cudaSuccess ? err : end));
        }
        cudaError_t ie = cudaGraphInstantiate(&h->exec[inst], graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return fail(h, DROT_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ie));
    }
    h->key = key;
    return DROT_OK;
}

// Time every fused-step plan candidate (variant x tile width) for this shape on a
// scratch plan, six launches each after one warm-up, and keep the fastest (with a
// 3 % margin in favour of the untuned plan).
// Runs after the scalar state is uploaded (the kernels read rho and the done flag);
// the real plan's set-up afterwards re-zeroes every total the candidates touched.
drot_status autotune_shape(drot_handle *h, long long m, long long n, long long ld, const float *C) {
    for (const auto &t : h->tuned)
        if (t.m == m && t.n == n) return DROT_OK;
    const size_t bytes = sizeof(float) * (size_t)m * ld;
    drot_status st = arena_reserve(h, h->tune_x, bytes);
    if (st != DROT_OK) return st;
    float *Xs = static_cast<float *>(h->tune_x.ptr);
    DROT_CUDA(h, cudaMemsetAsync(Xs, 0, bytes, h->stream));
    cudaEvent_t e0, e1;
    DROT_CUDA(h, cudaEventCreate(&e0));
    DROT_CUDA(h, cudaEventCreate(&e1));
    float best = 1e30f, dflt = 0.f;
    int best_v = 1, best_k = 1;
    const int dflt_k = n >= 1536 ? 4 : (n >= 384 ? 2 : 1);  // make_plan's choice without tuning
    drot_status out = DROT_OK;
    for (int variant = 1; variant <= 3 && out == DROT_OK; ++variant) {
        for (int K : {1, 2, 4}) {
            if (K > 1 && n < 64LL * K) continue;  // a tile more than twice the row width leaves most lanes idle
            Plan P;
            make_plan(h, m, n, P, variant, K);
            out = setup_workspace(h, m, n, P);
            if (out != DROT_OK) break;
            DROT_CUDA(h, cudaMemsetAsync(h->g, 0, sizeof(double) * m, h->stream));
            DROT_CUDA(h, cudaMemsetAsync(h->h, 0, sizeof(double) * n, h->stream));
            // alternating directions, as the solve runs them (the warm-up pass is odd, so
            // the first timed pass follows a backward one)
            drot::StepArgs A = step_args(h, P, m, n, ld, C, Xs);
            A.odd = 1;
            DROT_CUDA(h, launch_step<true>(P, A, h->stream));
            DROT_CUDA(h, cudaEventRecord(e0, h->stream));
            for (int r = 0; r < 6; ++r) {
                A.odd = r & 1;
                DROT_CUDA(h, launch_step<true>(P, A, h->stream));
            }
            DROT_CUDA(h, cudaEventRecord(e1, h->stream));
            DROT_CUDA(h, cudaEventSynchronize(e1));
            h->prof.kernel_launches += 7;
            float ms = 0.f;
            DROT_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
            if (variant == 1 && K == dflt_k) dflt = ms;
            if (ms < best) {
                best = ms;
                best_v = variant;
                best_k = K;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (out != DROT_OK) return out;
    // Keep the untuned choice unless a candidate beats it by 3 %: near-ties would
    // otherwise flip between runs on timing noise.
    if (dflt > 0.f && best > 0.97f * dflt) {
        best_v = 1;
        best_k = dflt_k;
    }
    h->tuned.push_back({m, n, best_v, best_k});
    return DROT_OK;
}

// The solve on device pointers.  f64: C and X are FP64 (drot_solve_f64), else FP32.
drot_status solve_device(drot_handle *h, long long m, long long n, const void *Cv, long long ld, const double *p,
                         const double *q, double rho, double tol, long long max_iter, void *Xv, double *mu,
                         double *nu, int warm, drot_result *res, bool f64 = false) {
    drot_status st = DROT_OK;
    const float *C = f64 ? nullptr : static_cast<const float *>(Cv);
    float *X = f64 ? nullptr : static_cast<float *>(Xv);
    const double *C64 = f64 ? static_cast<const double *>(Cv) : nullptr;
    double *X64 = f64 ? static_cast<double *>(Xv) : nullptr;
    // scalar state; marginal sums and the warm duals' sums first
    Scalars &S = *h->h_sc;
    std::memset(&S, 0, sizeof S);
    S.rho = rho;
    S.inv_rho = 1.0 / rho;
    S.tol = tol;
    S.max_iter = max_iter;
    S.stop_rule = (h->cfg.stop_rule & 7) ? (h->cfg.stop_rule & 7) : (DROT_STOP_GAP | DROT_STOP_RES_L1);
    S.done = drot::kRunning;
    DROT_CUDA(h, cudaMemcpyAsync(h->d_sc, &S, sizeof S, cudaMemcpyHostToDevice, h->stream));
    drot::drot_vector_sums_kernel<<<1, 1024, 0, h->stream>>>(p, q, warm ? mu : nullptr, warm ? nu : nullptr, m, n,
                                                             h->d_sc);
    DROT_CUDA(h, cudaGetLastError());
    h->prof.kernel_launches += 1;
    DROT_CUDA(h, cudaMemcpyAsync(h->h_status, h->d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
    DROT_CUDA(h, cudaStreamSynchronize(h->stream));
    const Scalars chk = *h->h_status;
    if (chk.nonfinite_input & 3)
        return fail(h, DROT_ERR_MARGINALS, "p or q has a negative or non-finite entry");
    if (chk.nonfinite_input & 4) return fail(h, DROT_ERR_INVALID_ARG, "warm-start duals are not finite");
    if (!(std::fabs(chk.sum_p - chk.sum_q) <= 1e-9 * std::max(1.0, std::fabs(chk.sum_p))))
        return fail(h, DROT_ERR_MARGINALS, "sum(p) = %.17g and sum(q) = %.17g differ", chk.sum_p, chk.sum_q);

    if (f64 && (h->cfg.persistent || h->cfg.c_skip))
        return fail(h, DROT_ERR_INVALID_ARG, "the FP64 solve has no persistent or C-skipping mode");
    if (h->cfg.autotune && !f64) {
        st = autotune_shape(h, m, n, ld, C);
        if (st != DROT_OK) return st;
    }
    Plan P;
    if (f64) make_plan(h, m, n, P, 1, drot::kTileW64 / 128);  // one FP64 variant, 256-column tiles
    else make_plan(h, m, n, P);
    st = setup_workspace(h, m, n, P);
    if (st != DROT_OK) return st;

    // X_0 and the state derived from it
    if (!warm) {
        const long long work = f64 ? m * n : m * ((n + 3) / 4);
        const int blocks = (int)std::min<long long>(8LL * h->num_sms, std::max<long long>(1, (work + 255) / 256));
        if (f64) drot::drot_init_plan_f64_kernel<<<blocks, 256, 0, h->stream>>>(X64, p, q, m, n, ld);
        else drot::drot_init_plan_kernel<<<blocks, 256, 0, h->stream>>>(X, p, q, m, n, ld);
        DROT_CUDA(h, cudaGetLastError());
        h->prof.kernel_launches += 1;
    }
    const drot::StepArgs A = step_args(h, P, m, n, ld, C, X);
    const drot::FinishArgs F = finish_args(h, m, n, P, p, q);
    const drot::StepArgs64 A64{A, C64, X64};
    DROT_CUDA(h, f64 ? launch_step64<false>(P, A64, h->stream) : launch_step<false>(P, A, h->stream));
    drot::drot_init_state_kernel<<<P.fin_blocks, drot::kFinishThreads, 0, h->stream>>>(F, warm ? mu : nullptr,
                                                                                      warm ? nu : nullptr);
    DROT_CUDA(h, cudaGetLastError());
    h->prof.kernel_launches += 2;

    long long iters_done = 0;
    int done = max_iter > 0 ? drot::kRunning : drot::kIterCap;
    const ClusterPlan cp = cluster_plan(m, n);
    // automatic: only when no setting asks for the streaming path explicitly
    const bool explicit_stream = h->cfg.step_variant != 0 || h->cfg.tile_k != 0 || h->cfg.grid_ctas != 0 ||
                                 h->cfg.persistent || h->cfg.deterministic || h->cfg.c_skip || h->cfg.trace;
    const bool use_cluster = cp.cs > 0 && !h->cfg.c_skip && !f64 &&
                             (h->cfg.cluster == 2 || (h->cfg.cluster == 0 && !explicit_stream));
    if (h->cfg.cluster == 2 && f64)
        return fail(h, DROT_ERR_INVALID_ARG, "the cluster-resident solve is FP32 only");
    if (h->cfg.cluster == 2 && !use_cluster)
        return fail(h, DROT_ERR_INVALID_ARG, "a %lld x %lld problem does not fit on one cluster", m, n);
    // grid-resident: rows of X and C in the shared memory of one CTA per SM (mid-size problems)
    const GridPlan gp = use_cluster ? GridPlan{} : grid_plan(m, n, h->num_sms);
    const bool psi_fits = (size_t)P.slots * P.TW * sizeof(double) >= (size_t)n * sizeof(float);
    const bool use_grid = !use_cluster && gp.G > 0 && psi_fits && !h->cfg.c_skip && !f64 &&
                          (h->cfg.cluster == 3 ||
                           (h->cfg.cluster == 0 && !explicit_stream && m * n >= kGridMinEntries));
    if (h->cfg.cluster == 3 && !use_grid)
        return fail(h, DROT_ERR_INVALID_ARG, "a %lld x %lld problem does not fit the grid-resident solve", m, n);
    if (max_iter > 0 && use_grid) {
        // one cooperative launch (one CTA per SM at most) runs up to `budget` iterations
        drot::GridArgs ga{};
        drot::ClusterArgs &ca = ga.P;
        ca.C = C;
        ca.X = X;
        ca.p = p;
        ca.q = q;
        ca.g = h->g;
        ca.h = h->h;
        ca.a = h->a;
        ca.b = h->b;
        ca.sc = h->d_sc;
        ca.m = m;
        ca.n = n;
        ca.ld = ld;
        ca.rows_per_cta = gp.R;
        ca.cols_per_cta = gp.Q;
        ca.npad = gp.npad;
        ca.inv_n = 1.0 / (double)n;
        ca.inv_m = 1.0 / (double)m;
        ca.inv_mn = 1.0 / (double)(m + n);
        ca.budget = std::min<long long>(max_iter, 200000);
        ga.v = h->v;
        ga.psi_g = reinterpret_cast<float *>(h->colpart);
        ga.totals = h->acc;
        ga.bar = &h->gsync->count;
        const long long max_launches = (max_iter + ca.budget - 1) / ca.budget + 2;
        for (long long l = 0; l < max_launches; ++l) {
            DROT_CUDA(h, cudaMemsetAsync(ga.v, 0, sizeof(double) * (size_t)n, h->stream));
            DROT_CUDA(h, cudaMemsetAsync(ga.totals, 0, sizeof(double) * 2 * drot::kGridTotals, h->stream));
            DROT_CUDA(h, cudaMemsetAsync(ga.bar, 0, sizeof(unsigned int), h->stream));
            void *kargs[] = {&ga};
            const cudaError_t e = cudaLaunchCooperativeKernel((const void *)drot::drot_grid_kernel, dim3(gp.G),
                                                              dim3(drot::kGridThreads), kargs, gp.smem, h->stream);
            if (e != cudaSuccess) return fail(h, DROT_ERR_CUDA, "grid-resident launch failed: %s", cudaGetErrorString(e));
            h->prof.kernel_launches += 1;
            DROT_CUDA(h, cudaMemcpyAsync(h->h_status, h->d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
            DROT_CUDA(h, cudaStreamSynchronize(h->stream));
            if (h->h_status->done != drot::kRunning || h->h_status->fault) {
                done = h->h_status->fault ? drot::kFault : h->h_status->done;
                break;
            }
        }
        if (done == drot::kRunning) return fail(h, DROT_ERR_CUDA, "grid-resident iteration did not report completion");
    } else if (max_iter > 0 && use_cluster) {
        // whole solve on one cluster; a launch runs up to `budget` iterations
        drot::ClusterArgs ca{};
        ca.C = C;
        ca.X = X;
        ca.p = p;
        ca.q = q;
        ca.g = h->g;
        ca.h = h->h;
        ca.a = h->a;
        ca.b = h->b;
        ca.sc = h->d_sc;
        ca.m = m;
        ca.n = n;
        ca.ld = ld;
        ca.rows_per_cta = cp.R;
        ca.cols_per_cta = cp.Q;
        ca.npad = cp.npad;
        ca.inv_n = 1.0 / (double)n;
        ca.inv_m = 1.0 / (double)m;
        ca.inv_mn = 1.0 / (double)(m + n);
        ca.budget = std::min<long long>(max_iter, 200000);
        const long long max_launches = (max_iter + ca.budget - 1) / ca.budget + 2;
        for (long long l = 0; l < max_launches; ++l) {
            const cudaError_t e = cp.cs == 16 ? launch_cluster<16>(cp, ca, h->stream) : launch_cluster<8>(cp, ca, h->stream);
            if (e != cudaSuccess) return fail(h, DROT_ERR_CUDA, "cluster launch failed: %s", cudaGetErrorString(e));
            h->prof.kernel_launches += 1;
            DROT_CUDA(h, cudaMemcpyAsync(h->h_status, h->d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
            DROT_CUDA(h, cudaStreamSynchronize(h->stream));
            if (h->h_status->done != drot::kRunning) {
                done = h->h_status->done;
                break;
            }
        }
        if (done == drot::kRunning) return fail(h, DROT_ERR_CUDA, "cluster iteration did not report completion");
        h->prof.step_variant = 4;  // cluster-resident
    } else if (max_iter > 0 && h->cfg.persistent) {
        // one cooperative launch runs up to `budget` iterations (about half a second of work)
        const double t_iter = 12.0 * (double)m * (double)n / 6.0e12 + 8.0e-6;
        const long long budget = std::max(1LL, std::min<long long>(max_iter, std::llround(0.5 / t_iter)));
        const long long max_launches = (max_iter + budget - 1) / budget + 2;
        for (long long l = 0; l < max_launches; ++l) {
            cudaError_t e = cudaMemsetAsync(&h->gsync->count, 0, sizeof(unsigned int), h->stream);  // barrier counter
            if (e != cudaSuccess) return fail(h, DROT_ERR_CUDA, "barrier reset failed: %s", cudaGetErrorString(e));
            switch (P.K) {
                case 1: e = launch_persistent<1>(P.G, A, F, h->gsync, budget, h->stream); break;
                case 2: e = launch_persistent<2>(P.G, A, F, h->gsync, budget, h->stream); break;
                default: e = launch_persistent<4>(P.G, A, F, h->gsync, budget, h->stream); break;
            }
            if (e != cudaSuccess) return fail(h, DROT_ERR_CUDA, "cooperative launch failed: %s", cudaGetErrorString(e));
            h->prof.kernel_launches += 1;
            DROT_CUDA(h, cudaMemcpyAsync(h->h_status, h->d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
            DROT_CUDA(h, cudaStreamSynchronize(h->stream));
            if (h->h_status->done != drot::kRunning || h->h_status->fault) {
                done = h->h_status->fault ? drot::kFault : h->h_status->done;
                break;
            }
        }
        drot::GridSync gs{};
        DROT_CUDA(h, cudaMemcpy(&gs, h->gsync, sizeof gs, cudaMemcpyDeviceToHost));
        h->prof.step_ms_total += (double)gs.step_ns * 1e-6;
        h->prof.step_launches += (long long)gs.iters;
        if (done == drot::kRunning)
            return fail(h, DROT_ERR_CUDA, "persistent iteration did not report completion");
    } else if (max_iter > 0) {
        GraphKey key;
        key.m = m; key.n = n; key.ld = ld; key.C = Cv; key.X = Xv; key.p = p; key.q = q;
        key.f64 = f64 ? 1 : 0;
        key.trace = h->cfg.trace;
        key.arena = h->work.ptr; key.K = P.K; key.G = P.G; key.graph_iters = P.graph_iters;
        key.variant = P.variant;
        key.accumulate = P.accumulate;
        key.c_skip = h->cfg.c_skip ? 1 : 0;
        key.profile = h->cfg.profile ? 1 : 0;
        if (!(key == h->key) || !h->exec[0]) {
            st = build_graphs(h, key, P, A, F, f64 ? &A64 : nullptr);
            if (st != DROT_OK) return st;
        }
        // keep two replays in flight; slot r%2 of h_status receives replay r's state
        const long long max_replays = (max_iter + P.graph_iters - 1) / P.graph_iters + 2;
        cudaEvent_t copied[2];
        DROT_CUDA(h, cudaEventCreateWithFlags(&copied[0], cudaEventDisableTiming));
        DROT_CUDA(h, cudaEventCreateWithFlags(&copied[1], cudaEventDisableTiming));
        long long issued = 0, consumed = 0, k_prev = 0;
        drot_status loop_st = DROT_OK;
        auto issue = [&](long long r) -> cudaError_t {
            const int inst = (int)(r & 1);
            cudaError_t e = cudaGraphLaunch(h->exec[inst], h->stream);
            if (e != cudaSuccess) return e;
            e = cudaMemcpyAsync(h->h_status + inst, h->d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream);
            if (e != cudaSuccess) return e;
            h->prof.graph_replays += 1;
            h->prof.kernel_launches += 2LL * P.graph_iters;
            return cudaEventRecord(copied[inst], h->stream);
        };
        while (true) {
            while (issued < consumed + 2 && issued < max_replays) {
                cudaError_t e = issue(issued);
                if (e != cudaSuccess) {
                    loop_st = fail(h, DROT_ERR_CUDA, "graph replay failed: %s", cudaGetErrorString(e));
                    break;
                }
                ++issued;
            }
            if (loop_st != DROT_OK || consumed >= issued) break;
            const int inst = (int)(consumed & 1);
            cudaError_t e = cudaEventSynchronize(copied[inst]);
            if (e != cudaSuccess) {
                loop_st = fail(h, DROT_ERR_CUDA, "replay wait failed: %s", cudaGetErrorString(e));
                break;
            }
            const Scalars s = h->h_status[inst];
            if (h->cfg.profile) {
                const long long ran = s.k - k_prev;
                for (long long it = 0; it < ran && it < P.graph_iters; ++it) {
                    float ms = 0.f, fms = 0.f, ims = 0.f;
                    if (cudaEventElapsedTime(&ms, h->ev[inst][3 * it], h->ev[inst][3 * it + 1]) == cudaSuccess &&
                        cudaEventElapsedTime(&fms, h->ev[inst][3 * it + 1], h->ev[inst][3 * it + 2]) == cudaSuccess &&
                        cudaEventElapsedTime(&ims, h->ev[inst][3 * it], h->ev[inst][3 * it + 2]) == cudaSuccess) {
                        h->prof.step_ms_total += ms;
                        h->prof.finish_ms_total += fms;
                        h->prof.iter_ms_total += ims;
                        h->prof.step_launches += 1;
                    }
                }
            }
            k_prev = s.k;
            ++consumed;
            if (s.done != drot::kRunning) {
                done = s.done;
                break;
            }
        }
        cudaError_t se = cudaStreamSynchronize(h->stream);
        cudaEventDestroy(copied[0]);
        cudaEventDestroy(copied[1]);
        if (loop_st != DROT_OK) return loop_st;
        if (se != cudaSuccess) return fail(h, DROT_ERR_CUDA, "stream sync failed: %s", cudaGetErrorString(se));
        if (done == drot::kRunning)
            return fail(h, DROT_ERR_CUDA, "iteration did not report completion after %lld replays", issued);
    }

    if (h->cfg.c_skip && max_iter > 0) {
        // after an odd number of passes the array holds X - rho C: restore X
        DROT_CUDA(h, cudaMemcpyAsync(h->h_status, h->d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
        DROT_CUDA(h, cudaStreamSynchronize(h->stream));
        if (h->h_status->k & 1) {
            const int rblocks = (int)std::min<long long>(8LL * h->num_sms, std::max<long long>(1, (m * n + 255) / 256));
            drot::drot_restore_plan_kernel<<<rblocks, 256, 0, h->stream>>>(X, C, m, n, ld, h->d_sc);
            DROT_CUDA(h, cudaGetLastError());
            h->prof.kernel_launches += 1;
        }
    }
    // outputs
    const int eblocks = (int)std::min<long long>(2LL * h->num_sms, std::max<long long>(1, (m + n + 255) / 256));
    drot::drot_export_duals_kernel<<<eblocks, 256, 0, h->stream>>>(h->g, h->h, h->d_sc, mu, nu, m, n, 1.0 / n,
                                                                   1.0 / m);
    DROT_CUDA(h, cudaGetLastError());
    DROT_CUDA(h, cudaMemsetAsync(&h->d_sc->nnz, 0, sizeof(unsigned long long), h->stream));
    const int nblocks = (int)std::min<long long>(8LL * h->num_sms, std::max<long long>(1, (m * n + 255) / 256));
    if (f64) drot::drot_count_nnz_f64_kernel<<<nblocks, 256, 0, h->stream>>>(X64, m, n, ld, h->d_sc);
    else drot::drot_count_nnz_kernel<<<nblocks, 256, 0, h->stream>>>(X, m, n, ld, h->d_sc);
    DROT_CUDA(h, cudaGetLastError());
    h->prof.kernel_launches += 2;
    DROT_CUDA(h, cudaMemcpyAsync(h->h_status, h->d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
    DROT_CUDA(h, cudaStreamSynchronize(h->stream));
    const Scalars fin = *h->h_status;
    iters_done = fin.k;

    h->prof.tile_k = P.K;
    h->prof.grid_ctas = P.G;
    h->prof.col_tiles = P.T;
    h->prof.graph_iters = P.graph_iters;
    h->prof.step_variant = f64 ? 5 : (use_cluster && max_iter > 0 ? 4 : (use_grid && max_iter > 0 ? 6 : P.variant));
    h->prof.stages = use_cluster && max_iter > 0 ? cp.cs : (use_grid && max_iter > 0 ? gp.G : P.S);

    drot_status out = DROT_OK;
    if (done == drot::kIterCap) out = DROT_NOT_CONVERGED;
    else if (done == drot::kNonFinite) out = DROT_ERR_NONFINITE;
    else if (done == drot::kFault) out = DROT_ERR_TIMEOUT;
    if (res) {
        res->iters = iters_done;
        res->primal_obj = fin.primal;
        res->dual_obj = fin.dual;
        res->gap = fin.gap;
        res->res_l1 = fin.res_l1;
        res->res_l2 = std::sqrt(fin.res_l2);         // the device keeps these two squared
        res->dual_res = std::sqrt(fin.dual_res_prev);
        res->nnz = (int64_t)fin.nnz;
        res->status = out;
        if (iters_done == 0) {
            res->primal_obj = res->dual_obj = res->gap = res->res_l1 = res->res_l2 = res->dual_res = NAN;
        }
    }
    return out;
}


// ------------------------------------------------------------------------------------
// Batched solve (drot_solve_batched with device buffers).

struct BatchLists {
    std::vector<int> active;
    std::vector<long long> unit0;   // nactive + 1
    std::vector<long long> wbound;  // G + 1
    std::vector<int> fin_prob, fin_local;  // FB
    // the narrow tiles' list (drot_batched_narrow_kernel); empty unless split
    bool split = false;
    std::vector<int> active_n;
    std::vector<long long> unit0_n;   // nactive_n + 1
    std::vector<long long> wbound_n;  // G + 1
};

// Wide tiles of a problem (more than 256 valid columns) come first; the others are narrow.
int wide_tiles(long long n, int K, int T) {
    if (K < 4) return 0;  // 128- and 256-column tiles are all narrow
    const long long last_w = n - (long long)(T - 1) * 128LL * K;
    return last_w <= 256 ? T - 1 : T;
}

// Tile width policy: K = 1 for n < t0, 2 for n < t1, else 4.
int batch_k(long long n, const int thr[2]) { return n < thr[0] ? 1 : (n < thr[1] ? 2 : 4); }

// Tile policies the batched autotuner times: (t0, t1) thresholds of batch_k.  The first
// (512-column tiles for every problem) is the default: in a batch of 512 problems of
// sizes 64 .. 2048 it ran an all-active iteration in 1.52 ms against 1.85 ms for the
// width-matched policy (384, 1536), because a warp keeps one row segment in flight per
// round trip and wider segments move more bytes per trip, ragged tails included.
constexpr int kBatchPolicies[][2] = {{0, 0}, {384, 384}, {384, 1024}, {384, 1536}};

// A signature of a batch's shapes (FNV-1a over m, n): the autotuned policy is reused
// while the shapes stay the same.
unsigned long long batch_signature(const drot_problem *pr, int B) {
    unsigned long long x = 1469598103934665603ull;
    auto mix = [&](unsigned long long v) {
        for (int i = 0; i < 8; ++i) {
            x ^= (v >> (8 * i)) & 0xffull;
            x *= 1099511628211ull;
        }
    };
    mix((unsigned long long)B);
    for (int b = 0; b < B; ++b) {
        mix((unsigned long long)pr[b].m);
        mix((unsigned long long)pr[b].n);
    }
    return x ? x : 1ull;
}

// Segment lists (wide tiles, narrow tiles), cost-balanced CTA ranges (SegCost) and
// finish-block groups of the active problems.
namespace {
// One list: the problems with segments in it, their first segments and the CTA ranges.
// part(P) gives the (tiles, first column count of those tiles, width sum) the list holds.
template <typename Part>
void build_list(const std::vector<drot::BatchProb> &hp, const std::vector<int> &active, int G, bool pack,
                Part part, std::vector<int> &act, std::vector<long long> &unit0, std::vector<long long> &wbound) {
    act.clear();
    unit0.assign(1, 0);
    std::vector<double> cost0(1, 0.0);
    std::vector<SegCost> costs;
    for (int b : active) {
        const drot::BatchProb &P = hp[b];
        long long tiles = 0, cols = 0;
        part(P, tiles, cols);
        if (tiles <= 0) continue;
        act.push_back(b);
        unit0.push_back(unit0.back() + tiles * P.m);
        costs.emplace_back(P.m, tiles, 128LL * P.K, cols, pack);
        cost0.push_back(cost0.back() + costs.back().total());
    }
    const int na = (int)act.size();
    const long long total = unit0[na];
    wbound.assign(G + 1, total);
    wbound[0] = 0;
    int a = 0;
    for (int g = 1; g < G; ++g) {
        const double target = cost0[na] * g / G;
        while (a + 1 < na && cost0[a + 1] <= target) ++a;
        long long u = total;
        if (na > 0) u = unit0[a] + costs[a].units_for(target - cost0[a]);
        wbound[g] = std::max(wbound[g - 1], std::min(u, total));
    }
    wbound[G] = total;
}
}  // namespace

// The narrow-tile kernel is a launch of its own, a few µs per iteration whatever its work;
// it pays only while the narrow tiles hold enough rows (packing saves ~0.2 ns per row on
// B300).  Below this many rows the wide-tile kernel takes every tile, unpacked.
constexpr long long kSplitRows = 65536;

void build_batch_lists(const std::vector<drot::BatchProb> &hp, const std::vector<int> &active, int G, int FB,
                       BatchLists &L, int narrow_mode) {
    long long narrow_rows = 0;
    for (int b : active) narrow_rows += (long long)(hp[b].T - hp[b].Tw) * hp[b].m;
    L.split = narrow_rows > 0 && (narrow_mode > 0 || (narrow_mode == 0 && narrow_rows >= kSplitRows));
    const bool split = L.split;
    // wide tiles 0 .. Tw-1 (all of them full width but a ragged last one wider than 256);
    // every tile when the narrow ones are not split off
    build_list(hp, active, G, false,
               [split](const drot::BatchProb &P, long long &tiles, long long &cols) {
                   tiles = split ? P.Tw : P.T;
                   cols = split ? std::min(P.n, (long long)P.Tw * 128LL * P.K) : P.n;
               },
               L.active, L.unit0, L.wbound);
    // narrow tiles Tw .. T-1
    build_list(hp, active, G, true,
               [split](const drot::BatchProb &P, long long &tiles, long long &cols) {
                   tiles = split ? P.T - P.Tw : 0;
                   cols = P.n - (long long)P.Tw * 128LL * P.K;
               },
               L.active_n, L.unit0_n, L.wbound_n);
    L.fin_prob.assign(FB, -1);
    L.fin_local.assign(FB, 0);
    int fb = 0;
    for (int x = 0; x < (int)active.size(); ++x) {
        const drot::BatchProb &P = hp[active[x]];
        for (int l = 0; l < P.fin_blocks && fb < FB; ++l, ++fb) {
            L.fin_prob[fb] = active[x];
            L.fin_local[fb] = l;
        }
    }
}

struct BatchDev {
    drot::BatchProb *probs;
    int *active, *nactive, *parity, *fin_prob, *fin_local, *flags;
    long long *unit0, *wbound;
    int *active_n, *nactive_n;
    long long *unit0_n, *wbound_n;
};

drot_status upload_lists(drot_handle *h, const BatchLists &L, const BatchDev &D, int FB) {
    const int na = (int)L.active.size();
    DROT_CUDA(h, cudaMemcpyAsync(D.nactive, &na, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    if (na > 0)
        DROT_CUDA(h, cudaMemcpyAsync(D.active, L.active.data(), sizeof(int) * na, cudaMemcpyHostToDevice, h->stream));
    DROT_CUDA(h, cudaMemcpyAsync(D.unit0, L.unit0.data(), sizeof(long long) * (na + 1), cudaMemcpyHostToDevice,
                                 h->stream));
    DROT_CUDA(h, cudaMemcpyAsync(D.wbound, L.wbound.data(), sizeof(long long) * L.wbound.size(),
                                 cudaMemcpyHostToDevice, h->stream));
    DROT_CUDA(h, cudaMemcpyAsync(D.fin_prob, L.fin_prob.data(), sizeof(int) * FB, cudaMemcpyHostToDevice, h->stream));
    DROT_CUDA(h, cudaMemcpyAsync(D.fin_local, L.fin_local.data(), sizeof(int) * FB, cudaMemcpyHostToDevice,
                                 h->stream));
    const int nn = (int)L.active_n.size();
    DROT_CUDA(h, cudaMemcpyAsync(D.nactive_n, &nn, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    if (nn > 0)
        DROT_CUDA(h, cudaMemcpyAsync(D.active_n, L.active_n.data(), sizeof(int) * nn, cudaMemcpyHostToDevice,
                                     h->stream));
    DROT_CUDA(h, cudaMemcpyAsync(D.unit0_n, L.unit0_n.data(), sizeof(long long) * (nn + 1), cudaMemcpyHostToDevice,
                                 h->stream));
    DROT_CUDA(h, cudaMemcpyAsync(D.wbound_n, L.wbound_n.data(), sizeof(long long) * L.wbound_n.size(),
                                 cudaMemcpyHostToDevice, h->stream));
    // pageable sources: the copies return once the host data has been staged, but keep
    // the stream ordered with the next launch anyway
    return DROT_OK;
}

drot_status solve_batched_device(drot_handle *h, int B, const drot_problem *pr, double tol, long long max_iter,
                                 int warm, drot_result *res) {
    const int rule = (h->cfg.stop_rule & 7) ? (h->cfg.stop_rule & 7) : (DROT_STOP_GAP | DROT_STOP_RES_L1);
    int thr[2] = {kBatchPolicies[0][0], kBatchPolicies[0][1]};
    const unsigned long long sig = batch_signature(pr, B);
    // an explicit tile_k gives every problem that tile width (no tuning)
    const bool forced_k = h->cfg.tile_k == 1 || h->cfg.tile_k == 2 || h->cfg.tile_k == 4;
    const bool tuned = forced_k || (h->cfg.autotune && h->batch_tuned_sig == sig);
    if (forced_k) {
        const long long big = 1LL << 30;
        thr[0] = h->cfg.tile_k == 1 ? (int)big : 0;
        thr[1] = h->cfg.tile_k <= 2 ? (int)big : 0;
    } else if (tuned) {
        thr[0] = h->batch_k_thresholds[0];
        thr[1] = h->batch_k_thresholds[1];
    }
    // layout: scalars[B] | per problem: g a u (m), h b v (n), acc[2], finpart | tables
    std::vector<drot::BatchProb> hp(B);
    std::vector<size_t> off(B);
    size_t bytes = align_up(sizeof(Scalars) * B, 256);
    int FB = 0;
    for (int b = 0; b < B; ++b) {
        const long long m = pr[b].m, n = pr[b].n;
        const int fb = (int)std::min<long long>(
            64, std::max<long long>(1, (m + n + drot::kBatchFinishElems - 1) / drot::kBatchFinishElems));
        hp[b].fin_blocks = fb;
        FB += fb;
        off[b] = bytes;
        bytes += align_up(sizeof(double) * m, 256) * 3 + align_up(sizeof(double) * n, 256) * 3 +
                 align_up(sizeof(double) * drot::kAccSlots * drot::kAccStride, 256) +
                 align_up(sizeof(double) * drot::kFinishAcc * fb, 256);
    }
    const size_t vec_bytes = bytes - align_up(sizeof(Scalars) * B, 256);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, drot::drot_batched_step_kernel<true>, drot::kThreads, 0);
    const int G = std::max(1, occ) * h->num_sms;
    const size_t tables = align_up(sizeof(drot::BatchProb) * B, 256) + align_up(sizeof(int) * B, 256) * 4 +
                          align_up(sizeof(long long) * (B + 1), 256) * 2 + align_up(sizeof(long long) * (G + 1), 256) * 2 +
                          align_up(sizeof(int) * FB, 256) * 2 + 256 * 2;
    drot_status st = arena_reserve(h, h->batch, bytes + tables);
    if (st != DROT_OK) return st;
    if (h->h_bstat_cap < (size_t)B) {
        if (h->h_bstat) cudaFreeHost(h->h_bstat);
        h->h_bstat = nullptr;
        h->h_bstat_cap = 0;
        DROT_CUDA(h, cudaMallocHost(&h->h_bstat, sizeof(Scalars) * B));
        h->h_bstat_cap = B;
    }
    char *base = static_cast<char *>(h->batch.ptr);
    Scalars *d_sc = reinterpret_cast<Scalars *>(base);
    for (int b = 0; b < B; ++b) {
        char *cur = base + off[b];
        const long long m = pr[b].m, n = pr[b].n;
        drot::BatchProb &P = hp[b];
        P.C = pr[b].C;
        P.X = pr[b].X;
        P.p = pr[b].p;
        P.q = pr[b].q;
        P.mu = pr[b].mu;
        P.nu = pr[b].nu;
        P.g = carve<double>(cur, m);
        P.a = carve<double>(cur, m);
        P.u = carve<double>(cur, m);
        P.h = carve<double>(cur, n);
        P.b = carve<double>(cur, n);
        P.v = carve<double>(cur, n);
        P.acc = carve<double>(cur, (size_t)drot::kAccSlots * drot::kAccStride);
        P.finpart = carve<double>(cur, (size_t)drot::kFinishAcc * P.fin_blocks);
        P.sc = d_sc + b;
        P.m = m;
        P.n = n;
        P.ld = pr[b].ld;
        P.inv_n = 1.0 / (double)n;
        P.inv_m = 1.0 / (double)m;
        P.K = batch_k(n, thr);
        P.T = (int)((n + 128LL * P.K - 1) / (128LL * P.K));
        P.Tw = wide_tiles(n, P.K, P.T);
    }
    char *cur = base + bytes;
    BatchDev D{};
    D.probs = carve<drot::BatchProb>(cur, B);
    D.active = carve<int>(cur, B);
    D.flags = carve<int>(cur, B);
    D.fin_prob = carve<int>(cur, FB);
    D.fin_local = carve<int>(cur, FB);
    D.unit0 = carve<long long>(cur, B + 1);
    D.wbound = carve<long long>(cur, G + 1);
    D.nactive = carve<int>(cur, 1);
    D.parity = carve<int>(cur, 1);
    D.active_n = carve<int>(cur, B);
    D.unit0_n = carve<long long>(cur, B + 1);
    D.wbound_n = carve<long long>(cur, G + 1);
    D.nactive_n = carve<int>(cur, 1);

    // scalar state of every problem, then the marginal checks
    std::vector<Scalars> hs(B);
    for (int b = 0; b < B; ++b) {
        std::memset(&hs[b], 0, sizeof(Scalars));
        hs[b].rho = pr[b].rho > 0.0 ? pr[b].rho : h->cfg.rho0 / (double)(pr[b].m + pr[b].n);
        hs[b].inv_rho = 1.0 / hs[b].rho;
        hs[b].tol = tol;
        hs[b].max_iter = max_iter;
        hs[b].stop_rule = rule;
        hs[b].done = drot::kRunning;
    }
    DROT_CUDA(h, cudaMemcpyAsync(d_sc, hs.data(), sizeof(Scalars) * B, cudaMemcpyHostToDevice, h->stream));
    DROT_CUDA(h, cudaMemsetAsync(base + align_up(sizeof(Scalars) * B, 256), 0, vec_bytes, h->stream));
    DROT_CUDA(h, cudaMemsetAsync(D.parity, 0, sizeof(int), h->stream));
    DROT_CUDA(h, cudaMemcpyAsync(D.probs, hp.data(), sizeof(drot::BatchProb) * B, cudaMemcpyHostToDevice, h->stream));
    drot::drot_batched_vector_sums_kernel<<<B, 1024, 0, h->stream>>>(D.probs, warm);
    DROT_CUDA(h, cudaGetLastError());
    DROT_CUDA(h, cudaMemcpyAsync(h->h_bstat, d_sc, sizeof(Scalars) * B, cudaMemcpyDeviceToHost, h->stream));
    DROT_CUDA(h, cudaStreamSynchronize(h->stream));
    h->prof.kernel_launches += 1;
    std::vector<drot_status> status(B, DROT_OK);
    std::vector<int> valid;
    for (int b = 0; b < B; ++b) {
        const Scalars &c = h->h_bstat[b];
        if (c.nonfinite_input & 3) status[b] = DROT_ERR_MARGINALS;
        else if (c.nonfinite_input & 4) status[b] = DROT_ERR_INVALID_ARG;
        else if (!(std::fabs(c.sum_p - c.sum_q) <= 1e-9 * std::max(1.0, std::fabs(c.sum_p))))
            status[b] = DROT_ERR_MARGINALS;
        else valid.push_back(b);
    }
    const int nvalid = (int)valid.size();

    drot::BatchArgs A{};
    A.probs = D.probs;
    A.active = D.active;
    A.unit0 = D.unit0;
    A.wbound = D.wbound;
    A.fin_prob = D.fin_prob;
    A.fin_local = D.fin_local;
    A.nactive = D.nactive;
    A.parity = D.parity;
    A.active_n = D.active_n;
    A.unit0_n = D.unit0_n;
    A.wbound_n = D.wbound_n;
    A.nactive_n = D.nactive_n;
    A.warm = warm;
    A.serp = h->cfg.serpentine >= 0 ? 1 : 0;
    A.odd = 0;

    // Tile policy autotuning (autotune = 1, cold starts, a batch shape not tuned yet):
    // time the fused step of this batch under every candidate policy, one warm-up and
    // three launches each, before X_0 is written (the launches run on the caller's X,
    // which the cold start overwrites next), then zero the totals they touched.
    if (h->cfg.autotune && !warm && nvalid > 0 && !tuned) {
        cudaEvent_t e0, e1;
        DROT_CUDA(h, cudaEventCreate(&e0));
        DROT_CUDA(h, cudaEventCreate(&e1));
        float best = 1e30f;
        int best_p = 0;
        drot_status tst = DROT_OK;
        const int npol = (int)(sizeof(kBatchPolicies) / sizeof(kBatchPolicies[0]));
        for (int pi = 0; pi < npol && tst == DROT_OK; ++pi) {
            for (int b = 0; b < B; ++b) {
                hp[b].K = batch_k(hp[b].n, kBatchPolicies[pi]);
                hp[b].T = (int)((hp[b].n + 128LL * hp[b].K - 1) / (128LL * hp[b].K));
                hp[b].Tw = wide_tiles(hp[b].n, hp[b].K, hp[b].T);
            }
            cudaError_t e = cudaMemcpyAsync(D.probs, hp.data(), sizeof(drot::BatchProb) * B, cudaMemcpyHostToDevice,
                                            h->stream);
            if (e != cudaSuccess) {
                tst = fail(h, DROT_ERR_CUDA, "tuning upload failed: %s", cudaGetErrorString(e));
                break;
            }
            BatchLists TL;
            build_batch_lists(hp, valid, G, FB, TL, h->cfg.batch_narrow);
            tst = upload_lists(h, TL, D, FB);
            if (tst != DROT_OK) break;
            // alternating directions, as the solve runs them
            drot::BatchArgs At = A;
            At.odd = 1;
            drot::drot_batched_step_kernel<true><<<G, drot::kThreads, 0, h->stream>>>(At);
            if (TL.split) drot::drot_batched_narrow_kernel<true><<<G, drot::kThreads, 0, h->stream>>>(At);
            e = cudaEventRecord(e0, h->stream);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
                At.odd = r & 1;
                drot::drot_batched_step_kernel<true><<<G, drot::kThreads, 0, h->stream>>>(At);
                if (TL.split) drot::drot_batched_narrow_kernel<true><<<G, drot::kThreads, 0, h->stream>>>(At);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                tst = fail(h, DROT_ERR_CUDA, "tuning launch failed: %s", cudaGetErrorString(e));
                break;
            }
            h->prof.kernel_launches += TL.split ? 8 : 4;
            if (ms < best) {
                best = ms;
                best_p = pi;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (tst != DROT_OK) return tst;
        thr[0] = kBatchPolicies[best_p][0];
        thr[1] = kBatchPolicies[best_p][1];
        h->batch_k_thresholds[0] = thr[0];
        h->batch_k_thresholds[1] = thr[1];
        h->batch_tuned_sig = sig;
        for (int b = 0; b < B; ++b) {
            hp[b].K = batch_k(hp[b].n, thr);
            hp[b].T = (int)((hp[b].n + 128LL * hp[b].K - 1) / (128LL * hp[b].K));
            hp[b].Tw = wide_tiles(hp[b].n, hp[b].K, hp[b].T);
        }
        DROT_CUDA(h, cudaMemcpyAsync(D.probs, hp.data(), sizeof(drot::BatchProb) * B, cudaMemcpyHostToDevice,
                                     h->stream));
        DROT_CUDA(h, cudaMemsetAsync(base + align_up(sizeof(Scalars) * B, 256), 0, vec_bytes, h->stream));
    }

    // cold start X_0 = p q^T, sums of X_0, a_0 / b_0 / alpha_0
    std::vector<int> flags(B, 0);
    for (int b : valid) flags[b] = warm ? 0 : 1;
    DROT_CUDA(h, cudaMemcpyAsync(D.flags, flags.data(), sizeof(int) * B, cudaMemcpyHostToDevice, h->stream));
    if (!warm && nvalid > 0) {
        drot::drot_batched_init_plan_kernel<<<dim3(64, B), 256, 0, h->stream>>>(D.probs, D.flags);
        DROT_CUDA(h, cudaGetLastError());
        h->prof.kernel_launches += 1;
    }
    BatchLists L;
    build_batch_lists(hp, valid, G, FB, L, h->cfg.batch_narrow);
    st = upload_lists(h, L, D, FB);
    if (st != DROT_OK) return st;
    drot::drot_batched_step_kernel<false><<<G, drot::kThreads, 0, h->stream>>>(A);
    DROT_CUDA(h, cudaGetLastError());
    if (L.split) {
        drot::drot_batched_narrow_kernel<false><<<G, drot::kThreads, 0, h->stream>>>(A);
        DROT_CUDA(h, cudaGetLastError());
        h->prof.kernel_launches += 1;
    }
    drot::drot_batched_init_state_kernel<<<FB, drot::kFinishThreads, 0, h->stream>>>(A);
    DROT_CUDA(h, cudaGetLastError());
    h->prof.kernel_launches += 2;

    // Graph replays of gi iterations over the active lists.  gi follows the work still
    // active (about 32 ms per replay, a power of 4 up to 256), so the replays stay long
    // enough to hide the host round trip as problems converge; one graph per (gi, whether
    // the narrow-tile kernel runs).
    std::vector<std::pair<int, cudaGraphExec_t>> graphs;
    auto release = [&]() {
        for (auto &g : graphs) cudaGraphExecDestroy(g.second);
        graphs.clear();
    };
    auto pick_gi = [&](const std::vector<int> &act) {
        if (h->cfg.graph_iters > 0) return h->cfg.graph_iters;
        // ~32 ms of the work still active per replay: the host reads every problem's flag
        // between replays, and on the 512-problem workload shorter replays (4 ms: one
        // iteration while all are active) cost 0.7 % of the solve in those round trips
        double bytes = 0.0;
        for (int b : act) bytes += 12.0 * (double)pr[b].m * (double)pr[b].n;
        const double want = 32.0e-3 / (bytes / 6.0e12 + 12.0e-6);
        int g = 1;
        while (g < 256 && 4.0 * g <= want) g *= 4;
        return g;
    };
    auto graph_for = [&](int g, bool split, cudaGraphExec_t *out) -> drot_status {
        const int key = 2 * g + (split ? 1 : 0);
        for (auto &e : graphs)
            if (e.first == key) {
                *out = e.second;
                return DROT_OK;
            }
        cudaGraph_t graph = nullptr;
        DROT_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t err = cudaSuccess;
        for (int it = 0; it < g && err == cudaSuccess; ++it) {
            drot::BatchArgs Ai = A;
            Ai.odd = it & 1;  // added to the parity word the host keeps between replays
            Ai.narrow_next = split ? 1 : 0;
            err = launch_k(drot::drot_batched_step_kernel<true>, dim3(G), dim3(drot::kThreads), 0, h->stream, true, Ai);
            if (err == cudaSuccess && split)
                err = launch_k(drot::drot_batched_narrow_kernel<true>, dim3(G), dim3(drot::kThreads), 0, h->stream,
                               true, Ai);
            if (err == cudaSuccess)
                err = launch_k(drot::drot_batched_finish_kernel, dim3(FB), dim3(drot::kBatchFinishThreads), 0, h->stream,
                               true, A);
        }
        cudaError_t endc = cudaStreamEndCapture(h->stream, &graph);
        if (err != cudaSuccess || endc != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(h, DROT_ERR_CUDA, "batched graph capture failed: %s",
                        cudaGetErrorString(err != cudaSuccess ? err : endc));
        }
        cudaGraphExec_t exec = nullptr;
        cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess)
            return fail(h, DROT_ERR_CUDA, "batched graph instantiate failed: %s", cudaGetErrorString(ie));
        graphs.emplace_back(key, exec);
        *out = exec;
        return DROT_OK;
    };
    if (max_iter > 0 && nvalid > 0) {
        std::vector<int> active = valid;
        const long long max_replays = max_iter + 2;  // every replay advances every active problem
        long long iters_run = 0;  // iterations every active problem has run so far
        int dev_parity = 0;       // the device's parity word
        for (long long r = 0; r < max_replays && !active.empty(); ++r) {
            const int gi = pick_gi(active);
            cudaGraphExec_t exec = nullptr;
            st = graph_for(gi, L.split, &exec);
            if (st != DROT_OK) {
                release();
                return st;
            }
            cudaError_t e = cudaSuccess;
            const int want = (int)(iters_run & 1);
            if (want != dev_parity) {  // after a replay of odd length (pageable source: staged before return)
                e = cudaMemcpyAsync(D.parity, &want, sizeof(int), cudaMemcpyHostToDevice, h->stream);
                dev_parity = want;
            }
            if (e == cudaSuccess) e = cudaGraphLaunch(exec, h->stream);
            iters_run += gi;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h->h_bstat, d_sc, sizeof(Scalars) * B, cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) {
                release();
                return fail(h, DROT_ERR_CUDA, "batched replay failed: %s", cudaGetErrorString(e));
            }
            h->prof.graph_replays += 1;
            h->prof.kernel_launches += (L.split ? 3LL : 2LL) * gi;
            std::vector<int> still;
            for (int b : active)
                if (h->h_bstat[b].done == drot::kRunning) still.push_back(b);
            if (still.size() != active.size() && !still.empty()) {
                build_batch_lists(hp, still, G, FB, L, h->cfg.batch_narrow);
                st = upload_lists(h, L, D, FB);
                if (st != DROT_OK) {
                    release();
                    return st;
                }
            }
            active.swap(still);
        }
        release();
        if (!active.empty())
            return fail(h, DROT_ERR_CUDA, "%zu problems did not report completion", active.size());
    }

    // duals and nnz
    if (nvalid > 0) {
        for (int b : valid) flags[b] = 1;
        DROT_CUDA(h, cudaMemcpyAsync(D.flags, flags.data(), sizeof(int) * B, cudaMemcpyHostToDevice, h->stream));
        drot::drot_batched_export_kernel<<<dim3(32, B), 256, 0, h->stream>>>(D.probs, D.flags);
        DROT_CUDA(h, cudaGetLastError());
        h->prof.kernel_launches += 1;
    }
    DROT_CUDA(h, cudaMemcpyAsync(h->h_bstat, d_sc, sizeof(Scalars) * B, cudaMemcpyDeviceToHost, h->stream));
    DROT_CUDA(h, cudaStreamSynchronize(h->stream));
    drot_status first_bad = DROT_OK;
    for (int b = 0; b < B; ++b) {
        const Scalars &c = h->h_bstat[b];
        if (status[b] == DROT_OK) {
            if (max_iter == 0 || c.done == drot::kIterCap) status[b] = DROT_NOT_CONVERGED;
            else if (c.done == drot::kNonFinite) status[b] = DROT_ERR_NONFINITE;
            else if (c.done == drot::kFault) status[b] = DROT_ERR_TIMEOUT;
        }
        if (status[b] != DROT_OK && first_bad == DROT_OK) first_bad = status[b];
        if (res) {
            drot_result &R = res[b];
            R.iters = status[b] == DROT_OK || status[b] == DROT_NOT_CONVERGED || status[b] == DROT_ERR_NONFINITE
                          ? c.k : 0;
            R.primal_obj = c.primal;
            R.dual_obj = c.dual;
            R.gap = c.gap;
            R.res_l1 = c.res_l1;
            R.res_l2 = std::sqrt(c.res_l2);
            R.dual_res = std::sqrt(c.dual_res_prev);
            R.nnz = (int64_t)c.nnz;
            R.status = status[b];
            R.seconds = 0.0;
            if (R.iters == 0) R.primal_obj = R.dual_obj = R.gap = R.res_l1 = R.res_l2 = R.dual_res = NAN;
        }
    }
    return first_bad;
}

drot_status check_args(drot_handle *h, long long m, long long n, const void *C, long long ld, const double *p,
                       const double *q, double tol, long long max_iter, void *X, double *mu, double *nu,
                       size_t elem = sizeof(float)) {
    if (!h) return DROT_ERR_INVALID_ARG;
    if (m < 1 || n < 1) return fail(h, DROT_ERR_INVALID_ARG, "m = %lld and n = %lld must be >= 1", m, n);
    const long long vec = 16 / (long long)elem;  // rows start on 16-byte boundaries
    if (ld < n || ld % vec != 0)
        return fail(h, DROT_ERR_INVALID_ARG, "ld = %lld must be >= n and a multiple of %lld", ld, vec);
    if (!C || !p || !q || !X || !mu || !nu) return fail(h, DROT_ERR_INVALID_ARG, "a buffer pointer is NULL");
    if ((reinterpret_cast<uintptr_t>(C) | reinterpret_cast<uintptr_t>(X)) & 15)
        return fail(h, DROT_ERR_INVALID_ARG, "C and X must be 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(q) | reinterpret_cast<uintptr_t>(mu) |
         reinterpret_cast<uintptr_t>(nu)) & 7)
        return fail(h, DROT_ERR_INVALID_ARG, "p, q, mu, nu must be 8-byte aligned");
    if (max_iter < 0) return fail(h, DROT_ERR_INVALID_ARG, "max_iter = %lld must be >= 0", max_iter);
    if (std::isnan(tol)) return fail(h, DROT_ERR_INVALID_ARG, "tol is NaN");
    if (m > (1LL << 40) / n) return fail(h, DROT_ERR_INVALID_ARG, "m * n too large");
    return DROT_OK;
}

// drot_solve (T = float) and drot_solve_f64 (T = double): argument checks, then the
// device solve, directly on device buffers or through a staging workspace for host buffers.
template <typename T>
drot_status solve_entry(drot_handle *h, int64_t m, int64_t n, const T *C, int64_t ld, const double *p,
                        const double *q, double rho, double tol, int64_t max_iter, T *X, double *mu, double *nu,
                        int warm, drot_result *res) {
    constexpr bool f64 = sizeof(T) == sizeof(double);
    const auto t0 = std::chrono::steady_clock::now();
    drot_status st = check_args(h, m, n, C, ld, p, q, tol, max_iter, X, mu, nu, sizeof(T));
    if (st != DROT_OK) return st;
    h->last_error.clear();
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, DROT_ERR_CUDA, "cudaSetDevice failed");
    if (!(rho > 0.0)) rho = h->cfg.rho0 / (double)(m + n);
    if (!std::isfinite(rho)) return fail(h, DROT_ERR_INVALID_ARG, "rho is not finite");

    const void *ptrs[7] = {C, p, q, X, mu, nu, nullptr};
    int ndev = 0;
    for (int i = 0; i < 6; ++i) ndev += is_device_ptr(ptrs[i], h->device) ? 1 : 0;
    if (ndev != 0 && ndev != 6)
        return fail(h, DROT_ERR_INVALID_ARG, "buffers mix device and host memory (%d of 6 on the device)", ndev);

    if (ndev == 6) {
        st = solve_device(h, m, n, C, ld, p, q, rho, tol, max_iter, X, mu, nu, warm, res, f64);
    } else {
        // host buffers: stage through a device workspace owned by the handle
        const size_t mat = align_up(sizeof(T) * (size_t)m * ld, 256);
        const size_t vm = align_up(sizeof(double) * m, 256), vn = align_up(sizeof(double) * n, 256);
        st = arena_reserve(h, h->staging, 2 * mat + 2 * vm + 2 * vn);
        if (st != DROT_OK) return st;
        char *cur = static_cast<char *>(h->staging.ptr);
        T *dC = carve<T>(cur, (size_t)m * ld);
        T *dX = carve<T>(cur, (size_t)m * ld);
        double *dp = carve<double>(cur, m), *dmu = carve<double>(cur, m);
        double *dq = carve<double>(cur, n), *dnu = carve<double>(cur, n);
        const size_t mb = sizeof(T) * (size_t)m * ld;
        DROT_CUDA(h, cudaMemcpyAsync(dC, C, mb, cudaMemcpyHostToDevice, h->stream));
        DROT_CUDA(h, cudaMemcpyAsync(dp, p, sizeof(double) * m, cudaMemcpyHostToDevice, h->stream));
        DROT_CUDA(h, cudaMemcpyAsync(dq, q, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
        if (warm) {
            DROT_CUDA(h, cudaMemcpyAsync(dX, X, mb, cudaMemcpyHostToDevice, h->stream));
            DROT_CUDA(h, cudaMemcpyAsync(dmu, mu, sizeof(double) * m, cudaMemcpyHostToDevice, h->stream));
            DROT_CUDA(h, cudaMemcpyAsync(dnu, nu, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
        }
        st = solve_device(h, m, n, dC, ld, dp, dq, rho, tol, max_iter, dX, dmu, dnu, warm, res, f64);
        if (st == DROT_OK || st == DROT_NOT_CONVERGED || st == DROT_ERR_NONFINITE) {
            // columns 0..n-1 of every row only: the caller's row padding is never written (a cold
            // start uploads no X, so the workspace's padding holds nothing of the caller's)
            if (ld == n) {
                DROT_CUDA(h, cudaMemcpyAsync(X, dX, mb, cudaMemcpyDeviceToHost, h->stream));
            } else {
                DROT_CUDA(h, cudaMemcpy2DAsync(X, sizeof(T) * ld, dX, sizeof(T) * ld, sizeof(T) * n, m,
                                               cudaMemcpyDeviceToHost, h->stream));
            }
            DROT_CUDA(h, cudaMemcpyAsync(mu, dmu, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream));
            DROT_CUDA(h, cudaMemcpyAsync(nu, dnu, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
            DROT_CUDA(h, cudaStreamSynchronize(h->stream));
        }
    }
    if (res) res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

}  // namespace

extern "C" {

void drot_config_default(drot_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->device = 0;
    cfg->stream = nullptr;
    cfg->stop_rule = DROT_STOP_GAP | DROT_STOP_RES_L1;
    cfg->rho0 = 2.0;
    cfg->graph_iters = 0;
    cfg->tile_k = 0;
    cfg->grid_ctas = 0;
    cfg->profile = 0;
    cfg->step_variant = 0;
    cfg->deterministic = 0;
    cfg->autotune = 0;
    cfg->persistent = 0;
    cfg->c_skip = 0;
    cfg->cluster = 0;
    cfg->batch_narrow = 0;
}

drot_status drot_create(drot_handle **out, const drot_config *cfg) {
    if (!out) return DROT_ERR_INVALID_ARG;
    drot_config c;
    if (cfg) c = *cfg;
    else drot_config_default(&c);
    if (!(c.rho0 > 0.0)) c.rho0 = 2.0;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
        cudaGetLastError();
        return DROT_ERR_CUDA;
    }
    if (c.device < 0 || c.device >= ndev) return DROT_ERR_INVALID_ARG;
    if (c.c_skip) c.persistent = 0;
    drot_handle *h = new (std::nothrow) drot_handle();
    if (!h) return DROT_ERR_OOM;
    h->cfg = c;
    h->device = c.device;
    auto bail = [&](drot_status s) {
        drot_destroy(h);
        return s;
    };
    if (cudaSetDevice(h->device) != cudaSuccess) return bail(DROT_ERR_CUDA);
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (set_kernel_attributes() != cudaSuccess) return bail(DROT_ERR_CUDA);
    if (fill_occupancy(h) != cudaSuccess) return bail(DROT_ERR_CUDA);
    if (c.stream) {
        h->stream = static_cast<cudaStream_t>(c.stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(DROT_ERR_CUDA);
        h->own_stream = true;
    }
    if (cudaMalloc(&h->d_sc, sizeof(Scalars)) != cudaSuccess) return bail(DROT_ERR_OOM);
    if (cudaMallocHost(&h->h_sc, sizeof(Scalars)) != cudaSuccess) return bail(DROT_ERR_OOM);
    if (cudaMallocHost(&h->h_status, 2 * sizeof(Scalars)) != cudaSuccess) return bail(DROT_ERR_OOM);
    std::memset(h->h_status, 0, 2 * sizeof(Scalars));
    *out = h;
    return DROT_OK;
}

drot_status drot_destroy(drot_handle *h) {
    if (!h) return DROT_OK;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    destroy_graphs(h);
    if (h->work.ptr) cudaFree(h->work.ptr);
    if (h->tune_x.ptr) cudaFree(h->tune_x.ptr);
    if (h->batch.ptr) cudaFree(h->batch.ptr);
    if (h->h_bstat) cudaFreeHost(h->h_bstat);
    if (h->staging.ptr) cudaFree(h->staging.ptr);
    if (h->d_sc) cudaFree(h->d_sc);
    if (h->h_sc) cudaFreeHost(h->h_sc);
    if (h->h_status) cudaFreeHost(h->h_status);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return DROT_OK;
}

drot_status drot_solve(drot_handle *h, int64_t m, int64_t n, const float *C, int64_t ld, const double *p,
                       const double *q, double rho, double tol, int64_t max_iter, float *X, double *mu, double *nu,
                       int warm, drot_result *res) {
    return solve_entry<float>(h, m, n, C, ld, p, q, rho, tol, max_iter, X, mu, nu, warm, res);
}

drot_status drot_solve_f64(drot_handle *h, int64_t m, int64_t n, const double *C, int64_t ld, const double *p,
                           const double *q, double rho, double tol, int64_t max_iter, double *X, double *mu,
                           double *nu, int warm, drot_result *res) {
    return solve_entry<double>(h, m, n, C, ld, p, q, rho, tol, max_iter, X, mu, nu, warm, res);
}

drot_status drot_solve_batched(drot_handle *h, int32_t B, const drot_problem *probs, double tol, int64_t max_iter,
                               int warm, drot_result *res) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!h || B < 0 || (B > 0 && !probs)) return DROT_ERR_INVALID_ARG;
    if (B == 0) return DROT_OK;
    h->last_error.clear();
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, DROT_ERR_CUDA, "cudaSetDevice failed");
    bool all_device = true;
    for (int32_t b = 0; b < B; ++b) {
        const drot_problem &P = probs[b];
        drot_status st = check_args(h, P.m, P.n, P.C, P.ld, P.p, P.q, tol, max_iter, P.X, P.mu, P.nu);
        if (st != DROT_OK) return fail(h, st, "problem %d: %s", (int)b, h->last_error.c_str());
        const void *ptrs[6] = {P.C, P.p, P.q, P.X, P.mu, P.nu};
        for (const void *ptr : ptrs) all_device = all_device && is_device_ptr(ptr, h->device);
    }
    drot_status first_bad = DROT_OK;
    if (all_device) {
        first_bad = solve_batched_device(h, B, probs, tol, max_iter, warm, res);
    } else {
        // host buffers: one problem at a time through the staging path of drot_solve
        for (int32_t b = 0; b < B; ++b) {
            const drot_problem &P = probs[b];
            drot_result r{};
            drot_status st = drot_solve(h, P.m, P.n, P.C, P.ld, P.p, P.q, P.rho, tol, max_iter, P.X, P.mu, P.nu,
                                        warm, res ? &r : nullptr);
            if (res) {
                r.status = st;
                res[b] = r;
            }
            if (st != DROT_OK && first_bad == DROT_OK) first_bad = st;
            if (st != DROT_OK && st != DROT_NOT_CONVERGED && st != DROT_ERR_NONFINITE) return st;
        }
    }
    if (res && all_device) {
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int32_t b = 0; b < B; ++b) res[b].seconds = secs;
    }
    return first_bad;
}

drot_status drot_get_profile(drot_handle *h, drot_profile *out) {
    if (!h || !out) return DROT_ERR_INVALID_ARG;
    *out = h->prof;
    return DROT_OK;
}

drot_status drot_reset_profile(drot_handle *h) {
    if (!h) return DROT_ERR_INVALID_ARG;
    const drot_profile keep = h->prof;
    h->prof = drot_profile{};
    h->prof.tile_k = keep.tile_k;
    h->prof.step_variant = keep.step_variant;
    h->prof.stages = keep.stages;
    h->prof.grid_ctas = keep.grid_ctas;
    h->prof.col_tiles = keep.col_tiles;
    h->prof.graph_iters = keep.graph_iters;
    return DROT_OK;
}

const char *drot_status_string(drot_status s) {
    switch (s) {
        case DROT_OK: return "converged";
        case DROT_ERR_INVALID_ARG: return "invalid argument";
        case DROT_ERR_MARGINALS: return "invalid marginals";
        case DROT_ERR_OOM: return "out of memory";
        case DROT_ERR_CUDA: return "CUDA error";
        case DROT_NOT_CONVERGED: return "iteration cap reached";
        case DROT_ERR_TIMEOUT: return "device wait timed out";
        case DROT_ERR_NONFINITE: return "non-finite value in the iteration";
        case DROT_ERR_TOO_LARGE: return "problem too large for the static workspace of drot_solve_static";
    }
    return "unknown status";
}

const char *drot_last_error(drot_handle *h) { return h ? h->last_error.c_str() : ""; }

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Allocation-free entry point (drot_solve_static).  For callers that may not allocate
// device memory when they solve; see include/drot.h.  The workspace is the file-scope
// array below; host code reaches it only through the address cudaGetSymbolAddress
// returns for the current device (the array's name is not a device address on the host).

static __device__ __align__(256) unsigned char drot_static_scratch[DROT_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kStaticMaxDevices = 64;
constexpr int kStaticMaxCtas = 512;
constexpr int kStaticMaxTiles = 8192;

// Host state of one device: the lock that serialises the calls on that device (they share
// its workspace and these launch tables) and the workspace's device address.
struct StaticDeviceState {
    std::mutex call_mu;
    void *addr = nullptr;
    long long wbound[kStaticMaxCtas + 1];
    int slot_base[kStaticMaxCtas];
    int tile_slot[kStaticMaxTiles + 1];
};
std::mutex g_static_mu;  // guards the address lookups
StaticDeviceState g_static_dev[kStaticMaxDevices];

// Device address of the static workspace on `dev` (looked up once per device, with `dev`
// current: the caller's current device).
cudaError_t static_workspace(int dev, void **out) {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_dev[dev].addr) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, drot_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_dev[dev].addr = ptr;
    }
    *out = g_static_dev[dev].addr;
    return cudaSuccess;
}

}  // namespace

extern "C" drot_status drot_solve_static(int64_t m, int64_t n, const float *C, int64_t ld, const double *p,
                                         const double *q, double rho, double tol, int64_t max_iter, float *X,
                                         double *mu, double *nu, int warm, void *stream_ptr, drot_result *res) {
    const auto t_start = std::chrono::steady_clock::now();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    if (m < 1 || n < 1 || ld < n || ld % 4 != 0 || max_iter < 0 || std::isnan(tol)) return DROT_ERR_INVALID_ARG;
    if (!C || !p || !q || !X || !mu || !nu) return DROT_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(C) | reinterpret_cast<uintptr_t>(X)) & 15) return DROT_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(q) | reinterpret_cast<uintptr_t>(mu) |
         reinterpret_cast<uintptr_t>(nu)) & 7)
        return DROT_ERR_INVALID_ARG;
    if (m > (1LL << 40) / n) return DROT_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return DROT_ERR_CUDA;
    const void *ptrs[6] = {C, p, q, X, mu, nu};
    for (const void *ptr : ptrs)
        if (!is_device_ptr(ptr, dev)) return DROT_ERR_INVALID_ARG;
    if (!(rho > 0.0)) rho = 2.0 / (double)(m + n);
    if (!std::isfinite(rho)) return DROT_ERR_INVALID_ARG;
    int num_sms = 148;
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);

    // launch plan: register-fed fused step, tables in fixed-size host arrays
    const int K = n >= 1536 ? 4 : (n >= 384 ? 2 : 1);
    const int TW = 128 * K;
    const long long T = (n + TW - 1) / TW;
    if (T > kStaticMaxTiles) return DROT_ERR_TOO_LARGE;
    const long long units = T * m;
    const int G = (int)std::min<long long>(
        std::min<long long>(2LL * num_sms, kStaticMaxCtas),
        std::max<long long>(1, (units + drot::kWarps - 1) / drot::kWarps));
    StaticDeviceState &ds = g_static_dev[dev];
    std::lock_guard<std::mutex> call_lock(ds.call_mu);
    long long *wbound = ds.wbound;
    int *slot_base = ds.slot_base;
    int *tile_slot = ds.tile_slot;
    const SegCost cost(m, T, TW, n);
    const double total_cost = cost.total();
    wbound[0] = 0;
    for (int g = 1; g < G; ++g) wbound[g] = std::max(wbound[g - 1], cost.units_for(total_cost * g / G));
    wbound[G] = units;
    int slots = 0;
    for (long long t = 0; t <= T; ++t) tile_slot[t] = -1;
    for (int g = 0; g < G; ++g) {
        slot_base[g] = slots;
        if (wbound[g + 1] <= wbound[g]) continue;
        for (long long t = wbound[g] / m; t <= (wbound[g + 1] - 1) / m; ++t) {
            if (tile_slot[t] < 0) tile_slot[t] = slots;
            ++slots;
        }
    }
    tile_slot[T] = slots;
    for (long long t = T - 1; t >= 0; --t)
        if (tile_slot[t] < 0) tile_slot[t] = tile_slot[t + 1];
    const int fin_blocks = (int)std::min<long long>(2LL * num_sms, std::max<long long>(1, (m + n + 255) / 256));

    // workspace layout inside the static array
    const size_t need = align_up(sizeof(Scalars), 256) + align_up(sizeof(double) * m, 256) * 2 +
                        align_up(sizeof(double) * n, 256) * 2 + align_up(sizeof(double) * (size_t)T * m, 256) +
                        align_up(sizeof(double) * (size_t)std::max(slots, 1) * TW, 256) +
                        align_up(sizeof(double) * 2 * G, 256) +
                        align_up(sizeof(double) * drot::kFinishAcc * fin_blocks, 256) +
                        align_up(sizeof(long long) * (G + 1), 256) + align_up(sizeof(int) * G, 256) +
                        align_up(sizeof(int) * (T + 1), 256);
    if (need > (size_t)DROT_STATIC_SCRATCH_BYTES) return DROT_ERR_TOO_LARGE;
    void *base = nullptr;
    if (static_workspace(dev, &base) != cudaSuccess) return DROT_ERR_CUDA;
    char *cur = static_cast<char *>(base);
    Scalars *sc = carve<Scalars>(cur, 1);
    double *g_num = carve<double>(cur, m), *a_vec = carve<double>(cur, m);
    double *h_num = carve<double>(cur, n), *b_vec = carve<double>(cur, n);
    double *rowpart = carve<double>(cur, (size_t)T * m);
    double *colpart = carve<double>(cur, (size_t)std::max(slots, 1) * TW);
    double *ctapart = carve<double>(cur, 2 * (size_t)G);
    double *finpart = carve<double>(cur, (size_t)drot::kFinishAcc * fin_blocks);
    long long *d_wbound = carve<long long>(cur, G + 1);
    int *d_slot_base = carve<int>(cur, G);
    int *d_tile_slot = carve<int>(cur, T + 1);

    // On a failed call, wait for the work already queued on the stream before returning:
    // the next call (on any thread, once the lock is released) reuses the workspace.
#define STATIC_CUDA(call)                              \
    do {                                               \
        if ((call) != cudaSuccess) {                   \
            cudaStreamSynchronize(stream);             \
            return DROT_ERR_CUDA;                      \
        }                                              \
    } while (0)

    STATIC_CUDA(cudaMemcpyAsync(d_wbound, wbound, sizeof(long long) * (G + 1), cudaMemcpyHostToDevice, stream));
    STATIC_CUDA(cudaMemcpyAsync(d_slot_base, slot_base, sizeof(int) * G, cudaMemcpyHostToDevice, stream));
    STATIC_CUDA(cudaMemcpyAsync(d_tile_slot, tile_slot, sizeof(int) * (T + 1), cudaMemcpyHostToDevice, stream));
    Scalars init{};
    init.rho = rho;
    init.inv_rho = 1.0 / rho;
    init.tol = tol;
    init.max_iter = max_iter;
    init.stop_rule = DROT_STOP_GAP | DROT_STOP_RES_L1;
    init.done = drot::kRunning;
    STATIC_CUDA(cudaMemcpyAsync(sc, &init, sizeof init, cudaMemcpyHostToDevice, stream));
    drot::drot_vector_sums_kernel<<<1, 1024, 0, stream>>>(p, q, warm ? mu : nullptr, warm ? nu : nullptr, m, n, sc);
    STATIC_CUDA(cudaGetLastError());
    Scalars st{};
    STATIC_CUDA(cudaMemcpyAsync(&st, sc, sizeof st, cudaMemcpyDeviceToHost, stream));
    STATIC_CUDA(cudaStreamSynchronize(stream));
    if (st.nonfinite_input & 3) return DROT_ERR_MARGINALS;
    if (st.nonfinite_input & 4) return DROT_ERR_INVALID_ARG;
    if (!(std::fabs(st.sum_p - st.sum_q) <= 1e-9 * std::max(1.0, std::fabs(st.sum_p)))) return DROT_ERR_MARGINALS;

    Plan P;
    P.K = K;
    P.TW = TW;
    P.T = (int)T;
    P.G = G;
    P.slots = std::max(slots, 1);
    P.fin_blocks = fin_blocks;
    P.variant = 1;
    drot::StepArgs A{};
    A.C = C; A.X = X; A.g = g_num; A.h = h_num; A.sc = sc;
    A.rowpart = rowpart; A.colpart = colpart; A.ctapart = ctapart;
    A.wbound = d_wbound; A.slot_base = d_slot_base;
    A.m = m; A.n = n; A.ld = ld; A.inv_n = 1.0 / (double)n; A.inv_m = 1.0 / (double)m;
    A.serp = 1;  // serpentine passes (the default order of drot_solve)
    drot::FinishArgs F{};
    F.rowpart = rowpart; F.colpart = colpart; F.ctapart = ctapart; F.tile_slot = d_tile_slot;
    F.p = p; F.q = q; F.a = a_vec; F.b = b_vec; F.g = g_num; F.h = h_num; F.finpart = finpart; F.sc = sc;
    F.m = m; F.n = n; F.T = (int)T; F.TW = TW; F.G = G; F.inv_n = 1.0 / (double)n; F.inv_m = 1.0 / (double)m;
    F.inv_mn = 1.0 / (double)(m + n);

    if (!warm) {
        const long long work = m * ((n + 3) / 4);
        const int blocks = (int)std::min<long long>(8LL * num_sms, std::max<long long>(1, (work + 255) / 256));
        drot::drot_init_plan_kernel<<<blocks, 256, 0, stream>>>(X, p, q, m, n, ld);
        STATIC_CUDA(cudaGetLastError());
    }
    STATIC_CUDA(launch_step<false>(P, A, stream));
    drot::drot_init_state_kernel<<<fin_blocks, drot::kFinishThreads, 0, stream>>>(F, warm ? mu : nullptr,
                                                                                 warm ? nu : nullptr);
    STATIC_CUDA(cudaGetLastError());

    int done = max_iter > 0 ? drot::kRunning : drot::kIterCap;
    if (max_iter > 0) {
        const double t_iter = 12.0 * (double)m * (double)n / 6.0e12 + 6.0e-6;
        const long long chunk = std::max(1L, std::min(256L, std::lround(2.0e-3 / t_iter)));
        const long long max_chunks = (max_iter + chunk - 1) / chunk + 1;
        for (long long c = 0; c < max_chunks && done == drot::kRunning; ++c) {
            for (long long it = 0; it < chunk; ++it) {
                A.odd = (int)((c * chunk + it) & 1);
                STATIC_CUDA(launch_step<true>(P, A, stream));
                drot::drot_finish_kernel<<<fin_blocks, drot::kFinishThreads, 0, stream>>>(F);
                STATIC_CUDA(cudaGetLastError());
            }
            STATIC_CUDA(cudaMemcpyAsync(&st, sc, sizeof st, cudaMemcpyDeviceToHost, stream));
            STATIC_CUDA(cudaStreamSynchronize(stream));
            done = st.done;
        }
        if (done == drot::kRunning) return DROT_ERR_CUDA;
    }
    const int eblocks = (int)std::min<long long>(2LL * num_sms, std::max<long long>(1, (m + n + 255) / 256));
    drot::drot_export_duals_kernel<<<eblocks, 256, 0, stream>>>(g_num, h_num, sc, mu, nu, m, n, 1.0 / n, 1.0 / m);
    STATIC_CUDA(cudaGetLastError());
    STATIC_CUDA(cudaMemsetAsync(&sc->nnz, 0, sizeof(unsigned long long), stream));
    const int nblocks = (int)std::min<long long>(8LL * num_sms, std::max<long long>(1, (m * n + 255) / 256));
    drot::drot_count_nnz_kernel<<<nblocks, 256, 0, stream>>>(X, m, n, ld, sc);
    STATIC_CUDA(cudaGetLastError());
    STATIC_CUDA(cudaMemcpyAsync(&st, sc, sizeof st, cudaMemcpyDeviceToHost, stream));
    STATIC_CUDA(cudaStreamSynchronize(stream));
#undef STATIC_CUDA

    drot_status out = DROT_OK;
    if (done == drot::kIterCap) out = DROT_NOT_CONVERGED;
    else if (done == drot::kNonFinite) out = DROT_ERR_NONFINITE;
    else if (done == drot::kFault) out = DROT_ERR_TIMEOUT;
    if (res) {
        res->iters = st.k;
        res->primal_obj = st.primal;
        res->dual_obj = st.dual;
        res->gap = st.gap;
        res->res_l1 = st.res_l1;
        res->res_l2 = std::sqrt(st.res_l2);
        res->dual_res = std::sqrt(st.dual_res_prev);
        res->nnz = (int64_t)st.nnz;
        res->status = out;
        if (st.k == 0) res->primal_obj = res->dual_obj = res->gap = res->res_l1 = res->res_l2 = res->dual_res = NAN;
        res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    }
    return out;
}

// ---------------------------------------------------------------------------------------
// Learned warm start (drot_mlp_*): an MLP from per-point features to dual potentials,
// trained by the kernels of drot_mlp.cuh.  Parameters are one flat FP32 vector:
// W1 [256 x 64] b1 [256] W2 [256 x 256] b2 [256] W3 [256 x 256] b3 [256] W4 [256] b4 [1].

struct drot_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    float *w = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;  // DROT_MLP_PARAMS each
    drot::mlp::bf16 *wb = nullptr;   // BF16 copies of W1, W2, W3
    drot::mlp::bf16 *wbT = nullptr;  // BF16 copies of W2^T, W3^T (the backward pass's B operands)
    int *err = nullptr;              // set by a tensor-core product whose wait gave up
    long long rows_cap = 0;
    drot::mlp::bf16 *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *D = nullptr, *D2 = nullptr;
    // transposes (K-major operands of the weight gradients): H1^T, H2^T, D^T (D3^T, then D1^T),
    // D2^T, F^T
    drot::mlp::bf16 *H1T = nullptr, *H2T = nullptr, *DT = nullptr, *D2T = nullptr, *FT = nullptr;
    float *out = nullptr, *g = nullptr, *ebar = nullptr, *wsum = nullptr, *loss = nullptr;
    int seg_cap = 0;
    long long step = 0;
    drot::mlp::bf16 *feat = nullptr;  // warm-start feature rows
    long long feat_cap = 0;
    float *pred = nullptr;
};

namespace {

namespace M = drot::mlp;
constexpr long long kW1 = (long long)M::kWidth * M::kIn, kB1 = M::kWidth;
constexpr long long kW2 = (long long)M::kWidth * M::kWidth, kB2 = M::kWidth;
constexpr long long kW3 = kW2, kB3 = M::kWidth, kW4 = M::kWidth, kB4 = 1;
constexpr long long kOffW1 = 0, kOffB1 = kOffW1 + kW1, kOffW2 = kOffB1 + kB1, kOffB2 = kOffW2 + kW2;
constexpr long long kOffW3 = kOffB2 + kB2, kOffB3 = kOffW3 + kW3, kOffW4 = kOffB3 + kB3, kOffB4 = kOffW4 + kW4;
constexpr long long kParams = kOffB4 + kB4;
static_assert(kParams == DROT_MLP_PARAMS, "parameter layout");
// BF16 copies: W1, W2, W3 back to back; transposed copies: W2^T, W3^T
constexpr long long kBfW1 = 0, kBfW2 = kW1, kBfW3 = kW1 + kW2, kBfCount = kW1 + kW2 + kW3;
constexpr long long kBfT2 = 0, kBfT3 = kW2, kBfTCount = kW2 + kW3;

#define MLP_CUDA(call)                                    \
    do {                                                  \
        if ((call) != cudaSuccess) return DROT_ERR_CUDA;  \
    } while (0)

drot_status mlp_reserve(drot_mlp *net, long long rows, int nseg) {
    if (rows > net->rows_cap) {
        void **bufs[] = {(void **)&net->H1, (void **)&net->H2, (void **)&net->H3, (void **)&net->D,
                         (void **)&net->D2, (void **)&net->out, (void **)&net->g, (void **)&net->H1T,
                         (void **)&net->H2T, (void **)&net->DT, (void **)&net->D2T, (void **)&net->FT};
        for (void **b : bufs) {
            if (*b) cudaFree(*b);
            *b = nullptr;
        }
        const size_t hb = sizeof(M::bf16) * (size_t)rows * M::kWidth;
        if (cudaMalloc(&net->H1, hb) != cudaSuccess || cudaMalloc(&net->H2, hb) != cudaSuccess ||
            cudaMalloc(&net->H3, hb) != cudaSuccess || cudaMalloc(&net->D, hb) != cudaSuccess ||
            cudaMalloc(&net->D2, hb) != cudaSuccess || cudaMalloc(&net->out, sizeof(float) * rows) != cudaSuccess ||
            cudaMalloc(&net->g, sizeof(float) * rows) != cudaSuccess || cudaMalloc(&net->H1T, hb) != cudaSuccess ||
            cudaMalloc(&net->H2T, hb) != cudaSuccess || cudaMalloc(&net->DT, hb) != cudaSuccess ||
            cudaMalloc(&net->D2T, hb) != cudaSuccess ||
            cudaMalloc(&net->FT, sizeof(M::bf16) * (size_t)rows * M::kIn) != cudaSuccess) {
            net->rows_cap = 0;
            return DROT_ERR_OOM;
        }
        net->rows_cap = rows;
    }
    if (nseg > net->seg_cap) {
        if (net->ebar) cudaFree(net->ebar);
        if (net->wsum) cudaFree(net->wsum);
        if (cudaMalloc(&net->ebar, sizeof(float) * nseg) != cudaSuccess ||
            cudaMalloc(&net->wsum, sizeof(float) * nseg) != cudaSuccess)
            return DROT_ERR_OOM;
        net->seg_cap = nseg;
    }
    return DROT_OK;
}

// C = A B^T on the tensor cores (A: Mr x K, B: Nc x K, both BF16 row-major).
cudaError_t mlp_gemm(drot_mlp *net, const M::bf16 *A, int Mr, int K, int lda, const M::bf16 *B, int Nc, int ldb,
                     int epi, float *Cf, M::bf16 *Cb, M::bf16 *CbT, int ldc, int ldt, const float *bias,
                     const M::bf16 *mask) {
    const drot::tc::EpiArgs E{epi, Cf, Cb, CbT, ldc, ldt, bias, mask, net->err};
    if (Nc == M::kWidth) return drot::tc::gemm_tn<M::kWidth>(net->stream, A, Mr, K, lda, B, ldb, E);
    if (Nc == M::kIn) return drot::tc::gemm_tn<M::kIn>(net->stream, A, Mr, K, lda, B, ldb, E);
    return cudaErrorInvalidValue;
}

// Forward pass over `rows` feature rows (a multiple of 64): out[r].  train: also H1^T, H2^T.
drot_status mlp_forward(drot_mlp *net, long long rows, const M::bf16 *F, bool train) {
    cudaStream_t s = net->stream;
    const int R = (int)rows;
    const int W = M::kWidth;
    MLP_CUDA(mlp_gemm(net, F, R, M::kIn, M::kIn, net->wb + kBfW1, W, M::kIn, M::kReluBiasBf16, nullptr, net->H1,
                      train ? net->H1T : nullptr, W, R, net->w + kOffB1, nullptr));
    MLP_CUDA(mlp_gemm(net, net->H1, R, W, W, net->wb + kBfW2, W, W, M::kReluBiasBf16, nullptr, net->H2,
                      train ? net->H2T : nullptr, W, R, net->w + kOffB2, nullptr));
    MLP_CUDA(mlp_gemm(net, net->H2, R, W, W, net->wb + kBfW3, W, W, M::kReluBiasBf16, nullptr, net->H3, nullptr, W,
                      R, net->w + kOffB3, nullptr));
    M::output_kernel<<<(R + 7) / 8, 256, 0, s>>>(net->H3, net->w + kOffW4, net->w + kOffB4, net->out, rows);
    MLP_CUDA(cudaGetLastError());
    return DROT_OK;
}

// BF16 copies of W1, W2, W3 and the transposes of W2, W3 from the FP32 parameters.
cudaError_t mlp_refresh_bf16(drot_mlp *net) {
    cudaStream_t s = net->stream;
    M::to_bf16_kernel<<<64, 256, 0, s>>>(net->w + kOffW1, net->wb + kBfW1, kW1);
    M::to_bf16_kernel<<<64, 256, 0, s>>>(net->w + kOffW2, net->wb + kBfW2, kW2);
    M::to_bf16_kernel<<<64, 256, 0, s>>>(net->w + kOffW3, net->wb + kBfW3, kW3);
    return cudaGetLastError();
}

cudaError_t mlp_refresh_transposes(drot_mlp *net) {
    const dim3 g(M::kWidth / 32, M::kWidth / 32);
    M::transpose_bf16_kernel<<<g, 256, 0, net->stream>>>(net->wb + kBfW2, net->wbT + kBfT2, M::kWidth, M::kWidth);
    M::transpose_bf16_kernel<<<g, 256, 0, net->stream>>>(net->wb + kBfW3, net->wbT + kBfT3, M::kWidth, M::kWidth);
    return cudaGetLastError();
}

// DROT_ERR_TIMEOUT (and the flag cleared) if a tensor-core product gave up waiting.
drot_status mlp_check_err(drot_mlp *net) {
    int e = 0;
    MLP_CUDA(cudaMemcpyAsync(&e, net->err, sizeof(int), cudaMemcpyDeviceToHost, net->stream));
    MLP_CUDA(cudaStreamSynchronize(net->stream));
    if (e) {
        MLP_CUDA(cudaMemsetAsync(net->err, 0, sizeof(int), net->stream));
        MLP_CUDA(cudaStreamSynchronize(net->stream));
        return DROT_ERR_TIMEOUT;
    }
    return DROT_OK;
}

}  // namespace

extern "C" {

drot_status drot_mlp_create(drot_mlp **out, int device) {
    if (!out) return DROT_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return DROT_ERR_CUDA;
    }
    drot_mlp *net = new (std::nothrow) drot_mlp();
    if (!net) return DROT_ERR_OOM;
    net->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete net;
        return DROT_ERR_CUDA;
    }
    const size_t pb = sizeof(float) * kParams;
    if (cudaMalloc(&net->w, pb) != cudaSuccess || cudaMalloc(&net->grad, pb) != cudaSuccess ||
        cudaMalloc(&net->m1, pb) != cudaSuccess || cudaMalloc(&net->m2, pb) != cudaSuccess ||
        cudaMalloc(&net->wb, sizeof(M::bf16) * kBfCount) != cudaSuccess ||
        cudaMalloc(&net->wbT, sizeof(M::bf16) * kBfTCount) != cudaSuccess ||
        cudaMalloc(&net->err, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&net->loss, sizeof(float)) != cudaSuccess) {
        drot_mlp_destroy(net);
        return DROT_ERR_OOM;
    }
    cudaMemsetAsync(net->w, 0, pb, net->stream);
    cudaMemsetAsync(net->m1, 0, pb, net->stream);
    cudaMemsetAsync(net->m2, 0, pb, net->stream);
    cudaMemsetAsync(net->wb, 0, sizeof(M::bf16) * kBfCount, net->stream);
    cudaMemsetAsync(net->wbT, 0, sizeof(M::bf16) * kBfTCount, net->stream);
    cudaMemsetAsync(net->err, 0, sizeof(int), net->stream);
    if (cudaStreamSynchronize(net->stream) != cudaSuccess) {
        drot_mlp_destroy(net);
        return DROT_ERR_CUDA;
    }
    *out = net;
    return DROT_OK;
}

drot_status drot_mlp_destroy(drot_mlp *net) {
    if (!net) return DROT_OK;
    cudaSetDevice(net->device);
    if (net->stream) cudaStreamSynchronize(net->stream);
    void *bufs[] = {net->w,   net->grad, net->m1,  net->m2,   net->wb,   net->wbT, net->err,  net->H1,
                    net->H2,  net->H3,   net->D,   net->D2,   net->H1T,  net->H2T, net->DT,   net->D2T,
                    net->FT,  net->out,  net->g,   net->ebar, net->wsum, net->loss, net->feat, net->pred};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (net->stream) cudaStreamDestroy(net->stream);
    delete net;
    return DROT_OK;
}

drot_status drot_mlp_set_params(drot_mlp *net, const float *params) {
    if (!net || !params) return DROT_ERR_INVALID_ARG;
    cudaSetDevice(net->device);
    cudaStream_t s = net->stream;
    const size_t pb = sizeof(float) * kParams;
    MLP_CUDA(cudaMemcpyAsync(net->w, params, pb, cudaMemcpyHostToDevice, s));
    MLP_CUDA(cudaMemsetAsync(net->m1, 0, pb, s));
    MLP_CUDA(cudaMemsetAsync(net->m2, 0, pb, s));
    MLP_CUDA(mlp_refresh_bf16(net));
    MLP_CUDA(mlp_refresh_transposes(net));
    net->step = 0;
    MLP_CUDA(cudaStreamSynchronize(s));
    return DROT_OK;
}

drot_status drot_mlp_get_params(drot_mlp *net, float *params) {
    if (!net || !params) return DROT_ERR_INVALID_ARG;
    cudaSetDevice(net->device);
    MLP_CUDA(cudaMemcpyAsync(params, net->w, sizeof(float) * kParams, cudaMemcpyDeviceToHost, net->stream));
    MLP_CUDA(cudaStreamSynchronize(net->stream));
    return DROT_OK;
}

drot_status drot_mlp_features(drot_mlp *net, int64_t m, int64_t n, const float *xs, const float *yt,
                              const double *p, const double *q, void *feat, int64_t row0) {
    if (!net || m < 1 || n < 1 || !xs || !yt || !p || !q || !feat || row0 < 0) return DROT_ERR_INVALID_ARG;
    cudaSetDevice(net->device);
    M::features_kernel<<<1, 256, 0, net->stream>>>(xs, yt, p, q, m, n, static_cast<M::bf16 *>(feat), row0);
    MLP_CUDA(cudaGetLastError());
    MLP_CUDA(cudaStreamSynchronize(net->stream));
    return DROT_OK;
}

drot_status drot_mlp_forward(drot_mlp *net, int64_t rows, const void *feat, float *out) {
    if (!net || rows < 64 || rows % 64 != 0 || !feat || !out) return DROT_ERR_INVALID_ARG;
    cudaSetDevice(net->device);
    drot_status st = mlp_reserve(net, rows, 1);
    if (st != DROT_OK) return st;
    st = mlp_forward(net, rows, static_cast<const M::bf16 *>(feat), false);
    if (st != DROT_OK) return st;
    MLP_CUDA(cudaMemcpyAsync(out, net->out, sizeof(float) * rows, cudaMemcpyDeviceToDevice, net->stream));
    return mlp_check_err(net);
}

drot_status drot_mlp_train_step(drot_mlp *net, int64_t rows, const void *feat, const float *target,
                                const float *weight, const int32_t *seg, int32_t nseg, float lr, int update,
                                float *loss, float *grad) {
    if (!net || rows < 64 || rows % 64 != 0 || !feat || !target || !weight || !seg || nseg < 1)
        return DROT_ERR_INVALID_ARG;
    cudaSetDevice(net->device);
    drot_status st = mlp_reserve(net, rows, nseg);
    if (st != DROT_OK) return st;
    cudaStream_t s = net->stream;
    const M::bf16 *F = static_cast<const M::bf16 *>(feat);
    st = mlp_forward(net, rows, F, true);
    if (st != DROT_OK) return st;
    const int R = (int)rows;
    const int W = M::kWidth;
    MLP_CUDA(cudaMemsetAsync(net->grad, 0, sizeof(float) * kParams, s));
    MLP_CUDA(cudaMemsetAsync(net->ebar, 0, sizeof(float) * nseg, s));
    MLP_CUDA(cudaMemsetAsync(net->wsum, 0, sizeof(float) * nseg, s));
    MLP_CUDA(cudaMemsetAsync(net->loss, 0, sizeof(float), s));
    M::loss_pass1_kernel<<<256, 256, 0, s>>>(net->out, target, weight, seg, rows, net->ebar, net->wsum);
    M::loss_pass2_kernel<<<256, 256, 0, s>>>(net->out, target, weight, seg, rows, net->ebar, net->wsum,
                                             1.f / (float)nseg, net->g, net->loss);
    // layer 4 and the gradient at the output of layer 3 (through its ReLU): D3 and D3^T
    M::output_backward_kernel<<<R / 64, W, 0, s>>>(net->g, net->H3, net->w + kOffW4, rows, net->grad + kOffW4,
                                                   net->grad + kOffB4, net->D, net->DT);
    // F^T for the weight gradient of layer 1
    M::transpose_bf16_kernel<<<dim3(M::kIn / 32, R / 32), 256, 0, s>>>(F, net->FT, R, M::kIn);
    MLP_CUDA(cudaGetLastError());
    // layer 3: dW3 = D3^T H2 (K = rows, split over the grid), db3 = colsum D3,
    // D2 = (D3 W3) o (H2 > 0) = D3 (W3^T)^T o mask, with D2^T
    MLP_CUDA(mlp_gemm(net, net->DT, W, R, R, net->H2T, W, R, M::kAtomicF32, net->grad + kOffW3, nullptr, nullptr,
                      W, 0, nullptr, nullptr));
    M::column_sum_kernel<<<R / 64, W, 0, s>>>(net->D, rows, net->grad + kOffB3);
    MLP_CUDA(mlp_gemm(net, net->D, R, W, W, net->wbT + kBfT3, W, W, M::kMaskBf16, nullptr, net->D2, net->D2T, W, R,
                      nullptr, net->H2));
    // layer 2: dW2 = D2^T H1, db2, D1 = (D2 W2) o (H1 > 0) with D1^T (D1 reuses D, D1^T reuses D^T)
    MLP_CUDA(mlp_gemm(net, net->D2T, W, R, R, net->H1T, W, R, M::kAtomicF32, net->grad + kOffW2, nullptr, nullptr,
                      W, 0, nullptr, nullptr));
    M::column_sum_kernel<<<R / 64, W, 0, s>>>(net->D2, rows, net->grad + kOffB2);
    MLP_CUDA(mlp_gemm(net, net->D2, R, W, W, net->wbT + kBfT2, W, W, M::kMaskBf16, nullptr, net->D, net->DT, W, R,
                      nullptr, net->H1));
    // layer 1: dW1 = D1^T F (N = feature width), db1
    MLP_CUDA(mlp_gemm(net, net->DT, W, R, R, net->FT, M::kIn, R, M::kAtomicF32, net->grad + kOffW1, nullptr,
                      nullptr, M::kIn, 0, nullptr, nullptr));
    M::column_sum_kernel<<<R / 64, W, 0, s>>>(net->D, rows, net->grad + kOffB1);
    MLP_CUDA(cudaGetLastError());
    if (update) {
        net->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, (float)net->step), c2 = 1.f - std::pow(b2, (float)net->step);
        struct Seg { long long off, cnt, bf; } segs[] = {
            {kOffW1, kW1, kBfW1}, {kOffB1, kB1, -1}, {kOffW2, kW2, kBfW2}, {kOffB2, kB2, -1},
            {kOffW3, kW3, kBfW3}, {kOffB3, kB3, -1}, {kOffW4, kW4 + kB4, -1}};
        for (const Seg &g : segs)
            M::adam_kernel<<<64, 256, 0, s>>>(net->w + g.off, net->grad + g.off, net->m1 + g.off, net->m2 + g.off,
                                              g.bf >= 0 ? net->wb + g.bf : nullptr, g.cnt, lr, b1, b2, 1e-8f, c1, c2);
        MLP_CUDA(cudaGetLastError());
        MLP_CUDA(mlp_refresh_transposes(net));
    }
    if (loss) MLP_CUDA(cudaMemcpyAsync(loss, net->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    if (grad) MLP_CUDA(cudaMemcpyAsync(grad, net->grad, sizeof(float) * kParams, cudaMemcpyDeviceToHost, s));
    return mlp_check_err(net);
}

drot_status drot_mlp_warm_start(drot_mlp *net, int64_t m, int64_t n, const float *xs, const float *yt,
                                const double *p, const double *q, double cost_scale, const float *C, int64_t ld,
                                float *X, double *mu, double *nu) {
    if (!net || m < 1 || n < 1 || !xs || !yt || !p || !q || !C || !X || !mu || !nu || ld < n || ld % 4 != 0 ||
        !(cost_scale > 0.0))
        return DROT_ERR_INVALID_ARG;
    cudaSetDevice(net->device);
    cudaStream_t s = net->stream;
    const long long rows = (m + 63) / 64 * 64;
    if (rows > net->feat_cap) {
        if (net->feat) cudaFree(net->feat);
        if (net->pred) cudaFree(net->pred);
        net->feat = nullptr;
        net->pred = nullptr;
        net->feat_cap = 0;
        if (cudaMalloc(&net->feat, sizeof(M::bf16) * rows * M::kIn) != cudaSuccess ||
            cudaMalloc(&net->pred, sizeof(float) * rows) != cudaSuccess)
            return DROT_ERR_OOM;
        net->feat_cap = rows;
    }
    drot_status st = mlp_reserve(net, rows, 1);
    if (st != DROT_OK) return st;
    MLP_CUDA(cudaMemsetAsync(net->feat, 0, sizeof(M::bf16) * rows * M::kIn, s));
    M::features_kernel<<<1, 256, 0, s>>>(xs, yt, p, q, m, n, net->feat, 0);
    MLP_CUDA(cudaGetLastError());
    st = mlp_forward(net, rows, net->feat, false);
    if (st != DROT_OK) return st;
    // centred prediction in units of C, then the c-transforms (exact dual feasibility)
    M::centre_prediction_kernel<<<1, 1024, 0, s>>>(net->out, p, m, 1.0 / cost_scale, mu);
    M::c_transform_cols_kernel<<<(int)std::max<long long>(1, (n + 127) / 128), 128, 0, s>>>(C, m, n, ld, mu, nu);
    M::c_transform_rows_kernel<<<(int)std::max<long long>(1, (m + 7) / 8), 256, 0, s>>>(C, m, n, ld, nu, mu);
    // X_0 = p q^T (Sec. 4)
    const long long work = m * ((n + 3) / 4);
    drot::drot_init_plan_kernel<<<(int)std::min<long long>(1184, std::max<long long>(1, (work + 255) / 256)), 256, 0,
                                  s>>>(X, p, q, m, n, ld);
    MLP_CUDA(cudaGetLastError());
    return mlp_check_err(net);
}

}  // extern "C"
