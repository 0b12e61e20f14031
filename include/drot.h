/*
 * drot.h - C ABI of the B300 (sm_103a) Douglas-Rachford optimal-transport solver.
 *
 * The solver computes an optimal transport plan for
 *
 *     minimise <C, X>  subject to  X >= 0,  X 1_n = p,  X^T 1_m = q        (Sec. 1, eq. ot:dist)
 *
 * by Douglas-Rachford splitting with f(X) = <C,X> + I_{X>=0} and g = indicator of the
 * marginal constraints (Sec. 3, eq. ot:dist:operator:primal:composite), executed in the
 * single-array form of Algorithm 1 (Sec. 3.1):
 *
 *     X_{k+1}   = [X_k + phi_k 1^T + 1 psi_k^T - rho C]_+                       (step 4)
 *     r = X_{k+1} 1 - p,  s = X_{k+1}^T 1 - q,  beta = sum(r) / (m+n)          (step 5)
 *     phi_{k+1} = (a_k - 2r + (2beta - alpha_k)) / n                            (step 6)
 *     psi_{k+1} = (b_k - 2s + (2beta - alpha_k)) / m                            (step 7)
 *     a -= r,  b -= s,  alpha -= beta                                           (step 8)
 *
 * (the paper names the column-side vector \varphi; it is psi here).  The dual variables
 * returned are mu = phi / rho and nu = psi / rho (Appendix A.2, eq. dual:var).
 *
 * Stopping test (Sec. 3.1, "Stopping criteria"), evaluated on the device after every
 * iteration on the quantities selected by drot_config.stop_rule (default: gap and l1
 * residual): gap = |<C, X_k> - (p^T phi_k + q^T psi_k)/rho| <= tol,
 * ||r||_1 + ||s||_1 <= tol, r_dual = ||[(phi/rho) 1^T + 1 (psi/rho)^T - C]_+||_F <= tol.
 * r_dual of (phi_k, psi_k) is produced by the pass that computes X_{k+1}, so the test
 * uses the value from the same pass (one iteration older than gap and residuals).
 *
 * Data layout: C and X are dense row-major FP32 m x n matrices with row pitch ld
 * (floats): entry (i, j) lives at base[i*ld + j].  ld must be >= n and a multiple of 4,
 * and both base pointers 16-byte aligned, so that every row starts on a 16-byte
 * boundary.  Columns n..ld-1 (row padding) may be read but take no part in the
 * arithmetic and are never written.  p, q, mu, nu are FP64 vectors.  Iterates X are FP32; every reduction that
 * feeds the stopping test or the vector updates (row/column sums, <C,X>, the norms,
 * the dual objective) is accumulated in FP64 across threads.
 *
 * Pointers: all buffers of one call are either device memory of the handle's device
 * or host memory (pageable or pinned); mixing the two in one call is rejected.  With
 * host buffers the library copies inputs to a device workspace owned by the handle,
 * solves, and copies X, mu, nu back before returning.  The caller owns every buffer
 * it passes; the handle owns only its workspace.
 *
 * Threading and streams: a handle is not thread-safe; use one handle per host thread.
 * Work is issued on the configured stream (or a stream the handle creates).  Every
 * solve call returns only after the final status has been read back, with X, mu, nu
 * and the result struct complete.
 *
 * Errors: every entry point returns a drot_status.  Invalid arguments are rejected on
 * the host before any launch.  Device-side waits exist and each one ends:
 *   - software waits on other blocks poll a bounded number of times: the persistent
 *     solve's grid barriers (drot_config.wait_limit, default 2^24 polls) and the TMA-fed
 *     step's mbarrier ring (2^20 polls per wait).  A wait that runs out sets a fault flag
 *     that makes every other block leave, and the call returns DROT_ERR_TIMEOUT with the
 *     CUDA context still usable;
 *   - the cluster-resident solve's hardware cluster barriers wait only on the CTAs of the
 *     same cluster, which the hardware schedules together, and on nothing outside it;
 *   - kernels chained by programmatic dependent launch wait (griddepcontrol.wait) for the
 *     kernel before them on the same stream, which never waits on a later one.
 * Kernels never trap; a NaN/Inf in the iteration ends the solve with DROT_ERR_NONFINITE.
 */
#ifndef DROT_H
#define DROT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct drot_handle drot_handle;

typedef enum {
    DROT_OK = 0,                /* converged: the stopping test fired */
    DROT_ERR_INVALID_ARG = 1,   /* bad size, pitch, alignment, pointer kind, tolerance ... */
    DROT_ERR_MARGINALS = 2,     /* p or q negative / non-finite, or |sum p - sum q| > 1e-9 */
    DROT_ERR_OOM = 3,           /* device or pinned-host allocation failed */
    DROT_ERR_CUDA = 4,          /* a CUDA runtime call failed (message via drot_last_error) */
    DROT_NOT_CONVERGED = 5,     /* max_iter iterations ran; outputs hold the last iterate */
    DROT_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up (persistent grid barrier, TMA ring);
                                   the context stays usable */
    DROT_ERR_NONFINITE = 7,     /* a NaN/Inf appeared in the iteration; outputs hold the last iterate */
    DROT_ERR_TOO_LARGE = 8      /* drot_solve_static: the problem's workspace exceeds DROT_STATIC_SCRATCH_BYTES */
} drot_status;

/* Quantities that gate the stopping test (bitmask, drot_config.stop_rule). */
#define DROT_STOP_GAP 1       /* |<C,X> - (p^T phi + q^T psi)/rho| <= tol */
#define DROT_STOP_RES_L1 2    /* ||X 1 - p||_1 + ||X^T 1 - q||_1 <= tol */
#define DROT_STOP_DUAL_RES 4  /* ||[(phi/rho) 1^T + 1 (psi/rho)^T - C]_+||_F <= tol */

typedef struct {
    int device;                 /* CUDA device ordinal (default 0) */
    void *stream;               /* cudaStream_t to issue work on; NULL: the handle creates one */
    int stop_rule;              /* bitmask of DROT_STOP_*; 0 selects DROT_STOP_GAP | DROT_STOP_RES_L1 */
    double rho0;                /* rho = rho0 / (m + n) when a call passes rho <= 0 (default 2, Sec. 4) */
    int graph_iters;            /* iterations per CUDA-graph replay; 0: chosen from the problem size */
    int tile_k;                 /* float4 chunks per lane per row segment (1, 2 or 4); 0: automatic.
                                   drot_solve_batched: every problem of the batch takes this tile
                                   width and the tile-policy autotuner is skipped */
    int grid_ctas;              /* CTAs of the fused step kernel; 0: automatic */
    int profile;                /* 1: time every fused-step launch with CUDA events (drot_get_profile) */
    int step_variant;           /* fused step: 1 register-fed (128-bit loads), 2 TMA-fed (bulk copies into a
                                   shared-memory ring), 3 async-copy-fed (per-warp cp.async ring);
                                   0: automatic */
    int deterministic;          /* 1: row/column sums as fixed-order FP64 partials (bitwise reproducible
                                   runs); 0 (default): FP64 atomic adds into the totals (faster; the
                                   summation order, hence the last bits, may vary between runs) */
    int autotune;               /* 1: on the first solve of each (m, n), time the fused-step variants and tile
                                   widths on a scratch plan and keep the fastest unless it beats the default
                                   plan by less than 3 % (costs one m x ld FP32 scratch buffer and a few
                                   launches); explicit step_variant / tile_k win.  drot_solve_batched: on a
                                   cold start of a batch shape not tuned yet, time four tile policies on the
                                   batch itself before X_0 is written and keep the fastest for that shape */
    int persistent;             /* 1: run the iterations in one cooperative launch (every CTA resident, two
                                   bounded grid barriers per iteration, register-fed step, FP64-atomic
                                   totals); 0: CUDA graphs of [step, finish] launches (default) */
    int c_skip;                 /* 1: skip the load of C every other iteration (Claim 1, Sec. 3.3): passes
                                   alternate between reading X and C while storing X - rho C, and reading
                                   only that array; 10 instead of 12 bytes per entry on average.  The
                                   stopping test runs after the C-reading passes only.  Uses the
                                   register-fed step and CUDA graphs (persistent is ignored) */
    int cluster;                /* small problems on one thread-block cluster (X and C held in shared
                                   memory for the whole solve, column and scalar totals exchanged in
                                   distributed shared memory), mid-size ones grid-resident (one
                                   cooperative launch of at most one CTA per SM, each holding its rows
                                   of X and C in shared memory, two grid barriers per iteration):
                                   0 automatic (the cluster where the problem fits, else grid-resident
                                   where it fits and has at least 2e6 entries, when none of step_variant, tile_k, grid_ctas,
                                   persistent, deterministic, c_skip, trace is set), 1 neither (the
                                   streaming path), 2 cluster required, 3 grid-resident required
                                   (2, 3: DROT_ERR_INVALID_ARG if the problem does not fit; FP32 only,
                                   c_skip off) */
    double *trace;              /* optional device buffer of 2 * trace_len doubles, written during a solve:
                                   trace[2(k-1)] = <C, X_k> and trace[2(k-1)+1] = ||X_k 1 - p||_1 +
                                   ||X_k^T 1 - q||_1 for iterations k = 1 .. min(K, trace_len) (the
                                   quantities of the stopping test, Sec. 3.1; with c_skip only the
                                   C-reading iterations are written).  NULL: no trace.  Setting it keeps
                                   the automatic choice off the cluster-resident path, which has none */
    int64_t trace_len;
    int64_t wait_limit;         /* polls before a grid-barrier wait of the persistent solve gives up
                                   (0: 2^24, about a second); the first CTA to give up sets a fault flag
                                   that makes every other CTA leave, and the solve returns
                                   DROT_ERR_TIMEOUT with the context intact.  A small value makes the
                                   barriers give up at once: it exists to test that path */
    int serpentine;             /* order of the FP32 fused-step passes: 1 alternate (every other pass walks
                                   each CTA's rows backwards, so it starts on the lines of X and C the pass
                                   before it left in L2; the automatic graph length is then even), -1 every
                                   pass forwards, 0 automatic (alternate).  Changes only the order in which
                                   partial sums are formed, hence the last bits of a run.  Also applies
                                   to drot_solve_batched; the FP64 solve always walks forwards */
    int batch_narrow;           /* drot_solve_batched: tiles with at most 256 valid columns go to a second
                                   kernel that packs four or eight rows into one warp iteration.  0 automatic
                                   (while the active problems' narrow tiles hold at least 65536 rows: below
                                   that the extra launch costs more than packing saves), 1 always, -1 never */
} drot_config;

typedef struct {
    int64_t iters;              /* iterations performed by this call */
    double primal_obj;          /* <C, X_K> */
    double dual_obj;            /* p^T mu + q^T nu */
    double gap;                 /* |primal_obj - dual_obj| */
    double res_l1;              /* ||X_K 1 - p||_1 + ||X_K^T 1 - q||_1 */
    double res_l2;              /* sqrt(||X_K 1 - p||^2 + ||X_K^T 1 - q||^2) */
    double dual_res;            /* r_dual of the vectors that entered the last pass */
    int64_t nnz;                /* number of strictly positive entries of X_K */
    int32_t status;             /* the drot_status of this solve */
    double seconds;             /* host wall time of the call */
} drot_result;

/* One problem of a batch: same meaning and layout rules as drot_solve's arguments. */
typedef struct {
    int64_t m, n, ld;
    const float *C;
    const double *p, *q;
    float *X;
    double *mu, *nu;
    double rho;                 /* <= 0: rho0 / (m + n) */
} drot_problem;

typedef struct {
    double step_ms_total;       /* summed device time of timed fused-step launches */
    int64_t step_launches;      /* fused-step launches that did work and were timed */
    int64_t kernel_launches;    /* all kernels this handle launched (including early exits) */
    int64_t graph_replays;      /* CUDA-graph replays issued */
    int32_t tile_k, grid_ctas, col_tiles, graph_iters;  /* the plan of the last solve */
    int32_t step_variant, stages;                       /* fused-step variant (1 register-fed, 2 TMA-fed,
                                                           3 async-copy ring, 4 cluster-resident, 5 FP64)
                                                           and ring depth (cluster size for 4) used */
    double finish_ms_total;     /* summed device time of the finish launches of the timed iterations */
    double iter_ms_total;       /* summed device time from each timed step launch to the next one */
} drot_profile;

/* Fill cfg with the defaults listed above. */
void drot_config_default(drot_config *cfg);

/* Create a handle on cfg->device (cfg NULL: defaults).  *h is set on DROT_OK only. */
drot_status drot_create(drot_handle **h, const drot_config *cfg);

/* Solve one problem (Algorithm 1, Sec. 3.1; stopping test as above).
 *   m, n       problem size, m >= 1, n >= 1
 *   C, ld      cost, row-major FP32 with pitch ld (unchanged by the call)
 *   p, q       marginals, FP64, nonnegative, equal total mass within 1e-9
 *   rho        penalty parameter; <= 0 selects rho0 / (m + n)
 *   tol        tolerance of the stopping test; < 0 runs exactly max_iter iterations
 *   max_iter   iteration cap, >= 0
 *   X          in/out plan, same layout as C.  warm == 0: overwritten with X_0 = p q^T
 *              (Sec. 4).  warm != 0: holds X_0 on entry.
 *   mu, nu     out: dual vectors phi/rho (m) and psi/rho (n).  warm != 0: on entry they
 *              hold mu_0, nu_0 and the iteration starts from phi_0 = rho mu_0,
 *              psi_0 = rho nu_0 with a_0 = Y_0 1 - p, b_0 = Y_0^T 1 - q,
 *              Y_0 = X_0 + phi_0 1^T + 1 psi_0^T.
 *   res        out (host), may be NULL.
 * Returns DROT_OK when the test fired, DROT_NOT_CONVERGED after max_iter iterations. */
drot_status drot_solve(drot_handle *h, int64_t m, int64_t n, const float *C, int64_t ld,
                       const double *p, const double *q, double rho, double tol, int64_t max_iter,
                       float *X, double *mu, double *nu, int warm, drot_result *res);

/* drot_solve in double precision (the paper runs its robustness experiments in FP32 and
 * FP64, Sec. 4).  Same arguments and meaning as drot_solve, with C and X FP64: row pitch
 * ld a multiple of 2 (16-byte aligned rows), 16-byte aligned base pointers.  Every
 * quantity of Algorithm 1 is FP64 (entries, phi, psi, the per-entry update and all
 * sums).  One step variant (register-fed, 256-column tiles, on the same work split,
 * finish kernel and iteration graphs); step_variant, tile_k and autotune are ignored,
 * the cluster-resident path is not used (cluster = 2: DROT_ERR_INVALID_ARG), and
 * persistent or c_skip return DROT_ERR_INVALID_ARG. */
drot_status drot_solve_f64(drot_handle *h, int64_t m, int64_t n, const double *C, int64_t ld,
                           const double *p, const double *q, double rho, double tol, int64_t max_iter,
                           double *X, double *mu, double *nu, int warm, drot_result *res);

/* Solve B independent problems of uneven sizes (no counterpart in the paper, which
 * solves one problem at a time; each problem follows drot_solve exactly).  All problems
 * share tol, max_iter and warm; each stops on its own test.  res: B entries (host),
 * may be NULL.  Returns DROT_OK if every problem converged, else the first non-OK
 * status among the problems (per-problem status in res[b].status). */
drot_status drot_solve_batched(drot_handle *h, int32_t B, const drot_problem *probs, double tol,
                               int64_t max_iter, int warm, drot_result *res);

/* Allocation-free solve.  The paper has no counterpart: this entry point exists for callers that
 * cannot allocate GPU memory at the time they solve - code that runs inside a memory pool or arena
 * owned by another component (a framework's caching allocator, a renderer or a simulator that reserved
 * all device memory at start-up), plugins whose host forbids cudaMalloc after initialisation, and
 * latency-critical loops that must never enter the allocator.  Everyone else should use drot_solve.
 *
 * It solves one problem exactly like drot_solve with a default configuration (same arguments and
 * meaning; rho <= 0 selects 2/(m+n); stop when gap <= tol and l1 residual <= tol), on device pointers
 * of the caller's current device, without a handle.  It allocates nothing: no cudaMalloc or cudaFree,
 * no pinned host memory, no CUDA graph.  Its workspace is one fixed array of
 * DROT_STATIC_SCRATCH_BYTES (16 MiB) in the library's own device memory, which every GPU that loads
 * the library keeps until the process exits.
 *   - Size limit: the workspace is about 8*(3m + 2n + T*m) + 4096*(T + 2*SMs) + 8 KiB bytes with
 *     T = ceil(n/512) (n >= 1536; narrower problems use narrower tiles).  m = n = 20000 fits (~8 MB).
 *     A problem that does not fit returns DROT_ERR_TOO_LARGE before anything is launched.
 *   - The array is placed in device memory when the CUDA runtime loads this library's device code on
 *     that device, which under lazy module loading (the default) is the first use of the library
 *     there - the first kernel launch or address lookup of any entry point.  A host that reserves all
 *     free device memory up front must therefore make one call into this library on each device
 *     before doing so (or run with CUDA_MODULE_LOADING=EAGER, which places it when the library is
 *     loaded); otherwise that first call can fail with DROT_ERR_CUDA (out of memory).
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress, with that
 *     device current).  Make that first call before any stream capture is started on the device.
 *   - Every call on a device uses the same array.  Two calls whose GPU work overlapped would race on
 *     it and corrupt each other's results, so the library prevents it: calls on the same device are
 *     serialised by a lock inside the library (a second host thread blocks until the first call has
 *     returned) and every call, error returns included, waits for its own GPU work before returning.
 *     Calls on different devices do not block each other.  Each call initialises every part of the
 *     array it reads, so nothing from an earlier call leaks into a later one.
 *   - Work is issued on `stream` (a cudaStream_t; NULL: the default stream) and the call returns
 *     after synchronising it, with X, mu, nu and *res (may be NULL) complete. */
#define DROT_STATIC_SCRATCH_BYTES (16u << 20)
drot_status drot_solve_static(int64_t m, int64_t n, const float *C, int64_t ld, const double *p,
                              const double *q, double rho, double tol, int64_t max_iter, float *X,
                              double *mu, double *nu, int warm, void *stream, drot_result *res);

/* ------------------------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper: the paper always starts from X_0 = p q^T).
 * An MLP maps per-point features of each source point to its dual potential; the seed follows
 * Lemma opt-rel (Appendix A.2): a primal-dual optimum (X*, mu*, nu*) gives the DR fixed point
 * Y* = X* + rho (mu* 1^T + 1 nu*^T), so predicted duals enter drot_solve as mu_0, nu_0 (warm = 1).
 *
 * Network: 64 features -> 256 -> 256 -> 256 -> 1 with ReLU; FP32 parameters (one flat vector of
 * DROT_MLP_PARAMS floats: W1[256x64] b1[256] W2[256x256] b2[256] W3[256x256] b3[256] W4[256] b4[1],
 * weights row-major [out x in]) with BF16 copies for the matrix products, BF16 activations,
 * FP32 accumulation, Adam updates.  Feature rows are BF16, DROT_MLP_FEATURES wide; see
 * drot_mlp_features for their content.  All buffers are device memory of the network's device.
 * The matrix products run on the tcgen05 tensor cores (operands staged by TMA, accumulators in
 * tensor memory); their waits are bounded, and a product that gave up makes drot_mlp_forward,
 * drot_mlp_train_step and drot_mlp_warm_start return DROT_ERR_TIMEOUT. */
#define DROT_MLP_FEATURES 64
#define DROT_MLP_WIDTH 256
#define DROT_MLP_PARAMS (256 * 64 + 256 + 2 * (256 * 256 + 256) + 256 + 1)
typedef struct drot_mlp drot_mlp;

/* Create a network on `device` with all parameters zero (set them with drot_mlp_set_params). */
drot_status drot_mlp_create(drot_mlp **net, int device);
drot_status drot_mlp_destroy(drot_mlp *net);
/* Copy DROT_MLP_PARAMS floats from / to host memory; setting resets the Adam state. */
drot_status drot_mlp_set_params(drot_mlp *net, const float *params);
drot_status drot_mlp_get_params(drot_mlp *net, float *params);

/* Feature rows of the m source points of one problem, written to rows [row0, row0 + m) of `feat`
 * (BF16, DROT_MLP_FEATURES per row).  xs: m x 2 and yt: n x 2 FP32 point coordinates in the unit
 * square; p, q FP64 marginals.  Row content: x_i (2), m p_i, 4x4 histograms of both clouds
 * weighted by their marginals (16 + 16), weighted means of both clouds (2 + 2), weighted
 * variances and covariance of the target cloud (3), a constant 1, zeros. */
drot_status drot_mlp_features(drot_mlp *net, int64_t m, int64_t n, const float *xs, const float *yt,
                              const double *p, const double *q, void *feat, int64_t row0);

/* out[r] = network(feat[r]) for `rows` rows (a multiple of 64). */
drot_status drot_mlp_forward(drot_mlp *net, int64_t rows, const void *feat, float *out);

/* One training step on `rows` feature rows (a multiple of 64) grouped into `nseg` problems by
 * seg[r] in [0, nseg) (-1: padding row, ignored).  Loss (gauge invariant: a constant added to a
 * problem's potentials does not change it): with e_r = out_r - target_r and ebar_s the
 * weight-averaged e over problem s, L = (1/nseg) sum_s sum_{r in s} weight_r (e_r - ebar_s)^2.
 * update != 0 applies one Adam step (lr; beta 0.9, 0.999; eps 1e-8).  loss (host, may be NULL)
 * receives L; grad (host, may be NULL) receives the DROT_MLP_PARAMS gradient before the update. */
drot_status drot_mlp_train_step(drot_mlp *net, int64_t rows, const void *feat, const float *target,
                                const float *weight, const int32_t *seg, int32_t nseg, float lr, int update,
                                float *loss, float *grad);

/* Warm start for one problem: predicts the source potentials, centres them (p-weighted mean 0),
 * divides by cost_scale (the factor by which the squared distances were divided to form C),
 * sets nu_j = min_i (C_ij - mu_i) and then mu_i = min_j (C_ij - nu_j), so mu_i + nu_j <= C_ij;
 * writes X = p q^T.  Pass X, mu, nu to drot_solve with warm = 1. */
drot_status drot_mlp_warm_start(drot_mlp *net, int64_t m, int64_t n, const float *xs, const float *yt,
                                const double *p, const double *q, double cost_scale, const float *C,
                                int64_t ld, float *X, double *mu, double *nu);

/* Release the handle and its workspace (NULL is accepted). */
drot_status drot_destroy(drot_handle *h);

/* Counters and timings accumulated since the handle was created or last reset. */
drot_status drot_get_profile(drot_handle *h, drot_profile *out);
drot_status drot_reset_profile(drot_handle *h);

/* Static description of a status code. */
const char *drot_status_string(drot_status s);

/* Text of the last error recorded on this handle ("" if none). */
const char *drot_last_error(drot_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* DROT_H */
