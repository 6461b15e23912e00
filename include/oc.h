/*
 * oc.h -- C ABI of the out-of-core stencil loop-chain executor (liboc.so).
 *
 * Method: "Beyond 16GB: Out-of-Core Stencil Computations" (arXiv 1709.02125).
 *   - Sec. 3: the OPS abstraction -- datasets on a structured block, stencils
 *     (sets of relative offsets), and parallel loops over an iteration range
 *     whose arguments carry an access mode (read / write / read-write). Points of
 *     a loop may run in any order. Loops are queued lazily; any call that returns
 *     data to the user ends the chain and forces execution, and a dependency
 *     analysis turns the chain into a skewed tiling along one axis.
 *   - Sec. 4, Algorithm 1: tiles are streamed through a bounded device memory
 *     with three CUDA streams (upload / compute / download).
 *   - Sec. 4.1: read-only data is never downloaded, write-first data is never
 *     uploaded, the unsafe "cyclic" option skips downloads of write-first data,
 *     and the first tile of the next chain is prefetched speculatively.
 *
 * Conventions shared by every entry point:
 *   - Every function returns OC_OK (0) or a negative OC_ERR_* code; the message of
 *     the last failure is returned by oc_last_error(). No entry point aborts the
 *     process on bad input.
 *   - One context per process, created by oc_init() and destroyed by
 *     oc_finalize(). The library is not thread-safe: call it from one host thread.
 *   - Handles (datasets, reductions) are small non-negative ints.
 *   - Coordinates: x is the fastest axis. The slowest axis (y in 2-D, z in 3-D) is
 *     the tiling axis. Interior indices run 0..n-1; halo indices are negative or
 *     >= n. A point p of a loop range is (x, y[, z]).
 *   - Host arrays handed to / returned by the library are dense C-order arrays of
 *     the full allocated extent INCLUDING halos: for a 2-D dataset of size
 *     (nx, ny) with halos (hlo, hhi) the array has shape
 *     (ny + hlo[1] + hhi[1], nx + hlo[0] + hhi[0]) and element (x, y) lives at
 *     [(y + hlo[1]) * (nx + hlo[0] + hhi[0]) + (x + hlo[0])]; 3-D likewise with z
 *     outermost.
 */
#ifndef OC_H
#define OC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define OC_OK            0
#define OC_ERR_ARG      -1  /* invalid argument, handle, range or stencil          */
#define OC_ERR_BUDGET   -2  /* the device budget cannot hold one tile of the chain  */
#define OC_ERR_CUDA     -3  /* a CUDA runtime call failed (message has the reason)  */
#define OC_ERR_TIMEOUT  -4  /* a bounded wait on a stream or event expired (below)  */
#define OC_ERR_STATE    -5  /* call out of order (no context, double init, ...)     */
#define OC_ERR_NOMEM    -6  /* host (pinned) allocation failed                      */

/* ---- element types ------------------------------------------------------- */
#define OC_F64 0
#define OC_F32 1

/* ---- access modes (Sec. 3: read / write / both; plus reductions) --------- */
#define OC_READ   1
#define OC_WRITE  2
#define OC_RW     3
#define OC_REDUCE 4   /* oc_arg.dat is a reduction handle, not a dataset */

/* ---- reduction operators ---------------------------------------------------- */
#define OC_SUM 0
#define OC_MAX 1
#define OC_MIN 2

/* ---- context flags (oc_init / oc_set_flag) ----------------------------------
 * OC_FLAG_CYCLIC   Sec. 4.1 "cyclic" optimisation: datasets whose first access in a
 *                  chain is a write are treated as per-chain temporaries and are
 *                  never downloaded by a streamed plan (resident datasets and managed
 *                  stores keep their values). Their host copy is then stale: oc_fetch_dat
 *                  returns unspecified values for them, and a later chain that reads one
 *                  before writing it fails with OC_ERR_STATE (nothing of it runs) until a
 *                  chain writes the dataset without skipping its download. Off by default.
 * OC_FLAG_PREFETCH Sec. 4.1 speculative prefetch: while the last tile of a chain
 *                  runs, upload the first tile of the next chain assuming it has
 *                  the same plan; the next chain uploads only what is missing.
 * OC_FLAG_GRAPHS   capture a chain once as a CUDA graph and replay it when the same
 *                  chain shape runs again: the whole chain (copies on all three
 *                  streams, kernels, reductions, prefetch) when neither TRACE nor
 *                  PROFILE is set and no in-core upload is pending, else the kernels
 *                  of each tile.
 * OC_FLAG_DRYRUN   no device at all: chains are analysed and planned (the plan can
 *                  be inspected with oc_plan_*), nothing is executed, and
 *                  oc_reduce / oc_fetch_dat return OC_ERR_STATE. Host-only use.
 * OC_FLAG_PROFILE  bracket every run of consecutive launches of one kernel id with
 *                  a pair of CUDA events on the compute stream and accumulate
 *                  per-kernel device time (oc_kernel_stats).
 * OC_FLAG_TRACE    record the device time line of every tile's upload, compute and
 *                  download of the last flush (oc_trace).
 * OC_FLAG_MANAGED  (oc_init only) the Unified Memory variant of Sec. 5.4: dataset stores
 *                  are managed memory (cudaMallocManaged) that the kernels address in
 *                  place; the tile plan is the explicit pipeline's (same budget, tiles and
 *                  phases), but a tile's copies become prefetches of its rows to the GPU
 *                  (upload stream) and, after their last tile, back to the host (download
 *                  stream). Rows first written in the chain are prefetched too (their pages
 *                  must be on the GPU). No slabs, residency, speculative prefetch, chain
 *                  graphs or autotuning trials (a trial would change the data in place); the
 *                  planner uses the fixed rule. A chain that fits the budget is one tile and
 *                  keeps its pages on the GPU. */
/* Kernel launches: the kernels of a tile (and the reduction combine) are launched with
 * programmatic stream serialisation (sm_90+ programmatic dependent launch): each kernel may
 * be launched while its predecessor on the compute stream finishes, and waits for the
 * predecessor's completion before it touches memory, so results are unchanged. The
 * environment variable OC_PDL=0, read at oc_init, launches them plainly instead. */
#define OC_FLAG_CYCLIC   0x1u
#define OC_FLAG_PREFETCH 0x2u
#define OC_FLAG_GRAPHS   0x4u
#define OC_FLAG_DRYRUN   0x8u
#define OC_FLAG_PROFILE  0x10u
#define OC_FLAG_TRACE    0x20u
#define OC_FLAG_MANAGED  0x40u

/* ---- planner modes ----------------------------------------------------------
 * OC_PLAN_FIXED     largest tile height whose plan fits the budget, depth 3, every
 *                   dataset streamed (Sec. 4: tiles sized by the fast memory alone).
 * OC_PLAN_AUTOTUNE  time every candidate of the grid on the first execution of a chain
 *                   shape and keep the fastest. A candidate is a residency level (share
 *                   of the budget for datasets kept whole in device memory across
 *                   chains: 0, 1/4, 1/2, 3/4), a depth 2..4 and a tile height (1, 3/4,
 *                   1/2 or 1/4 of the largest that fits with that residency and depth).
 * OC_PLAN_LEARNED   MLP prediction from chain features (oc_planner_load) of the gain of
 *                   two grid candidates over the fixed rule; falls back to AUTOTUNE when
 *                   no network is loaded or when a standardised feature of the chain lies
 *                   more than 4 training deviations from the training mean (a chain unlike
 *                   the training set).
 * Residency (an addition to the method: the paper streams every dataset of every
 * chain): a plan may keep some datasets whole in the device arena across chains, so that
 * their rows are neither uploaded nor downloaded per tile; the other datasets stream
 * through slabs sized from the rest of the budget. At a level L the datasets are taken
 * greedily by the link bytes one chain moves for them per byte they occupy, while their
 * total stays within L * budget. A resident dataset is uploaded once (with the first
 * chain that keeps it) and downloaded only when oc_fetch_dat asks for it or when a later
 * plan stops keeping it. */
#define OC_PLAN_FIXED    0
#define OC_PLAN_AUTOTUNE 1
#define OC_PLAN_LEARNED  2

/* ---- loop kernels (kernel_id of oc_enqueue_loop) ------------------------------
 * Every kernel is a pointwise function of its READ arguments sampled at their
 * stencil offsets; WRITE/RW arguments are accessed at offset 0 only. For every
 * point the result is evaluated in the order written below (IEEE round-to-nearest;
 * a multiply-add is fused only where stated), so two correct implementations differ
 * by at most the rounding of the fused steps; tiled and untiled executions of this
 * library agree bit for bit.
 *
 * OC_K_COPY     args: [0] WRITE dst (1 point, offset 0), [1] READ src (1 point).
 *               dst(p) = src(p + o).                               params: none.
 * OC_K_LINCOMB  args: [0] WRITE dst; [1..k] READ inputs, input j with n_j points.
 *               Let x_0..x_{M-1} be the samples in argument order, then point
 *               order (M = sum n_j). params = [alpha, c_0, ..., c_{M-1}].
 *               acc = c_0*x_0; acc = c_m*x_m + acc for m = 1..M-1 (this multiply-add
 *               may be fused: one rounding); if alpha != 0:
 *               acc = acc + ((alpha*a)*b) / (1 + c*c) with a = x_0,
 *               b = x_{1 mod M}, c = x_{2 mod M}. dst(p) = acc. FP32 datasets use
 *               the parameters rounded to float.
 * OC_K_REDUCE   args: [0] READ src0 (offset 0), optionally [1] READ src1 (offset 0),
 *               last: REDUCE handle. v = src0(p) (+ src1(p)); params = [mode]:
 *               0 -> v, 1 -> |v|, 2 -> v*v. The handle's operator folds v over the
 *               range into one FP64 partial per slow row and 4096-point chunk, in a
 *               fixed order (see oc_reduce). FP64 data fold in FP64. FP32 data fold
 *               without FP64 arithmetic per point: a sum is a compensated FP32 pair per
 *               thread and warp (TwoSum; a square enters as its exact FMA split),
 *               within ~1e-13 of sum |terms| of the exact sum; extremes are exact; a
 *               two-source |v|, square or extreme folds in FP64 (hi + lo exact there);
 *               a block whose FP32 sum overflows folds again in FP64.
 * OC_K_HILO_ADD args: [0] RW hi (F32), [1] RW lo (F32), [2] READ du (offset 0).
 *               params = [scale]. Compensated update of the pair value hi+lo by
 *               y = (float)scale * du, all in FP32: s = hi + y; z = s - hi;
 *               e = (hi - (s - z)) + (y - z); l = lo + e; hi' = s + l;
 *               lo' = l - (hi' - s).   (TwoSum followed by Fast2Sum.)
 * The Euler (OC_K_EULER_*) and Navier-Stokes (OC_K_NS_*) kernels are declared in
 * oc_physics.h.
 */
#define OC_K_COPY     1
#define OC_K_LINCOMB  2
#define OC_K_REDUCE   3
#define OC_K_HILO_ADD 4

/* One loop argument (Sec. 3: dataset + stencil + access mode). For OC_REDUCE,
 * `dat` is a reduction handle and npoints/offsets are ignored. `offsets` holds
 * npoints * ndim ints (x, y[, z] per point); it is copied at enqueue time. */
typedef struct oc_arg {
    int dat;
    int access;
    int npoints;
    const int* offsets;
} oc_arg;

/* Counters of the last flush and running totals (all chains since oc_init). */
typedef struct oc_stats_t {
    double seconds;        /* host wall time of the last flush, copies included      */
    double cell_updates;   /* sum over executed loops of their range points          */
    double hbm_bytes;      /* algorithmic bytes (Sec. 5.1: 1x read or write, 2x RW)  */
    double h2d_bytes;      /* bytes uploaded host -> device in the last flush        */
    double d2h_bytes;      /* bytes downloaded device -> host in the last flush      */
    double prefetched_bytes; /* bytes of the last flush's uploads already prefetched */
    int    tiles;          /* tiles of the last flush (1 = in-core)                  */
    int    tile_height;    /* slow-axis rows per tile chosen by the planner          */
    int    depth;          /* pipeline depth used (2..4)                             */
    int    loops;          /* loops in the last chain                                */
    int    graph_replays;  /* tiles of the last flush replayed from a CUDA graph     */
    int    kernel_launches;/* kernels the last flush launched (graph nodes included) */
    double total_seconds, total_cell_updates, total_hbm_bytes, total_h2d_bytes,
           total_d2h_bytes;
    long long chains;
    int    resident_dats;  /* datasets the last flush's plan keeps resident (streamed    */
    int    pad_;           /* plans; see oc_set_residency)                              */
    double resident_bytes; /* bytes of those datasets in the device arena               */
    double total_kernel_launches; /* kernels launched by all flushes since oc_init      */
} oc_stats_t;

/* Create the context. Sec. 4: all tiles live inside a device budget.
 *  device_budget_bytes  bytes of device memory the executor may use for dataset
 *                       slabs and reduction scratch (the "fast memory" size).
 *  device_arena         caller-owned device allocation of arena_bytes >= budget
 *                       (e.g. a torch uint8 tensor); the library never frees it.
 *                       NULL with arena_bytes == 0: the library allocates the
 *                       budget itself and frees it in oc_finalize.
 *  streams              three cudaStream_t handles (upload, compute, download) owned
 *                       by the caller, or NULL: the library creates its own. The
 *                       library also creates one more compute stream of its own, on
 *                       which loops of a tile that are independent of their
 *                       neighbours run concurrently; every tile's work is joined back
 *                       into the compute stream before anything else waits on it.
 *  flags                OC_FLAG_* bits.  planner_mode: OC_PLAN_*.
 * Errors: OC_ERR_STATE if a context exists; OC_ERR_ARG on an arena smaller than
 * the budget, arena_bytes without an arena, or an unknown planner mode; OC_ERR_CUDA if
 * the device cannot be used (not with OC_FLAG_DRYRUN). */
int oc_init(size_t device_budget_bytes, void* device_arena, size_t arena_bytes,
            void* const streams[3], uint32_t flags, int planner_mode);

/* Flush nothing, release every resource (pinned host stores, graphs, events,
 * library-owned streams and arena). Pending chains are discarded. */
int oc_finalize(void);

/* Declare a dataset (Sec. 3 "datasets"; data is handed to the library, Sec. 3).
 *  ndim 2 or 3; size = interior extent; halo_lo/halo_hi = halo depth per axis.
 *  dtype OC_F64 or OC_F32. host_init: dense array of the full extent (see top)
 *  copied into a library-owned pinned host store, or NULL for zeros.
 *  periodic_mask bit a: axis a is periodic. A periodic non-slow axis must have zero
 *  halo (kernels that support it wrap indices); a periodic slow axis has its halo
 *  layers refreshed from the opposite end at the start of every chain ("deep
 *  ghosts": a halo row y takes interior row y mod n), so loops may iterate into
 *  them.  *dat_out receives the handle. */
int oc_decl_dat(int ndim, const int size[3], const int halo_lo[3], const int halo_hi[3],
                int dtype, const void* host_init, int periodic_mask, int* dat_out);

/* Declare a reduction handle with operator OC_SUM / OC_MAX / OC_MIN. Its value is
 * folded over every loop of a chain that names it; a chain that names it again
 * after its value was read starts from the operator's identity. */
int oc_decl_reduction(int op, int* red_out);

/* Queue a loop (Sec. 3 parallel loop; lazy, nothing executes). range_lo/range_hi:
 * half-open iteration range per axis (ndim taken from the first dataset argument).
 * Validated now: dataset handles, access modes, a WRITE/RW argument must use exactly
 * the single offset 0, a dataset written by the loop may not also be read at a
 * non-zero offset, and every access must stay inside the allocated extent
 * (non-slow periodic axes excepted). Errors: OC_ERR_ARG. */
int oc_enqueue_loop(int kernel_id, const int range_lo[3], const int range_hi[3],
                    int nargs, const oc_arg* args, const double* params, int nparams);

/* Execute the queued chain (Sec. 3: a call returning data ends the chain; Sec. 4
 * Algorithm 1 streams its tiles). Returns when every result is in host memory.
 * Every host wait on the device (here, in oc_reduce and in oc_fetch_dat) is bounded:
 * 600 s, or the number of seconds in the environment variable OC_TIMEOUT_S when
 * oc_init ran. On expiry the call returns OC_ERR_TIMEOUT with the device work still
 * queued; the context is then in an unknown state and should be finalized. */
int oc_flush(void);

/* Flush, then return the value of reduction `red` of the last chain that named it. */
int oc_reduce(int red, double* out);

/* Flush, then copy dataset `dat` (full extent, dense, see top) into host_out. The halo
 * rows of a periodic slow axis are returned as the periodic images of the interior (halo
 * row y holds interior row y mod n), the state every chain starts from. */
int oc_fetch_dat(int dat, void* host_out);

/* Switch a OC_FLAG_CYCLIC / PREFETCH / GRAPHS bit on or off between chains (Sec. 4.1:
 * the cyclic flag is set by the user once the cyclic phase of the run begins). */
int oc_set_flag(uint32_t flag, int on);

/* Override the planner: tile height in slow-axis rows (0 = planner decides) and
 * pipeline depth 2..4 (0 = planner decides). Depth d uploads tile t+d-2 while tile t
 * computes and tile t-1 downloads. */
int oc_set_tiling(int tile_height, int depth);

/* Override the planner's residency level for streamed chains: the share of the budget
 * (0 <= level < 1) given to datasets kept resident across chains (see the planner modes
 * above); a negative level hands the choice back to the planner (OC_PLAN_FIXED: 0).
 * Errors: OC_ERR_ARG for level >= 1. */
int oc_set_residency(double level);

/* Copy the counters into *out. */
int oc_stats(oc_stats_t* out);

/* Per-kernel device time measured with OC_FLAG_PROFILE (accumulated until reset):
 * ms = event time of the kernel's launch runs (the gaps between launches of one run
 * included), launches = their count, bytes = algorithmic bytes of the launches (Sec. 5.1
 * formula: every dataset argument moves its range once, twice if read-write),
 * points = range points. */
typedef struct oc_kernel_stats_t {
    long long launches;
    double ms;
    double bytes;
    double points;
} oc_kernel_stats_t;
int oc_kernel_stats(int kernel_id, oc_kernel_stats_t* out);
int oc_kernel_stats_reset(void);

/* Time line of the last flush under OC_FLAG_TRACE: one record per tile and phase kind
 * (0 upload on stream 1, 1 compute on stream 0, 2 download on stream 2), with device
 * times in ms relative to the start of the flush and the bytes moved (uploads and
 * downloads). *n receives the number of records; at most cap are written. */
typedef struct oc_trace_rec {
    int tile;
    int kind;
    double start_ms;
    double end_ms;
    double bytes;
} oc_trace_rec;
int oc_trace(oc_trace_rec* out, int cap, int* n);

/* Host-side fault injection, for testing error paths without a device fault. Arms a
 * one-shot failure at `site` (0: a host-to-device row copy, 1: a device-to-host row copy,
 * 2: a kernel launch of a tile): the next `after` calls at that site proceed, and the one
 * after them returns OC_ERR_CUDA ("injected fault: ...") from the running call (oc_flush,
 * oc_reduce, oc_fetch_dat) without calling CUDA. Work queued before it still runs; the
 * chain is abandoned and the context should be finalized, as after any OC_ERR_CUDA.
 * after < 0 disarms the site. Errors: OC_ERR_STATE without a context, OC_ERR_ARG on an
 * unknown site. */
int oc_inject_fault(int site, long long after);

/* NUMA placement, for reading host-link measurements: *store_node receives the host
 * NUMA node of the first page of dataset `dat`'s pinned host store (-1 if unknown or not
 * allocated), *gpu_host_node the host node closest to the current device
 * (cudaDevAttrHostNumaId; -1 if the system reports none). Errors: OC_ERR_STATE without a
 * context, OC_ERR_ARG on a bad handle or null pointer. */
int oc_numa_nodes(int dat, int* store_node, int* gpu_host_node);

/* Message of the last error (static storage, valid until the next call). */
const char* oc_last_error(void);

/* ---- plan inspection (Sec. 3 skewed tiling, Sec. 4 footprints) -----------------
 * Describe the plan of the most recent flush (also in OC_FLAG_DRYRUN mode).
 * oc_plan_shape: number of tiles, loops, datasets used by the chain, tile height,
 *   depth, and the number of slow-axis rows spanned by the loop ranges.
 * oc_plan_ranges: se[(t*nloops + i)*2 + {0,1}] = half-open slow-axis range [s, e)
 *   of loop i in tile t (s == e: loop i does nothing in tile t).
 * oc_plan_dat: k-th dataset of the chain (0 <= k < ndats): its handle, slab rows S
 *   (rows are stored at slot (y - y_first) mod S; S = all rows when in-core), and
 *   the row intervals copied per tile, five ints each: up[5*j] = tile,
 *   up[5*j+1..2] = slow rows [a, b), up[5*j+3..4] = [x0, x1): x0 == x1 means whole
 *   rows; x0 < x1 means the rows are first written over x in [x0, x1) (Sec. 4.1
 *   "write-first") and only the columns outside it are uploaded; j < *nup (likewise
 *   down, always whole rows). Capacities cap_up / cap_down count intervals; if too
 *   small OC_ERR_ARG is returned and *nup / *ndown hold the required counts. */
int oc_plan_shape(int* ntiles, int* nloops, int* ndats, int* tile_height, int* depth,
                  int* slow_rows);
int oc_plan_ranges(int* se);
int oc_plan_dat(int k, int* dat, int* slab_rows, int* up, int cap_up, int* nup,
                int* down, int cap_down, int* ndown);

/* ---- tile planner (an addition to the method: the paper sizes tiles by the fast-memory
 * size only, Sec. 4) ----------------------------------------------------------------
 * Features of a chain, 8 floats: log2(loops), datasets used, slow-axis stencil radius,
 * bytes per cell, budget / footprint, dimensions, log2(footprint bytes), log2(slow rows).
 * oc_planner_features: features of the most recently planned chain.
 * oc_autotune_result: the table of the last autotuned chain (OC_PLAN_AUTOTUNE, or
 *   OC_PLAN_LEARNED without a network), 6 doubles per candidate: tile height, depth,
 *   device ms of the chain (median of 3 interleaved rounds), grid index (height =
 *   round(hmax * {1, 3/4, 1/2, 1/4}[index])), hmax (largest fitting height at that
 *   depth and residency), residency level. *n = rows.
 * oc_planner_load: install the network used by OC_PLAN_LEARNED: oc_mlp_nparams() floats
 *   and the features' standardisation (x - mean) / std. The network is a cost model of two
 *   alternatives A0, A1 to the fixed rule (hmax, depth 3, nothing resident): y_k = log2 of
 *   the time ratio t(fixed) / t(A_k). The planner keeps the fixed rule unless
 *   max(y0, y1) > 0.03, else takes the alternative with the larger predicted gain.
 *   Applies to chains planned afterwards, in this and later contexts of the process (it
 *   needs no context).
 * oc_planner_alternatives: name A0 and A1 as three ints each -- grid index (0..3),
 *   depth (2..4), residency level index (0: none, 1: 1/4, 2: 1/2, 3: 3/4 of the budget).
 *   Default {0, 3, 1} and {0, 3, 2}. Errors: OC_ERR_ARG outside the grid.
 * oc_mlp_*: the 8-64-64-2 ReLU network in FP32 on the GPU (host pointers; row-major
 *   X[n][8], Y/T[n][2]); parameter layout W1[64][8] b1[64] W2[64][64] b2[64] W3[2][64]
 *   b3[2]; loss = sum (y - t)^2 / (2n). oc_mlp_train runs `epochs` full-batch Adam steps
 *   (beta 0.9 / 0.999, eps 1e-8) in place on params; loss_hist (or NULL) gets the loss
 *   before each step. These calls need no context. */
int oc_planner_features(float* out8);
int oc_autotune_result(double* table, int cap, int* n);
int oc_planner_load(const float* params, int nparams, const float* feat_mean, const float* feat_std);
int oc_planner_alternatives(const int* alt6);
int oc_mlp_nparams(void);
int oc_mlp_forward(const float* params, const float* X, int n, float* Y);
int oc_mlp_loss_grad(const float* params, const float* X, const float* T, int n, float* grad, double* loss);
int oc_mlp_train(float* params, const float* X, const float* T, int n, int epochs, float lr, float* loss_hist);

/* ---- reduction for callers that cannot allocate ----------------------------------
 * The paper has no counterpart: this entry point exists for callers that may not
 * allocate device memory (code running inside someone else's CUDA-graph capture, an
 * allocator-free real-time or safety-critical component, a process whose memory pool
 * must not grow). It folds a 2-D region of a device array exactly as an OC_K_REDUCE
 * loop over the same values does (same per-row, per-4096-point partials, same fixed
 * combine order, so the results are bit-identical), but keeps its scratch -- the
 * partials -- in one file-scope device array of 65536 doubles (512 KiB) that every GPU
 * loading the library holds until the process exits. No memory is allocated or freed.
 *  data      device pointer: rows x row_len elements, consecutive rows row_pitch
 *            elements apart (row_pitch >= row_len); dtype OC_F64 or OC_F32.
 *  op        OC_SUM / OC_MAX / OC_MIN; mode 0: value, 1: |value|, 2: value^2.
 *  out       device pointer to one double receiving the result.
 *  stream    cudaStream_t (NULL: the legacy default stream). The call only enqueues
 *            work; synchronise the stream before reading *out.
 * Requires rows * ceil(row_len / 4096) <= 65536 (e.g. 65536 rows of up to 4096 elements,
 * or 16 rows of 65536), else OC_ERR_ARG. The first call on a
 * device (with that device current) looks up the array's device address; make it
 * before any stream capture. Calls share the array: calls whose work overlaps on the
 * GPU (e.g. on two streams at once) race and must be ordered by the caller. Errors:
 * OC_ERR_ARG, OC_ERR_CUDA; the message is in oc_noalloc_last_error(). Needs no context. */
int oc_reduce_noalloc(const void* data, int dtype, int rows, int row_len, long long row_pitch, int op, int mode,
                      double* out, void* stream);
const char* oc_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* OC_H */
