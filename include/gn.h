/*
 * gn.h -- C ABI of the GB300 Graph Normalization library (libgn.so).
 *
 * Graph Normalization (arXiv 2605.05330) iterates the weighted regularised map
 * (Def. WRGN, Sec. 2)
 *
 *     x_i  <-  x_i / ( x_i + gamma * sum_{j in N(i)} (v_j / v_i) x_j ),   v = sqrt(w),
 *
 * on a sparse conflict graph until the state binarises into the indicator of a
 * maximal independent set (Thm. 4).  The library runs the iteration on the GPU in
 * the weighted state y = v (.) x (App. B: y_i <- v_i y_i / ((I + gamma A) y)_i), in
 * FP32, with FP64 reductions.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Status codes: 0 = success, > 0 = warning (results are written), < 0 = error
 *   (outputs are unspecified).  No call throws, traps the GPU or aborts the process.
 *   gn_last_error() returns a message for the last non-zero status of this thread.
 * - Memory side: every pointer argument after gn_create lives on the side selected by
 *   the handle's I/O mode (GN_HOST or GN_DEVICE; set at gn_create, changed with
 *   gn_set_io).  Device pointers must belong to the handle's device.
 * - Streams: all device work of a handle is issued on its stream (gn_create's
 *   `stream`, a cudaStream_t, NULL = legacy default stream).  Calls that return
 *   results to the host, or a status that depends on device results, synchronise
 *   that stream before returning.
 * - Ownership: gn_create copies the caller's arrays into handle-owned device memory;
 *   the caller keeps ownership of every buffer it passes to any call.
 * - Vertex ids are 0-based in the caller's order.  An internal reordering (params
 *   `reorder`) is undone on every output.
 * - A handle is not thread-safe; distinct handles may be used concurrently.
 */
#ifndef GN_H_
#define GN_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GN_OK = 0,
  GN_WARN_NOT_CONVERGED = 1,    /* max_iters reached before the stop test fired */
  GN_WARN_NOT_BINARY = 2,       /* residual below tol on a state that is not binary */
  GN_WARN_NOT_MAXIMAL = 3,      /* extracted set is independent but not maximal */
  GN_ERR_ARG = -1,              /* bad argument or malformed CSR encoding */
  GN_ERR_NOT_SIMPLE = -2,       /* self-loop, duplicate/unsorted row, or asymmetric A */
  GN_ERR_WEIGHT = -3,           /* a weight is <= 0 or not finite */
  GN_ERR_NOT_NORMALIZABLE = -4, /* x0 < 0, not finite, or (A + I) x0 has a zero entry */
  GN_ERR_CUDA = -5,             /* a CUDA runtime call failed */
  GN_ERR_TIMEOUT = -6,          /* a device-side wait hit its limit; kernel returned early */
  GN_ERR_NOT_INDEPENDENT = -7,  /* the rounded set has an edge inside */
  GN_ERR_NO_RECORD = -8,        /* gn_backward without a recorded forward run */
  GN_ERR_TOO_LARGE = -9         /* size beyond a documented limit */
} gn_status;

#define GN_HOST 0
#define GN_DEVICE 1

#define GN_GAMMA_PURSUIT 0      /* gamma_k = t gamma1 + (1-t) gamma0, t = min(k,T-1)/(T-1) (Sec. 6) */
#define GN_GAMMA_FIXED 1        /* gamma_k = gamma1 */

#define GN_REORDER_NONE 0
#define GN_REORDER_RCM 1        /* reverse Cuthill-McKee: locality of neighbour gathers */
#define GN_REORDER_DEGREE 2     /* descending degree */

#define GN_SYNC_AUTO 0          /* halo mode: GN_SYNC_TAGGED; other modes: GN_SYNC_GRID */
#define GN_SYNC_GRID 1          /* a grid-wide barrier after every iteration */
#define GN_SYNC_NEIGHBOUR 2     /* halo mode: each CTA waits only for the CTAs whose rows it reads
                                   (per-CTA completed-iteration flags); grid-wide only at the stop
                                   test.  Same arithmetic, bit-identical results. */
#define GN_SYNC_TAGGED 3        /* halo mode: every exchanged value carries a one-bit tag of its
                                   iteration (three rotating buffers); a CTA polls its halo values
                                   until their tags are the iteration's, with no barrier between
                                   stop tests.  Same arithmetic, bit-identical results. */

#define GN_KERNEL_AUTO 0
#define GN_KERNEL_PERSISTENT 1  /* multi-CTA persistent kernel with a bounded grid barrier */
#define GN_KERNEL_CTA 2         /* whole graph in one CTA's shared memory (small graphs, up to
                                   16384 vertices; no grid barrier).  A run from start_iter 0,
                                   without record or resume; arithmetic of the global-gather
                                   mode.  GN_KERNEL_AUTO is the persistent kernel. */

typedef struct {
  int gamma_mode;       /* GN_GAMMA_PURSUIT (default) or GN_GAMMA_FIXED */
  double gamma0;        /* pursuit start (default 0.9, Sec. 6) */
  double gamma1;        /* pursuit end / fixed value (default 1.5, Sec. 6) */
  int ramp_iters;       /* pursuit length T (default 1000, Sec. 6) */
  int check_every;      /* stop-test cadence c >= 1 (default 10) */
  double theta_bin;     /* binarity threshold theta (default 1e-4) */
  int kernel;           /* GN_KERNEL_* (default AUTO) */
  int record;           /* 1: differentiable run for gn_backward: exactly max_iters - start_iter
                           steps (no stop test) through step kernels that keep a checkpoint
                           every ceil(sqrt(T)) steps */
  long long spin_limit; /* device wait limit in polls (0 = default 1<<22) */
  int debug_unreachable_barrier; /* test hook, must be 0 in use.  1: make the first grid
                                    barrier unreachable so that every CTA hits spin_limit.
                                    2: under GN_SYNC_TAGGED, the first halo wait expects a tag
                                    that no value carries (other modes: as 1) */
  int resume;           /* 1: continue from the full-precision state the last gn_run left on the
                           handle (x0 ignored); with start_iter = that run's end this reproduces
                           an uninterrupted run bit for bit */
  int sync;             /* GN_SYNC_* (default AUTO); other gather modes always use GRID */
} gn_params;

typedef struct {
  int iters;            /* iterations performed by this call */
  int converged;        /* 1 if the stop test fired */
  int binary;           /* 1 if every x_i <= theta or >= 1 - theta at the last check */
  int status;           /* the gn_status returned */
  double resid_inf;     /* max_i |x_i^{k+1} - x_i^k| of the last step */
  double resid_l1;      /* sum_i |x_i^{k+1} - x_i^k| of the last step (FP64) */
  double objective;     /* sum_i w_i x_i of the returned state (FP64), Thm. 3 */
  double energy;        /* E~(y) = 1/2 y^T (I + gamma A) y - v^T y (Sec. 3) of the state that
                           entered the last step, at that step's gamma (FP64) */
  long long safe_div_hits; /* steps where (B y)_i <= 1e-9 set x_i = 1/2 (appendix module) */
  float device_ms;      /* device time of the iteration kernel(s) */
  int kernel;           /* kernel that ran (GN_KERNEL_PERSISTENT or GN_KERNEL_CTA) */
} gn_run_info;

typedef struct gn_graph gn_graph;

/* Fills *p with the defaults listed in gn_params. */
void gn_default_params(gn_params* p);

/*
 * gn_create -- a1 of the path: validate, upload and prepare a graph.  Sec. 2: A must be
 * the adjacency matrix of a simple undirected graph (symmetric, zero diagonal); Def. WRGN:
 * w in R_{++}^n, v = sqrt(w).
 *   n        number of vertices, 0 <= n < 2^31 - 1
 *   row_ptr  int32[n+1], row_ptr[0] = 0, non-decreasing; nnz = row_ptr[n] directed entries
 *   col_idx  int32[nnz]; row i lists N(i) strictly increasing, no i itself; j in N(i)
 *            iff i in N(j)
 *   w        float32[n], finite and > 0
 *   mem      GN_HOST or GN_DEVICE: where row_ptr/col_idx/w live; becomes the I/O mode
 *   reorder  GN_REORDER_*: internal vertex order (undone on output)
 *   stream   cudaStream_t for all device work of the handle (NULL = default stream)
 * On success *g owns device copies of everything.  Errors: GN_ERR_ARG, GN_ERR_NOT_SIMPLE,
 * GN_ERR_WEIGHT, GN_ERR_CUDA (no handle is returned on error).
 */
gn_status gn_create(gn_graph** g, int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                    const float* w, int mem, int reorder, void* stream);

#define GN_GATHER_AUTO 0      /* the fastest mode that fits (halo, else CSR in smem, else global) */
#define GN_GATHER_GLOBAL 1    /* neighbour ids and values read through L1/L2 */
#define GN_GATHER_SMEM_CSR 2  /* each CTA's neighbour ids in shared memory, values through L1/L2 */
#define GN_GATHER_HALO 3      /* each CTA's distinct external neighbours staged in shared memory,
                                 exchanged by pull or push as the halo density suggests */
#define GN_GATHER_HALO_PULL 4 /* halo mode, pull exchange (each halo value read from its owner's
                                 slot) */
#define GN_GATHER_HALO_PUSH 5 /* halo mode, push exchange (owners write per-consumer inboxes that
                                 the consumer reads) */

typedef struct {
  int reorder;          /* GN_REORDER_* */
  int gather;           /* GN_GATHER_*; a forced mode that does not fit gives GN_ERR_TOO_LARGE */
} gn_create_opts;

/* gn_create with options (NULL = reorder none, gather auto).  Same contract as gn_create. */
gn_status gn_create_ex(gn_graph** g, int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                       const float* w, int mem, const gn_create_opts* opts, void* stream);

/* Gather mode the handle's persistent kernel uses (GN_GATHER_GLOBAL, _SMEM_CSR or _HALO). */
int gn_gather_mode(const gn_graph* g);

/* Halo exchange of a GN_GATHER_HALO handle: 1 pull, 2 push; 0 for other modes or NULL. */
int gn_halo_exchange(const gn_graph* g);

/* Releases every resource of the handle (NULL is a no-op). */
void gn_destroy(gn_graph* g);

/* Changes the memory side (GN_HOST / GN_DEVICE) of the pointers of later calls. */
gn_status gn_set_io(gn_graph* g, int mem);

/*
 * gn_set_weights -- replaces the vertex weights w of Def. 3 (WRGN) on an existing handle, with
 * v = sqrt(w) recomputed as a float pair, so that a caller who changes only the weights (the
 * differentiable form's parameters, a sweep over weightings) pays neither validation of the
 * CSR nor reordering nor the per-CTA block build again.
 *   w   float32[n] in caller order, on the side of the handle's I/O mode; every entry must be
 *       finite and > 0
 * The handle's graph, vertex order and layout are unchanged.  Its recorded forward run (if
 * any), its resumable state and its CTA-kernel copy of the instance are dropped: gn_backward
 * then returns GN_ERR_NO_RECORD and a resume GN_ERR_ARG until the next run.  Errors:
 * GN_ERR_ARG, GN_ERR_WEIGHT (the old weights stay in place), GN_ERR_CUDA.
 */
gn_status gn_set_weights(gn_graph* g, const float* w);

/* Graph size queries. */
int32_t gn_num_vertices(const gn_graph* g);
int64_t gn_num_entries(const gn_graph* g);

/*
 * gn_vertex_order -- the handle's internal vertex order: order[r] = the caller's id of internal
 * vertex r (the identity for GN_REORDER_NONE).  GN_REORDER_RCM is the reverse Cuthill-McKee
 * order: each component is searched breadth-first from its unplaced vertex of least degree
 * (ties by id), the unplaced neighbours of each vertex follow in increasing degree (ties in
 * adjacency order), and the whole sequence is reversed.  GN_REORDER_DEGREE is descending degree,
 * ties by id.  Internal only: no output of the library depends on it beyond rounding order.
 *   order  int32[n] HOST buffer, written whatever the handle's I/O mode
 * Errors: GN_ERR_ARG (NULL handle or buffer), GN_ERR_CUDA.
 */
gn_status gn_vertex_order(const gn_graph* g, int32_t* order);

#define GN_ORDER_FROM_HOST 1    /* the order was computed on the host */
#define GN_ORDER_FROM_DEVICE 2  /* by the breadth-first search of one thread-block cluster on the
                                   device (RCM on graphs of >= 16,384 vertices and degrees <= 254
                                   whose levels fit its shared-memory buffers and level budget;
                                   the same order as the host's), renumbered there too */
/* Where the handle's internal order was computed: GN_ORDER_FROM_*, 0 without reordering or for
 * NULL. */
int gn_vertex_order_source(const gn_graph* g);

/*
 * gn_run -- a2..a7 of the path: iterated WRGN (Def. WRGN, Def. IGN) with the gamma
 * schedule of Sec. 6, from x0, until the stop test fires or the iteration index reaches
 * max_iters; then x_out = clamp(x, 0, 1) (appendix module).
 *   x0          float32[n] start (finite, >= 0, (A + I) x0 > 0 -- Def. 1), or NULL for
 *               x0_i = 1/(deg_i + 1)
 *   max_iters   absolute bound: iterations k = start_iter .. max_iters-1 run at most
 *   tol         residual stop: max_i |x_i^{k+1} - x_i^k| <= tol (negative disables)
 *   p           parameters (NULL = defaults)
 *   start_iter  absolute index of the first iteration (gamma_k depends on k); a run resumed
 *               with start_iter = K from a saved FP32 state x^K follows the uninterrupted one
 *               to within the FP32 rounding of x^K (params.resume continues bit for bit)
 *   x_out       float32[n] result (may alias x0); NULL leaves the state on the device only
 *   info        optional run summary
 * Stop test (after step k when (k+1) % check_every == 0 or k+1 == max_iters): every
 * x_i <= theta or >= 1-theta and gamma_k (1-theta) > theta (then the rounded set is
 * independent), or the residual test.  One launch of the persistent kernel runs all
 * iterations.  Returns GN_OK (binary), GN_WARN_NOT_BINARY, GN_WARN_NOT_CONVERGED, or an
 * error (GN_ERR_ARG, GN_ERR_NOT_NORMALIZABLE, GN_ERR_TIMEOUT, GN_ERR_CUDA).
 */
gn_status gn_run(gn_graph* g, const float* x0, int max_iters, double tol, const gn_params* p,
                 int start_iter, float* x_out, gn_run_info* info);

/*
 * gn_extract_is -- a8 of the path (Sec. 2 independent sets; Sec. 6 "valid MIS after
 * rounding"): S = {i : x_i > 1/2}; exact independence check over every edge; maximality
 * check; |S|; W(S) = sum_{i in S} w_i in FP64.
 *   x        float32[n] state (NULL = the state left by the last gn_run)
 *   mask     uint8[n] output, 1 for members (may be NULL)
 *   members  int32[n] output, member ids ascending (may be NULL)
 *   count    |S| (may be NULL); weight W(S) (may be NULL)
 * Returns GN_OK, GN_WARN_NOT_MAXIMAL, GN_ERR_NOT_INDEPENDENT (outputs still written), or an
 * error.
 */
gn_status gn_extract_is(gn_graph* g, const float* x, uint8_t* mask, int32_t* members,
                        int32_t* count, double* weight);

/*
 * gn_objective -- FP64 relaxed MWIS objective sum_i w_i x_i (Thm. 3) and the energy
 * E~(y) = 1/2 y^T (I + gamma A) y - v^T y, y = v (.) x (Sec. 3), of a state x (NULL = the
 * state left by the last gn_run).  Either output may be NULL.
 */
gn_status gn_objective(gn_graph* g, const float* x, double gamma, double* obj, double* energy);

/*
 * gn_backward -- reverse mode of the last recorded gn_run (params.record = 1: T fixed steps).
 * Derived from the step's Jacobian (App. G, Lemma 2 in its general form): with s = (I + gamma A) y
 * and x' = y / s, the adjoint of y' = v (.) x' is
 *   gbar_y = v (.) gbar' / s - (I + gamma A)(v (.) gbar' (.) y / s^2),
 *   gbar_v += gbar' (.) x',
 * chained through y_0 = v (.) x_0, x_T = y_T / v and v = sqrt(w).  Each segment between
 * checkpoints is recomputed, then reversed (two gathers per step).  Arithmetic is FP32.
 *   dL_dxT  float32[n] gradient of the loss w.r.t. the returned x (before the clamp, which
 *           is the identity on the iterates)
 *   dL_dw   float32[n] output, gradient w.r.t. w (may be NULL)
 *   dL_dx0  float32[n] output, gradient w.r.t. x0 (may be NULL)
 * Safe-division hits have zero gradient.  Errors: GN_ERR_NO_RECORD, GN_ERR_ARG, GN_ERR_CUDA.
 */
gn_status gn_backward(gn_graph* g, const float* dL_dxT, float* dL_dw, float* dL_dx0);

/*
 * gn_run_noalloc -- gn_run for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of the same persistent iteration kernel.
 *
 * Some callers are handed device buffers by a host runtime and may not call cudaMalloc
 * themselves (a plugin inside another framework's memory pool, a service that allocates
 * everything at start-up, work issued while the allocator is locked).  This entry point
 * allocates nothing: no cudaMalloc, no cudaFree, no handle.  All of the kernel's scratch
 * (the working states, v = sqrt(w) as a float pair, per-CTA check partials, the grid-barrier
 * counter, the run summary, the gamma schedule) lives in one fixed array of about 2 MB in
 * the library's device globals, which every GPU that loads the library holds until the
 * process exits.  The gamma pursuit may span at most 16384 table entries.
 *   n, row_ptr, col_idx, w   the graph, DEVICE pointers, same layout and rules as gn_create;
 *                            n <= 65536 (GN_ERR_TOO_LARGE beyond); row_ptr[n] is read on the
 *                            host, then the CSR is validated on the device (every row's range
 *                            within [0, row_ptr[n]] before its entries are read, order,
 *                            self-loops, symmetry, weights)
 *   x0, max_iters, tol, p, start_iter, info   as gn_run (DEVICE x0 or NULL); p->resume is
 *                            not available (GN_ERR_ARG)
 *   x_out                    float32[n] DEVICE output, written only when the call succeeds
 *                            (GN_OK or a warning); an error leaves it untouched
 *   stream                   cudaStream_t for all the work (NULL = default stream)
 * Results equal those of gn_run on a handle made with GN_GATHER_GLOBAL and GN_REORDER_NONE
 * (the same kernel and per-row summation order; only the split of rows over CTAs differs);
 * against gn_run's default (halo gather, RCM order) they agree within the per-vertex parity
 * tolerance.  Calls share the fixed array and leave their contents in it: calls whose device
 * work overlaps (several host threads or streams) race and must be serialised by the caller.
 * Every call reads row_ptr[n] and the run summary back to the host and synchronises the
 * stream, so it cannot be made while the stream is being captured into a CUDA graph.  The
 * first call on each device resolves the array's address with cudaGetSymbolAddress and sets a
 * kernel attribute.  Returns the same codes as gn_run, plus GN_ERR_ARG / GN_ERR_NOT_SIMPLE /
 * GN_ERR_WEIGHT for a bad graph.
 */
gn_status gn_run_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const float* w,
                         const float* x0, int max_iters, double tol, const gn_params* p,
                         int start_iter, float* x_out, gn_run_info* info, void* stream);

/* ==========================================================================================
 * Batched GN: many independent instances in one persistent launch (one CTA per instance at a
 * time from a work queue; each instance stops on its own stop test).  The iteration, schedule
 * and stop test are gn_run's.  The run sequence is captured into a CUDA graph and replayed.
 */
#define GN_INSTANCE_CSR 0         /* a general simple graph given as CSR with local ids */
#define GN_INSTANCE_ASSIGNMENT 1  /* the assignment conflict graph of a k x k matrix (Sec. 2: cells
                                     (r, c) adjacent when they share a row or a column), n = k*k,
                                     vertex r*k + c; no entries are passed: the neighbour sum is
                                     the row sum plus the column sum minus twice the cell */

typedef struct gn_batch gn_batch;

typedef struct {
  int iters;            /* iterations of this instance */
  int status;           /* GN_OK, GN_WARN_NOT_BINARY or GN_WARN_NOT_CONVERGED */
  int converged, binary;
  double resid_inf;     /* at the last check */
  double objective;     /* sum_i w_i x_i at the last check (float-pair sums, FP64 result) */
  long long safe_div_hits;
  double resid_l1;      /* sum_i |x_i' - x_i| at the last check */
  double energy;        /* E~ of the state entering the last check's step (Sec. 3) */
} gn_batch_info;

/*
 * gn_batch_create -- validate and upload `count` instances (each as in gn_create, n_i >= 1,
 * n_i <= 16384; assignment instances k <= 128).
 *   vtx_off  int64[count+1], prefix sums of n_i (w, x0, x_out, masks are concatenated by it)
 *   ent_off  int64[count+1], prefix sums of the instances' CSR entries (0 for assignment ones)
 *   row_ptr  int32[sum(n_i + 1)]: instance i's local row pointers start at vtx_off[i] + i
 *            (values of assignment instances are ignored; NULL when every instance is one)
 *   col_idx  int32[ent_off[count]] local neighbour ids (may be NULL when there are none)
 *   w        float32[vtx_off[count]] weights, > 0
 *   kind     int32[count] GN_INSTANCE_* (NULL = all CSR)
 *   mem      GN_HOST or GN_DEVICE for every pointer of this and later batch calls
 *   stream   cudaStream_t (NULL: the handle creates its own non-blocking stream)
 * Errors as gn_create (GN_ERR_TOO_LARGE when an instance exceeds shared memory).
 */
gn_status gn_batch_create(gn_batch** b, int32_t count, const int64_t* vtx_off, const int64_t* ent_off,
                          const int32_t* row_ptr, const int32_t* col_idx, const float* w,
                          const int32_t* kind, int mem, void* stream);
void gn_batch_destroy(gn_batch* b);

/* gn_run for every instance: x0 float32[vtx_off[count]] or NULL (1/(deg+1)); x_out may be NULL;
 * info gn_batch_info[count] may be NULL.  Returns the worst instance status (or an error). */
gn_status gn_batch_run(gn_batch* b, const float* x0, int max_iters, double tol, const gn_params* p,
                       float* x_out, gn_batch_info* info);

/* Device time (ms) of the last gn_batch_run's captured sequence. */
float gn_batch_last_ms(gn_batch* b);

/* CTA size of the batch kernel (128, 256, 512 or 1024). */
gn_status gn_batch_set_threads(gn_batch* b, int threads);

/* Instance packing: instances of at most warp_max_vertices vertices (0: none) that fit one warp's
 * share of the CTA's shared memory run a warp each, several per CTA, once the CTA-per-instance
 * queue is empty (same launch).  Iterates are bit-identical to CTA mode (same lanes per row, same
 * summation order).  gn_batch_packing reports the threshold and how many instances it moves. */
gn_status gn_batch_set_packing(gn_batch* b, int warp_max_vertices);
gn_status gn_batch_packing(const gn_batch* b, int* warp_max_vertices, int* warp_instances);

/* Autotuner: times the batch kernel for max_iters iterations (twice each) at every CTA size
 * {256, 512, 1024} crossed with every packing threshold {0, 64, 128, 256, 512} that moves a
 * different set of instances into warp mode, and keeps the fastest pair; *threads_out receives
 * the CTA size (may be NULL), gn_batch_packing the threshold. */
gn_status gn_batch_tune(gn_batch* b, const gn_params* p, int max_iters, int* threads_out);

/* gn_extract_is for every instance of the last run: mask uint8[vtx_off[count]], counts int32[count],
 * weights double[count] (FP64 W(S)), statuses int32[count]; any may be NULL.  Returns the worst
 * status (GN_ERR_NOT_INDEPENDENT if any instance's set has an inner edge). */
gn_status gn_batch_extract(gn_batch* b, uint8_t* mask, int32_t* counts, double* weights, int32_t* statuses);

/*
 * gn_random_start -- the random simplex start of the appendix module, for B starts at once:
 * p = -log u, p <- p / max(p) (one maximum over all m = B*n draws, as the module divides by the
 * maximum of the whole batch), x0 = clamp(p, 1e-3, 1).
 *   m    number of values (B * n)
 *   u    float32[m] DEVICE uniform draws in (0, 1] (the caller's generator)
 *   x0   float32[m] DEVICE output (may alias u)
 * Synchronous.  GN_ERR_ARG if a draw lies outside (0, 1].
 */
gn_status gn_random_start(int64_t m, const float* u, float* x0, void* stream);

/* ==========================================================================================
 * Learned warm start (the paper's warm-start idea, Sec. 6, with a predictor learned from GN's
 * own converged states; the network itself is not in the paper).  A 3-layer message-passing
 * network, hidden width 64, FP32 master weights rounded to bf16 for every pass, FP32
 * activations and accumulation:
 *   f_i = [log w_i, log(1+deg_i), mean_{N(i)} log w_j, max_{N(i)} log w_j]
 *   h^l_i = relu(W_s^l h^{l-1}_i + W_n^l mean_{j in N(i)} h^{l-1}_j + b^l)
 *   p_i = sigmoid(w_o . h^3_i + b_o),  x0_i = clamp(p_i, 1e-3, 1)
 *   loss = mean_i BCE(p_i, t_i) against a target state t (the rounded converged GN state).
 * Parameters are one FP32 vector of gn_mpnn_num_params() values in the order
 * [W_s^1 (64x4), W_n^1 (64x4), b^1, W_s^2 (64x64), W_n^2, b^2, W_s^3, W_n^3, b^3, w_o, b_o]
 * (row-major, output index first).
 */
typedef struct gn_mpnn gn_mpnn;

int gn_mpnn_num_params(void);
/* init_params: float32[gn_mpnn_num_params()] HOST initial weights; stream for all work. */
gn_status gn_mpnn_create(gn_mpnn** m, const float* init_params, void* stream);
void gn_mpnn_destroy(gn_mpnn* m);
/* Forward on a graph (its internal order): x0_out float32[n] DEVICE (caller order, may be NULL);
 * target float32[n] DEVICE caller order in {0,1} or NULL (inference); *loss HOST (may be NULL).
 * With a target, the activations are kept for gn_mpnn_backward. */
gn_status gn_mpnn_forward(gn_mpnn* m, const gn_graph* g, float* x0_out, const float* target, double* loss);
/* Inference: x0_out float32[n] DEVICE caller order = clamp((1/(deg+1))^(1-alpha) p^alpha, 1e-3, 1),
 * the prediction blended geometrically with the cold start (alpha in [0, 1]; 1 = prediction only).
 * Synchronous. */
gn_status gn_mpnn_predict(gn_mpnn* m, const gn_graph* g, float alpha, float* x0_out);
/* Adds the gradient of the last forward's loss to the gradient buffer (w.r.t. the bf16 weights). */
gn_status gn_mpnn_backward(gn_mpnn* m, const gn_graph* g);
gn_status gn_mpnn_zero_grad(gn_mpnn* m);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr; zeroes the gradients. */
gn_status gn_mpnn_step(gn_mpnn* m, float lr);
/* FP32 master weights / accumulated gradients to HOST float32[gn_mpnn_num_params()]. */
gn_status gn_mpnn_get_params(gn_mpnn* m, float* out);
gn_status gn_mpnn_get_grads(gn_mpnn* m, float* out);

/* Number of CUDA kernels this library has launched in the process so far (all handles,
 * all threads).  Lets a caller count the device work behind a sequence of calls. */
int64_t gn_kernel_launches(void);

/* Message of the last non-zero status returned on this thread ("" if none). */
const char* gn_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
