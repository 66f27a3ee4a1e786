/*
 * ocm.h -- C ABI of the GB300 optimal-cycle-mean solver.
 *
 * Problem (Barnat, Bauch, Brim, Ceska, "Computing Optimal Cycle Mean in
 * Parallel on CUDA", Sec. 2.1): for a digraph G = (V, E) with integer edge
 * weights w, the mean of a cycle C is w(C)/|C|.  The solver returns the
 * maximum (OCM_MAX) or minimum (OCM_MIN) cycle mean lambda* as an exact
 * reduced rational num/den, and a critical cycle attaining it.
 *
 * Method: Howard's policy iteration (Sec. 2.4, Alg. 1), decomposed into
 * data-parallel primitives as in Sec. 3 (Alg. 2): an improvement sweep over
 * the CSR edges (Alg. 2 SPFPassIter), cycle detection in the policy graph,
 * per-cycle means, and value propagation along policy edges (Alg. 3).  The
 * primitives here are hand-written sm_103a kernels of this library's own
 * design: pointer jumping replaces the paper's elimination / connectGpi /
 * valuePropagate fixpoints, and every policy cycle keeps its own exact mean
 * (multichain policy iteration) instead of rebuilding the policy graph around
 * one chosen cycle.  All arithmetic is integer, so results are bit-exact and
 * deterministic.
 *
 * Graph format (Sec. 2.3, Fig. 2b: arrays A_i and A_t): CSR with
 *   row_ptr[n+1]  int32, row_ptr[0] = 0, non-decreasing, row_ptr[n] = m;
 *   col_idx[m]    int32 targets, 0 <= col_idx[e] < n;
 *   w[m]          int32 weights, w[e] != INT32_MIN.
 * Edge e leaves vertex v iff row_ptr[v] <= e < row_ptr[v+1].  Every vertex
 * must have at least one out-edge.  Self-loops and parallel edges are allowed;
 * strong connectivity is NOT required (lambda* is then the optimum over all
 * cycles of G, as in Prop. 2.2).  Exactness bound: 2 * n^2 * max|w| < 2^62.
 *
 * Conventions for every entry point:
 *   - array pointers are CUDA device memory unless marked "host";
 *   - the caller owns all memory; the library allocates no device buffers
 *     and works only on the given stream (a cudaStream_t passed as void*,
 *     NULL = the legacy default stream); the entry points synchronise that
 *     stream and so must not be called while it is being captured;
 *   - the solve loop (evaluate the policy, improve it, stop when stable) is
 *     a CUDA graph with a conditional WHILE node whose body ends in a
 *     one-thread kernel that sets the loop condition: one graph launch and
 *     one synchronisation per solve.  The library instantiates that graph
 *     on first use and caches a few of them keyed by the arguments baked
 *     into it (device, array pointers, sizes, sense, launch shape); the
 *     driver-held graph resources are the only memory kept between calls;
 *   - on any error the outputs are left untouched and a negative OCM_ERR_*
 *     code is returned (ocm_status_string gives a message);
 *   - results are deterministic: the same input gives the same bits.
 */
#ifndef OCM_H_
#define OCM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define OCM_OK 0
#define OCM_ERR_INVALID_ARG (-1)   /* null pointer, n or m out of range, bad mode   */
#define OCM_ERR_BAD_CSR (-2)       /* row_ptr not monotone / wrong ends, col out of range */
#define OCM_ERR_NO_OUT_EDGE (-3)   /* a vertex has no out-edge                      */
#define OCM_ERR_OVERFLOW (-4)      /* w = INT32_MIN, or 2 n^2 max|w| >= 2^62         */
#define OCM_ERR_NOT_CONVERGED (-5) /* iteration cap reached                         */
#define OCM_ERR_TIMEOUT (-6)       /* a bounded device-side wait gave up            */
#define OCM_ERR_WORKSPACE (-7)     /* workspace missing, too small or misaligned    */
#define OCM_ERR_CUDA (-8)          /* a CUDA runtime call failed                    */
#define OCM_ERR_INTERNAL (-9)      /* an internal consistency check failed          */

/* optimisation sense */
#define OCM_MAX 0
#define OCM_MIN 1

/* Optional inputs/outputs of ocm_solve.  Zero-initialise, then set fields.
 * The per-vertex outputs describe the final policy in the MAXIMISING sense of
 * s*w, s = +1 for OCM_MAX and -1 for OCM_MIN: eta_num[v]/eta_den[v] is the
 * (reduced) mean of the policy cycle that v reaches, and potential[v] is the
 * value V(v) = eta_den[v] * (s*w-weight of v's policy path to that cycle's
 * smallest vertex) - eta_num[v] * (its length).  Together they certify
 * optimality as the LP dual of Eq. (1): for every edge e = (v, t),
 * eta(t) <= eta(v), and when equal, q*s*w(e) - p + V(t) - V(v) <= 0.       */
typedef struct ocm_options {
    int32_t max_iters;   /* improvement steps before OCM_ERR_NOT_CONVERGED; <= 0: 4n + 64 */
    int32_t flags;       /* OCM_FLAG_* bits; 0 for normal use                       */
    int64_t *eta_num;    /* optional device [n]                                     */
    int32_t *eta_den;    /* optional device [n]                                     */
    int64_t *potential;  /* optional device [n]                                     */
    int32_t *policy;     /* optional device [n]: final policy edge of each vertex   */
    /* Launch tuning of the improvement sweep (0 = library default: 8 edges
     * per lane, 512 threads; the Python package has an autotuner):
     * edges_per_lane as described under OCM_SWEEP_* below, sweep_threads the
     * sweep's block size (64 to 512, see there).  Results do not depend on
     * these.                                                                 */
    int32_t edges_per_lane;
    int32_t sweep_threads;
    int32_t sweep_kind;  /* OCM_SWEEP_*; 0 = library default (see there)           */
    /* Limit of every device-side wait of the call (the grid barriers of the
     * cooperative kernels), in milliseconds of GPU wall-clock time; a wait
     * that runs out makes the call return OCM_ERR_TIMEOUT and leaves the
     * device context usable.  <= 0: 2,000 ms (10 ms with OCM_FLAG_TEST_STALL).
     * The SCC decomposition of ocm_scc / ocm_solve_scc keeps the default. */
    int32_t wait_limit_ms;
    /* Warm start (optional, device [n]; [N] with global edge ids for
     * ocm_solve_batch): the policy the iteration starts from, one out-edge
     * per vertex, row_ptr[v] <= init_policy[v] < row_ptr[v+1]
     * (OCM_ERR_INVALID_ARG otherwise).  NULL = the first pass of Alg. 1
     * from val = 0, lambda = 0 (heaviest out-edge).  Policy iteration reaches
     * an optimal policy from any start (Sec. 2.4), so lambda* does not
     * depend on it; the number of iterations does, and where several cycles
     * are optimal, so may the returned one.  Passing the final policy of an
     * earlier solve (the `policy` output) resumes from it: re-solving after
     * a small weight change typically takes a few iterations.             */
    const int32_t *init_policy;
    /* Optimal cycle ratio (optional, device [m]; [M] for ocm_solve_batch):
     * a transit time t(e) >= 1 per edge (OCM_ERR_INVALID_ARG otherwise), the
     * "time" label of a transition next to its cost w (Sec. 2.2).  The solve
     * then returns the maximum (minimum) over cycles C of w(C)/t(C) as
     * num/den and a cycle attaining it; t = 1 everywhere gives the mean.
     * The per-vertex outputs are the ratio of the reached cycle and the
     * value V(v) = eta_den[v] * (s*w-weight of v's path to the cycle's
     * smallest vertex) - eta_num[v] * (its transit time).  Exactness bound:
     * 4 n^2 max|w| max t < 2^62 and n max t < 2^31 (OCM_ERR_OVERFLOW).  The
     * improvement sweep always uses OCM_SWEEP_CLASSES in this mode.         */
    const int32_t *transit;
    /* ocm_solve_batch only: graphs with at most this many vertices (and at
     * most 16 times as many edges) are solved by a persistent kernel in which
     * one thread block runs every iteration of one graph, blocks taking the
     * graphs largest first from a queue; the larger graphs are solved
     * together as one disjoint union afterwards.  0 = automatic: every graph
     * with at most max(4,096, 4 N / B) vertices, B the number of resident
     * blocks of that kernel (152 on a GB300), so that only graphs large next
     * to the batch's share per block take the union path; < 0 = every graph
     * takes the union path.  Results do not depend on it.  Not used with
     * transit times or per-vertex outputs (every graph then takes the union
     * path).                                                                */
    int32_t batch_small_vertices;
    int32_t reserved1;
} ocm_options;

/* Layouts of the improvement sweep (results do not depend on the choice).
 * In both, the initial pass, and in OCM_SWEEP_CLASSES the sweep itself, treat
 * a vertex with more than 1,024 out-edges as heavy: the heavy vertices' edges
 * are cut into chunks of 1,024, one thread block per chunk, and the chunks'
 * best candidates are combined per vertex, so a hub of millions of edges
 * costs no more than the same number of edges spread over many vertices.
 * OCM_SWEEP_TILES: the CSR edge array is cut into aligned tiles of 32 *
 *   edges_per_lane edges (edges_per_lane 4 or 8; default 8), one warp per
 *   tile, each lane scanning consecutive edges; vertices crossing lanes or
 *   tiles are joined by a segmented scan and a fix-up pass.  Blocks of 64,
 *   128 or 256 threads (512 runs as 256).
 * OCM_SWEEP_CLASSES: vertices grouped by degree class; a vertex of out-degree
 *   d is served by the smallest power-of-two lane group g <= 32 with
 *   d <= edges_per_lane * g (edges_per_lane 1..64; default 8).  On graphs
 *   of more than 2^22 vertices the grid takes the classes band by band (2^18
 *   consecutive vertices at a time), so the target records a band's edges
 *   gather stay in L2 between the class passes.
 * OCM_SWEEP_WINDOW: for graphs whose edges mostly point near their source in
 *   vertex order.  One thread block per SM walks a contiguous chunk of
 *   vertices in tiles of 2,048; bulk copies keep the records of a window of
 *   10,240 vertices around the tile in shared memory (the window starts hb
 *   vertices before the tile, hb in {0, 2048, ..., 8192} chosen by the
 *   initial pass as the placement holding most edges), and targets inside
 *   it are read from there.  Inside a tile vertices are grouped by degree
 *   class as in OCM_SWEEP_CLASSES (edges_per_lane likewise; sweep_threads is
 *   not used).  Not for the cycle ratio (OCM_SWEEP_CLASSES then).  On the
 *   2^25-vertex locality graph it runs slower than OCM_SWEEP_CLASSES (fewer
 *   warps in flight per SM), so it is never chosen by default.
 * OCM_SWEEP_DEFAULT is OCM_SWEEP_CLASSES; ocm_stats.sweep_kind reports the
 *   layout used.                                                           */
#define OCM_SWEEP_DEFAULT 0
#define OCM_SWEEP_CLASSES 1
#define OCM_SWEEP_TILES 2
#define OCM_SWEEP_WINDOW 3

/* Test-only: the first grid barrier of the evaluation waits for an arrival
 * that never comes, with its wait limit cut to 10 ms (or to
 * ocm_options.wait_limit_ms when set), so the solve exercises the
 * bounded-wait path and returns OCM_ERR_TIMEOUT.  The device context stays
 * usable.
 *
 * Test hook of the error paths (no GPU fault is made): when the environment
 * variable OCM_FAULT is "launch", the solve entry points return OCM_ERR_CUDA
 * before their first launch; "validate" makes ocm_solve, ocm_solve_batch and
 * ocm_solve_static return OCM_ERR_BAD_CSR as if the CSR checks had failed,
 * also before any device work; "alloc" makes the CUDA-graph loop fail to
 * instantiate, so the solve runs the host-driven loop (same results,
 * ocm_stats.graph_loop = 0).  Unset in normal use. */
#define OCM_FLAG_TEST_STALL 1

/* Drive the policy iteration from the host: after every improvement step the
 * host reads the control block (one stream synchronisation per step) and
 * decides whether to go on.  Without this flag the loop runs as a CUDA graph
 * (below); the results are the same bits either way.  Implied while the
 * benchmark instrumentation is enabled and by ocm_solve_static. */
#define OCM_FLAG_HOST_LOOP 2

/* The paper's own form of the iteration (Alg. 1 as written, Alg. 2's
 * markMinComponent / connectGpi / valuePropagate), for comparison with the
 * default multichain form: after every evaluation the policy cycle of largest
 * mean (ties: smallest root) is kept with its whole policy component, and
 * every other vertex is re-pointed, one backward breadth-first level at a
 * time, to its smallest-index out-edge into the vertices connected at earlier
 * levels; all values then refer to that one cycle's mean.  Needs every vertex
 * to reach the chosen cycle, which holds for strongly connected graphs
 * (OCM_ERR_INVALID_ARG otherwise), and the larger workspace
 * ocm_workspace_size_single(n, m) (the transposed graph and the search
 * frontiers).  ocm_solve only (not the batch).  lambda* is the same; the
 * iteration count, and where several cycles are optimal the returned cycle,
 * may differ from the default form's. */
#define OCM_FLAG_SINGLE_LAMBDA 4

/* Choice of the policy evaluation (results are the same bits either way).
 * By default ocm_solve measures, once per solve, the fraction of edges whose
 * target lies in the same block range of the evaluation grid as its source
 * (ranges of about n / 152 consecutive vertices on a GB300); graphs of at
 * least 2^18 vertices with at least 85% of such edges get the two-level
 * evaluation: every block first resolves the policy paths inside its own
 * range with block barriers only, leaving the vertices whose successor lies
 * outside it ("exits"), and the cycles that cross ranges are then found and
 * valued on the much smaller graph of the exits.  OCM_FLAG_EVAL_LOCAL forces
 * the two-level evaluation, OCM_FLAG_EVAL_GLOBAL forbids it (setting both is
 * OCM_ERR_INVALID_ARG).  The two-level form serves ocm_solve without transit
 * times and without OCM_FLAG_SINGLE_LAMBDA; the other calls always use the
 * one-level evaluation. */
#define OCM_FLAG_EVAL_LOCAL 8
#define OCM_FLAG_EVAL_GLOBAL 16

/* Test-only: the two-level evaluation runs without its shared-memory bitmaps
 * (every vertex of a range takes part in the jump rounds), the form it takes
 * on its own for ranges of more than 436,906 vertices.  Same results. */
#define OCM_FLAG_TEST_NO_BITMAP 32

/* Test-only: the degree-class sweep and the initial pass take their warp
 * tasks in bands of 1,024 vertices (the band-by-band order large graphs get,
 * with many more bands).  Same results. */
#define OCM_FLAG_TEST_SMALL_BANDS 64

/* Test-only: the frontier sweep after every evaluation but the first.  By
 * default the record pass marks the records it changes when the sweep before
 * it switched fewer than n/512 vertices, and the next sweep then skips the
 * vertices none of whose out-edges' targets changed its record, when fewer
 * than n/8 records changed (such a vertex would choose as in the last sweep);
 * not in the single-lambda form, whose rebuild writes records itself.  With
 * this flag the marks and the skipping happen whatever the counts.  Same
 * results. */
#define OCM_FLAG_TEST_FRONTIER 128

/* Test-only: the local phase of the two-level evaluation.  By default every
 * block resolves its range in chunks of 4,096 vertices from the top of the
 * range down: a vertex whose successor lies in a chunk done before starts
 * from that vertex's finished state, the paths inside a chunk are resolved by
 * pointer jumping in shared memory, and the paths that go back to a lower
 * chunk are finished by jumping over the range at the end (on a graph whose
 * edges point forward there are none, and each range costs one streaming
 * pass).  Once a range leaves more than an eighth of its vertices to that
 * last step, the solve's later evaluations use leaf-trimmed jump rounds over
 * the whole range instead.  OCM_FLAG_TEST_LOCAL_CHUNKS keeps the chunks in
 * every evaluation, OCM_FLAG_TEST_NO_LOCAL_CHUNKS never uses them (setting
 * both is OCM_ERR_INVALID_ARG).  Same results. */
#define OCM_FLAG_TEST_LOCAL_CHUNKS 256
#define OCM_FLAG_TEST_NO_LOCAL_CHUNKS 512

/* Counters of one solve (host struct, filled when a pointer is given). */
typedef struct ocm_stats {
    int32_t iterations;     /* improvement sweeps that changed the policy           */
    int32_t cycles;         /* cycles in the final policy graph                     */
    int32_t detect_rounds;  /* cycle-detection jump rounds, summed over iterations  */
    int32_t value_rounds;   /* value-propagation jump rounds, summed over iterations */
    int64_t switched;       /* vertex policy switches summed over iterations        */
    int64_t launches;       /* kernels launched by this call                        */
    int64_t detect_items;   /* vertex-rounds of work in cycle detection             */
    int64_t value_items;    /* vertex-rounds of work in value propagation           */
    int32_t graph_loop;     /* 1: the iteration ran as a CUDA graph, 0: host-driven */
    int32_t rebuild_levels; /* OCM_FLAG_SINGLE_LAMBDA: backward-search levels of the
                               rebuilds, summed over iterations; 0 otherwise         */
    int32_t batch_small_graphs; /* ocm_solve_batch: graphs solved one per thread block
                                   (see ocm_options.batch_small_vertices)          */
    int32_t sweep_kind;     /* OCM_SWEEP_* layout the improvement sweep used        */
} ocm_stats;

/* Bytes of device workspace ocm_solve needs for a graph with n vertices and m
 * edges (256-byte aligned base required).  Returns 0 if n or m is out of
 * range.  The workspace holds the policy, per-vertex values, pointer-jumping
 * buffers and per-cycle records; its contents are scratch between calls.    */
size_t ocm_workspace_size(int32_t n, int32_t m);

/* Bytes of device workspace for ocm_solve with OCM_FLAG_SINGLE_LAMBDA:
 * ocm_workspace_size(n, m) plus about 4 m + 20 n bytes.  0 if out of range. */
size_t ocm_workspace_size_single(int32_t n, int32_t m);

/*
 * ocm_solve -- optimal cycle mean of one graph.
 *   row_ptr, col_idx, w : device CSR as described above (read only)
 *   n, m                : vertex and edge counts, 1 <= n, 1 <= m < 2^31
 *   mode                : OCM_MAX or OCM_MIN
 *   num, den            : host; lambda* = *num / *den, *den > 0, gcd(|num|, den) = 1
 *   cycle_out           : device [n]; receives the critical cycle as CSR edge
 *                         indices in cycle order, starting with the policy edge
 *                         of the cycle's smallest vertex (Alg. 1 MinVertex)
 *   cycle_len           : host; number of edges written to cycle_out
 *   workspace, ws_bytes : device scratch of at least ocm_workspace_size(n, m) bytes
 *   stream              : cudaStream_t as void*
 *   opt                 : NULL for defaults
 *   stats               : host, NULL to skip
 * Synchronises the stream before returning (the scalars are host values).
 * Among several optimal cycles, the returned one is fixed by the iteration:
 * the policy cycle of largest mean whose smallest vertex is smallest.
 */
int ocm_solve(const int32_t *row_ptr, const int32_t *col_idx, const int32_t *w, int32_t n,
              int32_t m, int mode, int64_t *num, int32_t *den, int32_t *cycle_out,
              int32_t *cycle_len, void *workspace, size_t ws_bytes, void *stream,
              const ocm_options *opt, ocm_stats *stats);

/*
 * ocm_solve_batch -- optimal cycle means of G independent graphs in one call
 * (the paper runs its regions concurrently, Sec. 3.3; here the regions are
 * separate graphs).  The graphs form one disjoint-union CSR:
 *   graph_vptr[G+1] : device; graph g owns vertices [graph_vptr[g], graph_vptr[g+1]),
 *                     graph_vptr[0] = 0, graph_vptr[G] = N, every graph non-empty
 *   row_ptr[N+1], col_idx[M], w[M] : device CSR with global vertex ids; every
 *                     edge must stay inside its own graph (OCM_ERR_BAD_CSR otherwise)
 *   num[G], den[G], cycle_len[G] : device outputs, one reduced mean and cycle
 *                     length per graph (in the given sense)
 *   cycle_out[N]    : device; graph g's critical cycle (CSR edge indices,
 *                     starting with the policy edge of its smallest vertex) is
 *                     written at offset graph_vptr[g] (a simple cycle of g has
 *                     at most n_g edges)
 *   workspace       : at least ocm_workspace_size_batch(G, N, M) bytes
 * Every graph's result is bit-identical to solving it alone with ocm_solve.
 * Exactness bound: 2 * n_max^2 * max|w| < 2^62 with n_max the largest graph.
 * Synchronises the stream before returning; on error the device outputs may
 * be partly written.
 */
size_t ocm_workspace_size_batch(int32_t G, int32_t N, int32_t M);
int ocm_solve_batch(const int32_t *graph_vptr, const int32_t *row_ptr, const int32_t *col_idx,
                    const int32_t *w, int32_t G, int32_t N, int32_t M, int mode, int64_t *num,
                    int32_t *den, int32_t *cycle_len, int32_t *cycle_out, void *workspace,
                    size_t ws_bytes, void *stream, const ocm_options *opt, ocm_stats *stats);

/*
 * ocm_backward -- gradient of lambda* with respect to the edge weights.
 * While the critical cycle C* stays optimal, lambda* = w(C*)/|C*| is linear in
 * the weights of C*, so the derivative of lambda* by w(e) = 1/|C*| for e in C* and 0 otherwise
 * (the same in both senses).  Writes grad_w[e] = grad_lambda[0] * that value.
 *   cycle_edges : device [cycle_len], distinct edge indices in [0, m)
 *   grad_lambda : device [1] float, upstream gradient
 *   grad_w      : device [m] float, fully overwritten
 * Asynchronous on `stream`.
 */
int ocm_backward(const int32_t *cycle_edges, int32_t cycle_len, const float *grad_lambda,
                 int32_t m, float *grad_w, void *stream);

/*
 * ocm_backward_ratio -- the gradient of an optimal cycle ratio
 * lambda* = w(C*)/t(C*) (a solve with ocm_options.transit).  While C* stays
 * optimal, lambda* is linear in the weights of C* with slope 1/t(C*), so
 * grad_w[e] = grad_lambda[0] / t(C*) for e in C* and 0 otherwise; t(C*) is
 * summed on the device from transit over cycle_edges.
 *   cycle_edges : device [cycle_len], distinct edge indices in [0, m)
 *   transit     : device [m] int32 transit times, as given to the solve
 *   grad_lambda : device [1] float, upstream gradient
 *   grad_w      : device [m] float, fully overwritten
 * Asynchronous on `stream`.
 */
int ocm_backward_ratio(const int32_t *cycle_edges, int32_t cycle_len, const int32_t *transit,
                       const float *grad_lambda, int32_t m, float *grad_w, void *stream);

/*
 * ocm_backward_batch -- the gradient of every graph's lambda* for a batched
 * solve: grad_w[e] = grad_lambda[g] / cycle_len[g] for each edge e of graph
 * g's critical cycle, 0 for every other edge (as ocm_backward, per graph).
 *   graph_vptr[G+1], cycle_out[N], cycle_len[G] : device, as produced by
 *                    ocm_solve_batch (graph g's cycle at offset graph_vptr[g])
 *   grad_lambda[G] : device float, upstream gradient per graph
 *   grad_w[M]      : device float, fully overwritten
 * Asynchronous on `stream`; edge indices outside [0, M) are ignored.
 */
int ocm_backward_batch(const int32_t *graph_vptr, const int32_t *cycle_out,
                       const int32_t *cycle_len, const float *grad_lambda, int32_t G, int32_t M,
                       float *grad_w, void *stream);

/* Instrumentation for benchmarks (not needed to solve).  While enabled,
 * every kernel launch of ocm_solve is bracketed by CUDA events recorded on
 * the solve's stream, grouped by class:
 *   0 CSR checks + initial policy, 1 improvement sweep, 2 policy evaluation
 *   (cycle detection, value propagation, cycle means and ranks, values),
 *   3 critical-cycle extraction and optional outputs.
 * ocm_profile_enable returns the previous setting.  ocm_profile_collect waits
 * for the recorded events, adds their durations (ms) and launch counts per
 * class into ms_out[0..3] and launches_out[0..3] (host arrays, either may be
 * NULL), forgets them, and returns the number of classes (4).  Not
 * thread-safe: use from one host thread.                                    */
#define OCM_PROFILE_CLASSES 4
int ocm_profile_enable(int on);
int ocm_profile_collect(double *ms_out, int64_t *launches_out);

/*
 * ocm_solve_static -- ocm_solve without a caller-provided workspace, for
 * callers that cannot allocate device memory (a process whose device memory
 * is capped or already handed out, a plugin or real-time loop that must not
 * allocate after start-up).  The paper has no counterpart: this is a
 * deployment convenience of this library.
 *
 * The scratch space is a fixed array of OCM_STATIC_WORKSPACE_BYTES inside
 * the library's GPU image: every device that loads the library holds it
 * until the process exits.  Graphs with ocm_workspace_size(n, m) larger than
 * that (about 192,000 vertices at mean out-degree 4) are rejected with
 * OCM_ERR_WORKSPACE before any device work.  The call allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine (benchmark
 * instrumentation is paused while it runs).  Arguments, outputs,
 * synchronisation and errors are those of ocm_solve.
 *
 * Every call looks up the array's device address in the current context
 * (the device must be current, as for every entry point) instead of caching
 * it, so a context that was reset and created again is handled.  With lazy
 * module loading (CUDA_MODULE_LOADING=LAZY, the CUDA default) the array is
 * created when the library's GPU code is first loaded on the device, which
 * may be the first call of this function: a caller whose device memory is
 * capped should make one call at start-up (any small graph), before its
 * budget is handed out, so that later calls find the array in place.  Like
 * ocm_solve it synchronises the stream, so it is not called while that
 * stream is being captured.  All calls on a device share the one array:
 * calls whose GPU work overlaps (several host threads or streams at once)
 * race and corrupt each other, so serialise them.  The array keeps the last
 * call's contents, which the next call does not need: everything the solver
 * reads is initialised by the solver first.
 */
#define OCM_STATIC_WORKSPACE_BYTES (32u << 20)
int ocm_solve_static(const int32_t *row_ptr, const int32_t *col_idx, const int32_t *w,
                     int32_t n, int32_t m, int mode, int64_t *num, int32_t *den,
                     int32_t *cycle_out, int32_t *cycle_len, void *stream,
                     const ocm_options *opt, ocm_stats *stats);

/*
 * ocm_scc -- strongly connected components (the decomposition the paper runs
 * before its solver, Sec. 3.3; Prop. 2.2 reduces the optimal cycle mean of a
 * graph to those of its components).  Forward-backward searches with trimming
 * over colour classes, on the GPU; any CSR digraph (vertices without
 * out-edges allowed, m may be 0).
 *   row_ptr[n+1], col_idx[m] : device CSR (no weights needed)
 *   scc[n]      : device output; scc[v] = the smallest vertex of v's component
 *   num_scc     : host output; number of components
 *   workspace   : at least ocm_workspace_size_scc(n, m) bytes, 256-byte aligned
 * Synchronises the stream.  Errors: OCM_ERR_INVALID_ARG (null pointers, n < 1,
 * m < 0, n > (2^31 - 3) / 3), OCM_ERR_BAD_CSR, OCM_ERR_WORKSPACE, OCM_ERR_CUDA,
 * OCM_ERR_TIMEOUT; outputs untouched on an argument or CSR error.
 */
size_t ocm_workspace_size_scc(int32_t n, int32_t m);
int ocm_scc(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int32_t m, int32_t *scc,
            int32_t *num_scc, void *workspace, size_t ws_bytes, void *stream);

/*
 * ocm_solve_scc -- the optimal cycle mean of every strongly connected
 * component that holds a cycle (Sec. 3.3: the components are solved
 * concurrently as regions).  The graph may have vertices without out-edges
 * and acyclic parts; components without a cycle (a single vertex without a
 * self-loop) are left out.  Each component is solved as its induced subgraph
 * with its vertices in their original order (same value, cycle and
 * iteration as ocm_solve on that subgraph); the optimum over components is
 * the optimal cycle mean of the whole graph.
 *   row_ptr, col_idx, w, n, m, mode : as for ocm_solve, except that out-degree
 *                 0 is allowed and m may be 0
 *   scc[n]      : device; component labels as for ocm_scc
 *   num_comp    : host; G = number of components with a cycle (0 if none)
 *   comp_root[n], num[n], den[n], cycle_len[n] : device; entries 0..G-1, one
 *                 per component in increasing order of its smallest vertex
 *                 (comp_root[c]), with its reduced mean num/den (in the given
 *                 sense) and its critical cycle's length
 *   comp_off[n+1], cycle_out[n] : device; component c's critical cycle, as
 *                 CSR edge indices of the input graph starting with the policy
 *                 edge of its smallest vertex, is cycle_out[comp_off[c] ..
 *                 comp_off[c] + cycle_len[c])
 *   workspace   : at least ocm_workspace_size_solve_scc(n, m) bytes
 *   opt         : max_iters, flags (OCM_FLAG_HOST_LOOP) and the sweep's launch
 *                 fields apply; init_policy and transit must be NULL
 *   stats       : counters of the batched solve, launches of the whole call
 * Synchronises the stream.  Errors as for ocm_scc and ocm_solve_batch.
 */
size_t ocm_workspace_size_solve_scc(int32_t n, int32_t m);
int ocm_solve_scc(const int32_t *row_ptr, const int32_t *col_idx, const int32_t *w, int32_t n,
                  int32_t m, int mode, int32_t *scc, int32_t *num_comp, int32_t *comp_root,
                  int32_t *comp_off, int64_t *num, int32_t *den, int32_t *cycle_len,
                  int32_t *cycle_out, void *workspace, size_t ws_bytes, void *stream,
                  const ocm_options *opt, ocm_stats *stats);

/* Text for a status code (static storage). */
const char *ocm_status_string(int status);

/* ABI version: 100 * major + minor (101: ocm_options.init_policy; 102:
 * ocm_options.transit and ocm_backward_ratio; 103: ocm_scc and
 * ocm_solve_scc; 104: OCM_FLAG_SINGLE_LAMBDA, ocm_workspace_size_single,
 * ocm_stats.rebuild_levels; 105: ocm_solve_static,
 * OCM_STATIC_WORKSPACE_BYTES; 106: ocm_options.wait_limit_ms, the OCM_FAULT
 * test hook; 107: ocm_options.batch_small_vertices,
 * ocm_stats.batch_small_graphs; 108: OCM_FLAG_EVAL_LOCAL, OCM_FLAG_EVAL_GLOBAL,
 * OCM_FLAG_TEST_NO_BITMAP; 109: OCM_SWEEP_WINDOW, ocm_stats.sweep_kind; 110:
 * OCM_FLAG_TEST_SMALL_BANDS; 111: OCM_FLAG_TEST_FRONTIER and the frontier
 * sweep; 112: OCM_FLAG_TEST_LOCAL_CHUNKS, OCM_FLAG_TEST_NO_LOCAL_CHUNKS and
 * the chunked local phase). */
int ocm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OCM_H_ */
