// common.cuh -- device-side layout shared by the solver's kernels.
//
// Notation follows the paper (Sec. 2.4, Alg. 1): pi is the policy (one
// out-edge per vertex), G_pi the policy graph, and every cycle of G_pi has a
// root, its smallest vertex (Alg. 1 MinVertex).  Internally the solver always
// maximises s*w (s = +1 for the maximum cycle mean, -1 for the minimum).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ocm.h"

namespace ocm {

constexpr int kThreads = 256;          // block size of every kernel
constexpr int kSweepTileV = 256;       // vertices per improvement-sweep tile
constexpr int kEvalThreads = 1024;     // block size of the persistent evaluation kernel
// Degree classes of the improvement sweep: class c serves a vertex with a
// group of 2^c lanes; a vertex of out-degree d belongs to the smallest class
// with d <= kEdgesPerLane * 2^c (the last class takes everything larger).
constexpr int kClasses = 6;
// A vertex with more than kHeavyEdges out-edges leaves the lane-group classes
// for the heavy path: the heavy vertices' edges, taken as one sequence, are
// cut into chunks of kHeavyChunk edges, one block per chunk, and the chunks'
// partial results are combined per vertex (a chunk meets at most two heavy
// vertices because each has more than kHeavyChunk edges).
constexpr int kHeavyEdges = 1024;
constexpr int kHeavyChunk = 1024;
constexpr int kHeavyThreads = 256;
constexpr int kClassSlots = kClasses + 1;   // the lane-group classes, then the heavy class
constexpr int kEdgesPerLane = 8;       // default; ocm_options.edges_per_lane overrides
constexpr int kSweepMaxThreads = 512;  // largest sweep block (ocm_options.sweep_threads)
constexpr int kSweepThreads = 512;     // default sweep block
constexpr int kClassifyBlock = 1024;   // vertices per classification block
// The degree-class sweep takes its warp tasks band by band: all classes of
// the vertices [b * kSweepBand, (b + 1) * kSweepBand), then the next band, so
// that the records the band's edges gather stay in L2 across the class passes.
// A graph of at most kSweepOneBandN vertices (records of at most 64 MB, which
// L2 holds anyway) is one band: class by class over the whole graph.
constexpr int kSweepBand = 1 << 18;
constexpr int kSweepOneBandN = 1 << 22;
// Classification blocks per band (the default), and the sweep's (band,
// class) groups for bands of B classification blocks.
__host__ __device__ inline int sweep_band_blocks(int n) {
    return n <= kSweepOneBandN ? (n + kClassifyBlock - 1) / kClassifyBlock
                               : kSweepBand / kClassifyBlock;
}
__host__ __device__ inline int sweep_groups(int n, int B) {
    const long long band = (long long)B * kClassifyBlock;
    return kClasses * (int)((n + band - 1) / band);
}
constexpr int kBatchSmallDefault = 4096;   // batch: smallest automatic per-block size limit
// The two-level evaluation is chosen for graphs of at least this many
// vertices with at least this fraction of edges inside their block range.
constexpr int kLocalEvalMinN = 1 << 18;
constexpr double kLocalEvalMinFraction = 0.85;
// Window sweep (sweep_window.cu): tiles of kWinTile vertices, each seeing the
// records of kWinHalo more vertices in shared memory, the window starting hb
// before the tile; the initial pass counts, for hb = j * kWinTile (j <
// kWinShapes), the edges whose target lies in [v - hb, v - hb + kWinHalo),
// and the sweep takes the hb that holds the most.
constexpr int kWinTile = 2048;
constexpr int kWinHalo = 4 * kWinTile;
constexpr int kWinShapes = 5;

// Per-vertex record the improvement sweep gathers for every edge target t:
// the value V(t) (scaled by the denominator q of t's cycle mean), the rank of
// t's cycle mean among the current cycles, and q.  16 bytes, one vector load.
struct __align__(16) Rec {
    long long V;
    int rank;
    int q;
};

// Cycle-detection jump state: J = succ^(2^k)(v), M = smallest vertex among the
// 2^k vertices starting at v.
struct __align__(8) JM {
    int J;
    int M;
};

// Value-propagation jump state: J = a vertex on v's policy path (the root once
// done), len and S = length and s*w-weight of the path from v to J.
struct __align__(16) JLS {
    int J;
    int len;
    long long S;
};

// State of the grid-wide barrier of one cooperative kernel (grid_sync.cuh):
// arrivals counted since the launch, and the summed counts of the barriers
// in four rotating slots.  Zero when the kernel is launched.
struct GridBar {
    unsigned long long arrive;
    int sum[4];
    int sum2[4];          // a second count (grid_sum2_barrier)
    int pad[2];
};

// Control block in device memory (one per solve).
struct Ctrl {
    int err;              // OR of kErr* bits
    int bad_index;        // first offending index seen (for diagnostics)
    int changed;          // the sweep switched at least one vertex
    int switched;         // number of switched vertices in the last sweep
    int cnt[3];           // rotating worklist counters
    int nrep;             // number of policy cycles (roots)
    int maxabsw;          // max |w| over all edges
    int ncand;            // cycle-extraction candidates
    int rounds_detect;    // jump rounds that had work (cycle detection)
    int rounds_value;     // jump rounds that had work (value propagation)
    long long items_detect;   // worklist items processed, all detect rounds
    long long items_value;    // worklist items processed, all value rounds
    unsigned long long best;  // packed (rank, INT_MAX - root) of the best cycle
    GridBar bar[2];           // grid barriers: [0] evaluation (and the SCC kernels), [1] rebuild
    int pending[3];           // detect: rotating per-round counts of unfinished vertices
    int pendv[3];             // values: the same
    int cls_cnt[8];           // improvement sweep: vertices per degree class (then heavy)
    int cls_off[8];           // start of each class in the class list
    int heavy_edges;          // improvement sweep: edges of all heavy vertices
    // result of a solve, copied to the host in one transfer
    long long res_num;
    int res_den;
    int res_len;
    int res_root;
    int res_cycles;
    int max_ng;               // batch: largest graph
    int active_graphs;        // batch: graphs whose policy may still change
    // iteration state, advanced on the device by the loop control kernel
    int iter;                 // index of the current evaluation (0 = initial policy)
    int loop_more;            // the last step asks for another one
    int not_converged;        // the iteration cap was reached
    long long switched_total; // switches summed over all sweeps
    int maxt;                 // cycle ratio: largest transit time
    int qmax;                 // cycle ratio: largest ratio denominator of the current cycles
    int fcnt[3];              // single-lambda rebuild: rotating frontier counters
    int hcnt[2][3];           // SCC searches: rotating counters of the heavy frontiers (fw, bw)
    int connect_levels;       // single-lambda rebuild: backward-search levels, all iterations
    long long wait_ns;        // limit of every device-side wait (grid barriers), nanoseconds
    // batch: the per-graph solver of the small graphs (batch_small.cu)
    int small_bucket[32];     // graphs per size bucket floor(log2 n_g)
    int small_cursor[32];     // fill cursors of the buckets
    int small_total;          // graphs in the queue
    int small_head;           // next queue position to pop
    int small_iters;          // largest iteration count among them
    int node_cnt;             // two-level evaluation: exits listed (nodes of the contracted graph)
    int fix_k;                // two-level evaluation: roots found on the node graph (capped)
    int fix_cnt;              // two-level evaluation: vertices listed for the root fix
    int fix_root[32];         // those roots
    int fix_tag[32];          // and their tags before the fix (n + their exit)
    long long local_edges;    // edges whose target lies in the source's block range
    long long win_edges[kWinShapes];   // edges inside each window shape of the window sweep
    // frontier sweep: 0 off (single-lambda form), 1 when few vertices switched,
    // 2 (test) after every evaluation but the first
    int frontier;
    int dirty_on;             // the last record pass marked the records it changed
    // two-level evaluation: chunked local pass (0 off, 1 on until a range
    // leaves more than an eighth of its vertices pending, 2 always), and the
    // report of such a range
    int local_chunks;
    int chunk_bad;
    int walk_ok;              // extraction: the segment walk found the critical cycle
    long long dirty_cnt;      // how many it changed
};

// The record pass marks the records it changes when the sweep before it
// switched fewer than n >> kFrontierSwitchShift vertices, and the next sweep
// then skips the vertices none of whose targets' records changed when fewer
// than n >> kFrontierDirtyShift did (their choice would be the same as in the
// last sweep).
// A second bitmap marks blocks of kDirtyBlock vertices with a changed record
// (a few KB, held in L1), and the sweep looks at a target's own bit only
// where its block's bit is set; a whole block of kClassifyBlock vertices none
// of whose edges reaches a changed block (by the range of target blocks the
// initial pass records) is skipped without reading its edges.
constexpr int kFrontierSwitchShift = 9;
constexpr int kFrontierDirtyShift = 3;
constexpr int kDirtyBlock = 1024;
// A vertex whose block's targets span more than this many dirty-bitmap words
// checks its edges one by one.
constexpr int kFrontierRangeWords = 64;

// Default limit of a device-side wait, and the one the test-only stall flag
// uses unless the caller sets ocm_options.wait_limit_ms.
constexpr long long kDefaultWaitNs = 2000000000LL;   // two seconds
constexpr long long kStallTestWaitNs = 10000000LL;   // 10 ms

enum : int {
    kErrRowPtr = 1,
    kErrNoOutEdge = 2,
    kErrCol = 4,
    kErrWeightMin = 8,
    kErrDetect = 16,      // cycle detection did not finish in the round budget
    kErrValue = 32,       // value propagation did not finish in the round budget
    kErrExtract = 64,     // critical-cycle extraction inconsistent
    kErrTimeout = 128,    // a grid barrier wait exceeded its spin limit
    kErrSweep = 256,      // a vertex's current policy edge was not among its edges
    kErrInitPolicy = 512, // a caller-given initial policy edge is not an out-edge of its vertex
    kErrTransit = 1024,   // a transit time below 1
    kErrRatioKey = 2048,  // cycle ratio: the exact order keys of the current cycles overflow int64
    kErrUnreached = 4096, // single-lambda rebuild: a vertex cannot reach the chosen cycle
    kErrConnect = 8192,   // single-lambda rebuild: inconsistent state (no chosen cycle, no edge)
};

// Workspace carved from one caller-provided buffer.
struct Workspace {
    int *pi, *succ, *wpi;
    Rec *rec;
    JM *jm[2];
    int *aprev;
    int *rep;
    JLS *jls[2];
    int *list[3];
    int *cyc_root;
    long long *cyc_p;
    int *cyc_q;
    int *cyc_L;
    long long *cyc_key;
    int *cyc_rank;
    int *cid_of_root;
    unsigned *done;       // bitmap: vertex resolved and its state in both buffers
    unsigned *rec_dirty;  // bitmap: the last record pass changed v's record (Ctrl::dirty_on)
    unsigned *need_blk;   // bitmap over blocks of kClassifyBlock vertices: some target of
                          //     the block's edges lies in a block with a changed record
    int2 *blk_tgt;        // [n / kClassifyBlock] smallest and largest target block (of
                          //     kDirtyBlock vertices) of the out-edges of each block of
                          //     kClassifyBlock vertices (heavy vertices left out)
    int4 *scratch16;      // [n] two-level evaluation: packed jump states, then node values
                          //     (the records stay intact for the frontier comparison)
    unsigned *rec_dirty_blk;  // bitmap: ... some record of v's block of kDirtyBlock vertices
    int *sw_iter;         // evaluation index after the sweep that last switched v
    int *cls_list;        // vertices grouped by degree class (stable within a class)
    int *cls_hist;        // per-block class counts, then their exclusive scan
    int4 *band_grp;       // [bands * kClasses + 1] per (band, class), band-major: first
                          //   warp task, first class-list entry, entries, class; the
                          //   last .x = all tasks
    int *heavy_off;       // [n+1] heavy vertex i's edges are entries heavy_off[i] .. heavy_off[i+1]
                          //       of the heavy edge sequence
    struct Cand *heavy_part;  // [2 * (m / kHeavyChunk + 2)] per chunk: best of its first and
                              //       of its second heavy vertex
    // edge-tiled sweep: tile t covers edges [t*ET, (t+1)*ET)
    int *tile_v;          // [T+1] source vertex of each tile's first edge
    int *tile_pend;       // [T] vertex whose edges run past the tile's end and whose
                          //     first edge lies in it (-1: none)
    int *tile_fopen;      // [T] the tile's first vertex (begun in an earlier tile)
                          //     still has edges after this tile
    struct TilePart *tile_first;  // [T] best and current-edge key of that vertex in this tile
    struct TilePart *tile_last;   // [T] the same for tile_pend's vertex, up to the tile's end
    // optimal cycle ratio (used only when transit != nullptr)
    const int *transit;   // caller's transit times t(e) >= 1 (input, not workspace memory)
    int *tpi;             // [n] transit time of the policy edge
    long long *jt[2];     // [n] value jumping: transit time of the path from v to J
    long long *recp;      // [n] numerator p of the ratio of v's cycle (gathered by the sweep)
    int *root_mark;       // [n] two-level evaluation: evaluation stamp of a root found on the node graph
    int2 *chunk_info;     // [n / 1024 + 2] chunked local pass, per block range: (status, exits)
    Ctrl *ctrl;
};

// Candidate edge of the improvement sweep and its total order: larger
// rank(t) first, then larger key q_t * s*w(e) + V(t), then smaller edge index
// (the deterministic tie-break that makes the choice unique).
struct Cand {
    int rank;
    int e;
    long long key;
};

// Degree class of a vertex of out-degree d in the lane-group sweeps (the
// smallest c with d <= epl * 2^c, capped at kClasses - 1); kClasses: heavy.
__device__ __forceinline__ int degree_class(int d, int epl) {
    if (d > kHeavyEdges) return kClasses;   // the heavy path
    int c = 0;
    while (c < kClasses - 1 && d > (epl << c)) ++c;
    return c;
}

__device__ __forceinline__ bool better(const Cand &a, const Cand &b) {
    if (a.rank != b.rank) return a.rank > b.rank;
    if (a.key != b.key) return a.key > b.key;
    return a.e < b.e;
}

// The part of a vertex's sweep that one tile saw: the best candidate among
// its edges there, and the key of its current policy edge if that edge lies
// in the tile (crank = INT_MIN otherwise).
struct __align__(16) TilePart {
    int rank;
    int e;
    long long key;
    int crank;
    int pad;
    long long ckey;
};

// Extra state of a batched solve (G graphs as one disjoint-union CSR);
// all pointers are null for a single-graph solve.
struct BatchState {
    const int *vptr;              // [G+1] vertex offsets of the graphs
    int *gid;                     // [N] graph of each vertex
    unsigned long long *gbest;    // [G] packed (rank, INT_MAX - root) of each graph's best cycle
    int *groot;                   // [G] root of each graph's critical cycle
    int *glen;                    // [G] its length
    int *gfound;                  // [G] cycle vertices found by the extraction
    long long *gp;                // [G] reduced mean of the critical cycle: numerator
    int *gq;                      //     and denominator
    int *gconv;                   // [G] 1 once the graph's policy is final
    int *gsw;                     // [G] evaluation index after the last sweep that switched in g
    int *small_queue;             // [G] graphs solved by one block each, largest first
    int G;
};

// Layout of the workspace for n vertices; returns total bytes and fills ws
// when base != nullptr.
size_t carve_workspace(void *base, int n, int m, Workspace *ws);

// Extra state of the single-lambda iteration (OCM_FLAG_SINGLE_LAMBDA), carved
// after the workspace above: the transposed graph for the backward search
// and its levels and frontiers.
struct SingleWs {
    int *in_ptr;    // [n+1] CSC offsets
    int *in_src;    // [m] source vertex of each in-edge
    int *cursor;    // [n] CSC scatter cursors
    int *bsum;      // [n / 1024 + 2] block sums of the offset scan
    int *lev;       // [n] search level: -1 unconnected, -2 reached at the current level
    int *fr[2];     // [n] frontiers of consecutive levels
};
size_t carve_single(void *base, int n, int m, SingleWs *sw);

// Smallest tile of the edge-tiled sweep (32 lanes x 4 edges); the workspace
// holds the per-tile arrays for this size, enough for every larger one.
constexpr int kMinTileEdges = 128;

// Block 0, thread 0 of every sweep: publish the best cycle of the evaluation
// the sweep reads (the answer if nothing switches).  best is 0 only when that
// evaluation stopped early on an error, which the host reports.
__device__ __forceinline__ void publish_result(const Workspace &ws, int n) {
    Ctrl *cc = ws.ctrl;
    const unsigned long long bb = cc->best;
    const int root = 0x7fffffff - (int)(unsigned)(bb & 0xffffffffu);
    if (bb != 0 && root >= 0 && root < n) {
        const int i = ws.cid_of_root[root];
        cc->res_root = root;
        cc->res_len = ws.cyc_L[i];
        cc->res_num = ws.cyc_p[i];
        cc->res_den = ws.cyc_q[i];
        cc->res_cycles = cc->nrep;
    }
}

// Local state of v after the two-level evaluation's local phase.  After the
// leaf-trimmed rounds (local_onepass) a vertex that no vertex of its range
// jumps to (a "leaf": no predecessor in the range, or leaves only) keeps the
// one step to its successor, J = succ(v) >= 0, len 1 and its edge weight,
// and is completed here by following those steps: at most two, since the
// successor of a leaf whose predecessors are all leaves has a state of its
// own.  Every other state (all of them after the chunked pass) is returned
// as stored.
__device__ __forceinline__ JLS local_state(const JLS *jls0, int v) {
    JLS st = jls0[v];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (st.J < 0) break;
        const JLS nx = jls0[st.J];
        st = JLS{nx.J, st.len + nx.len, st.S + nx.S};
    }
    return st;
}

// Final value state (J = ~root, len, S) of vertex v from the evaluation's
// value buffer.  After the two-level evaluation a vertex whose path leaves its
// block range holds its state to the exit x it leaves by (J = ~(n + x)), and
// its final state adds x's (an exit's own state is final); a leaf holds one
// step to its successor (local_state).  After the one-level evaluation every
// state is final and this is a plain load.
__device__ __forceinline__ JLS final_value(const JLS *jls0, int n, int v) {
    JLS st = local_state(jls0, v);
    const int tag = ~st.J;
    if (tag >= n) {
        const JLS nf = jls0[tag - n];
        st = JLS{nf.J, st.len + nf.len, st.S + nf.S};
    }
    return st;
}

__device__ __forceinline__ int warp_append(int *counter, bool pred, int lane) {
    unsigned mask = __ballot_sync(0xffffffffu, pred);
    int base = 0;
    if (mask) {
        int leader = __ffs(mask) - 1;
        if (lane == leader) base = atomicAdd(counter, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
    }
    return base + __popc(mask & ((1u << lane) - 1u));
}

__device__ __forceinline__ long long gcd_ll(long long a, long long b) {
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b != 0) {
        long long t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// floor(p * N2 / q) for q > 0: an order-preserving integer image of p/q that
// separates any two distinct fractions with denominators <= sqrt(N2).
__device__ __forceinline__ long long mean_key(long long p, long long q, long long N2) {
    __int128 a = (__int128)p * (__int128)N2;
    __int128 d = a / q;
    if ((a % q) != 0 && a < 0) d -= 1;
    return (long long)d;
}

// profiling hooks (api.cu): bracket a kernel launch of class cls with events
enum ProfClass : int { kProfInit = 0, kProfSweep = 1, kProfEvaluate = 2, kProfExtract = 3, kProfCount = 4 };
void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, cudaStream_t st);
// Pauses the instrumentation for the calling host thread while in scope
// (the solve without allocation must not create CUDA events).
struct ProfilePause {
    ProfilePause();
    ~ProfilePause();
    bool prev;
};
bool prof_active();
bool injected_fault(const char *what);
// NVTX range over a host-side phase of an entry point (visible in Nsight
// Systems timelines; free when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name);
    ~NvtxRange();
};

// kernel launchers (defined in the .cu files)
void launch_check_row_ptr(const int *row_ptr, int n, int m, Ctrl *ctrl, cudaStream_t st);
void launch_init_policy(const int *row_ptr, const int *col, const int *w, int sign, int n, int m,
                        const int *init, Workspace ws, const BatchState *bs, cudaStream_t st,
                        int local_R = 0, int count_win = 0, int band_blocks = 1);
int launch_sweep(const int *row_ptr, const int *col, const int *w, int sign, int n,
                 Workspace ws, const int *cls_cnt, int heavy_edges, BatchState bs, int threads,
                 int band_blocks, cudaStream_t st);
int launch_tile_index(const int *row_ptr, int n, int m, int tile_edges, Workspace ws,
                      cudaStream_t st);
int launch_sweep_heavy(const int *row_ptr, const int *col, const int *w, int sign, Workspace ws,
                       int H, int heavy_edges, BatchState bs, cudaStream_t st);
int launch_sweep_window(const int *row_ptr, const int *col, const int *w, int sign, int n,
                        int epl, int hb, Workspace ws, const int *cls_cnt, int heavy_edges,
                        BatchState bs, cudaStream_t st);
// Host-side kernel configuration (shared-memory opt-in, occupancy), done
// before the loop so that a captured loop graph holds launches only;
// 0 on success.
int prepare_evaluate(bool ratio);
int prepare_sweep_classes(int threads, bool ratio);
int prepare_sweep_tiles(int edges_per_lane, int threads);
int prepare_sweep_window();
int launch_sweep_tiles(const int *row_ptr, const int *col, const int *w, int sign, int n, int m,
                       int edges_per_lane, Workspace ws, BatchState bs, int threads,
                       cudaStream_t st);
int launch_batch_converge(BatchState bs, Workspace ws, cudaStream_t st);
int launch_classify(const int *row_ptr, int n, int epl, int band_blocks, Workspace ws,
                    cudaStream_t st);
int launch_evaluate(int n, long long N2, Workspace ws, int stall_test, BatchState bs,
                    cudaStream_t st, bool local = false, bool no_bitmap = false);
int prepare_evaluate_local();
int evaluate_local_blocks(int n);
int launch_batch_prepare(int N, int M, BatchState bs, Workspace ws, cudaStream_t st);
int launch_batch_small(const int *row_ptr, const int *col, const int *w, int sign, int max_n,
                       long long N, long long max_iters, int *queue, Workspace ws, BatchState bs,
                       cudaStream_t st);
int launch_batch_finish(int N, int sign, int Lbits, BatchState bs, Workspace ws, int64_t *num,
                        int32_t *den, int32_t *cycle_len, int32_t *cycle_out, int grid,
                        cudaStream_t st);
int launch_extract(int n, int Lstar, Workspace ws, int *cycle_out, int grid, int local_R,
                   cudaStream_t st);
// Transposed CSR (scc.cu); returns the number of kernels launched.
int launch_csc(const int *row_ptr, const int *col, int n, int m, int *in_ptr, int *in_src,
               int *cursor, int *bsum, cudaStream_t st);
// Single-lambda rebuild after an evaluation (single.cu); 1, or -1 on a launch failure.
int prepare_connect();
int launch_connect(const int *row_ptr, const int *col, const int *w, int sign, int n,
                   Workspace ws, SingleWs sw, cudaStream_t st);
void launch_outputs(int n, Workspace ws, int64_t *eta_num, int32_t *eta_den, int64_t *potential,
                    int32_t *policy, cudaStream_t st);
void launch_backward(const int *cycle_edges, int cycle_len, const float *grad_lambda, int m,
                     float *grad_w, cudaStream_t st);

}  // namespace ocm
