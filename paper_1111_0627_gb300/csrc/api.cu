// api.cu -- the C ABI declared in include/ocm.h: argument and CSR validation,
// workspace layout, the host loop of Howard's iteration (Alg. 2's host code,
// restructured: evaluate -> sweep -> stop when no vertex switched), the
// extraction of the critical cycle, and the backward scatter.
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace ocm {

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

size_t carve_workspace(void *base, int n, int m, Workspace *ws) {
    char *b = static_cast<char *>(base);
    size_t off = 0;
    const size_t N = static_cast<size_t>(n);
    const size_t T = (static_cast<size_t>(m) + kMinTileEdges - 1) / kMinTileEdges;
    auto take = [&](size_t bytes) -> void * {
        off = align_up(off, 256);
        void *p = b ? b + off : nullptr;
        off += bytes;
        return p;
    };
    Workspace w{};
    w.pi = static_cast<int *>(take(4 * N));
    w.succ = static_cast<int *>(take(4 * N));
    w.wpi = static_cast<int *>(take(4 * N));
    w.rec = static_cast<Rec *>(take(sizeof(Rec) * N));
    w.jm[0] = static_cast<JM *>(take(sizeof(JM) * N));
    w.jm[1] = static_cast<JM *>(take(sizeof(JM) * N));
    w.aprev = static_cast<int *>(take(4 * N));
    w.rep = static_cast<int *>(take(4 * N));
    w.jls[0] = static_cast<JLS *>(take(sizeof(JLS) * N));
    w.jls[1] = static_cast<JLS *>(take(sizeof(JLS) * N));
    for (int i = 0; i < 3; ++i) w.list[i] = static_cast<int *>(take(4 * N));
    w.cyc_root = static_cast<int *>(take(4 * N));
    w.cyc_p = static_cast<long long *>(take(8 * N));
    w.cyc_q = static_cast<int *>(take(4 * N));
    w.cyc_L = static_cast<int *>(take(4 * N));
    w.cyc_key = static_cast<long long *>(take(8 * N));
    w.cyc_rank = static_cast<int *>(take(4 * N));
    w.cid_of_root = static_cast<int *>(take(4 * N));
    w.done = static_cast<unsigned *>(take(4 * ((N + 31) / 32)));
    w.rec_dirty = static_cast<unsigned *>(take(4 * ((N + 31) / 32)));
    w.scratch16 = static_cast<int4 *>(take(sizeof(int4) * N));
    w.blk_tgt = static_cast<int2 *>(take(sizeof(int2) * ((N + kClassifyBlock - 1) / kClassifyBlock)));
    w.need_blk = static_cast<unsigned *>(
        take(4 * (((N + kClassifyBlock - 1) / kClassifyBlock + 31) / 32)));
    w.rec_dirty_blk = static_cast<unsigned *>(
        take(4 * (((N + kDirtyBlock - 1) / kDirtyBlock + 31) / 32)));
    w.sw_iter = static_cast<int *>(take(4 * N));
    w.cls_list = static_cast<int *>(take(4 * N));
    w.cls_hist = static_cast<int *>(take(4 * (size_t)kClassSlots * ((N + kClassifyBlock - 1) / kClassifyBlock)));
    w.band_grp = static_cast<int4 *>(
        take(sizeof(int4) * ((size_t)kClasses * ((N + kClassifyBlock - 1) / kClassifyBlock) + 1)));
    w.heavy_off = static_cast<int *>(take(4 * (N + 1)));
    w.heavy_part = static_cast<Cand *>(take(sizeof(Cand) * 2 * ((size_t)m / kHeavyChunk + 2)));
    w.tile_v = static_cast<int *>(take(4 * (T + 1)));
    w.tile_pend = static_cast<int *>(take(4 * T));
    w.tile_fopen = static_cast<int *>(take(4 * T));
    w.tile_first = static_cast<TilePart *>(take(sizeof(TilePart) * T));
    w.tile_last = static_cast<TilePart *>(take(sizeof(TilePart) * T));
    w.tpi = static_cast<int *>(take(4 * N));
    w.jt[0] = static_cast<long long *>(take(8 * N));
    w.jt[1] = static_cast<long long *>(take(8 * N));
    w.recp = static_cast<long long *>(take(8 * N));
    w.root_mark = static_cast<int *>(take(4 * N));
    w.chunk_info = static_cast<int2 *>(take(sizeof(int2) * (N / kEvalThreads + 2)));
    w.transit = nullptr;
    w.ctrl = static_cast<Ctrl *>(take(sizeof(Ctrl)));
    if (ws) *ws = w;
    return align_up(off, 256);
}

__global__ void ctrl_init_kernel(Ctrl *c, long long wait_ns, int frontier, int local_chunks) {
    Ctrl z;
    memset(&z, 0, sizeof z);
    z.bad_index = INT_MAX;
    z.wait_ns = wait_ns;
    z.frontier = frontier;
    z.local_chunks = local_chunks;
    *c = z;
}

__global__ void __launch_bounds__(kThreads)
zero_float_kernel(float *g, int m) {
    int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) g[i] = 0.0f;
}

__global__ void __launch_bounds__(kThreads)
cycle_grad_kernel(const int *cyc, int L, const float *gl, float *g, int m) {
    float val = __fdiv_rn(gl[0], (float)L);
    int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += stride) {
        int e = cyc[i];
        if ((unsigned)e < (unsigned)m) g[e] = val;
    }
}

// One warp per graph: every edge of graph g's critical cycle gets g's
// upstream gradient divided by the cycle length.
__global__ void __launch_bounds__(kThreads)
batch_cycle_grad_kernel(const int *vptr, const int *cyc, const int *clen, const float *gl, int G,
                        float *g, int m) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < G; k += warps) {
        const int L = clen[k];
        if (L < 1) continue;
        const float val = __fdiv_rn(gl[k], (float)L);
        const int base = vptr[k];
        for (int i = lane; i < L; i += 32) {
            const int e = cyc[base + i];
            if ((unsigned)e < (unsigned)m) g[e] = val;
        }
    }
}

// Cycle ratio: every edge of C* gets grad_lambda / t(C*); one block sums
// t(C*) and then scatters (the cycle is short next to the m-long zero fill).
__global__ void __launch_bounds__(kThreads)
cycle_grad_ratio_kernel(const int *cyc, int L, const int *transit, const float *gl, float *g,
                        int m) {
    __shared__ long long s_sum[kThreads / 32];
    long long T = 0;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const int e = cyc[i];
        if ((unsigned)e < (unsigned)m) T += transit[e];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) T += __shfl_xor_sync(0xffffffffu, T, o);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = T;
    __syncthreads();
    long long tot = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += s_sum[k];
    const float val = __fdiv_rn(gl[0], (float)tot);
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const int e = cyc[i];
        if ((unsigned)e < (unsigned)m) g[e] = val;
    }
}

void launch_backward(const int *cycle_edges, int cycle_len, const float *grad_lambda, int m,
                     float *grad_w, cudaStream_t st) {
    int blocks = (m + kThreads - 1) / kThreads;
    if (blocks > 8192) blocks = 8192;
    zero_float_kernel<<<blocks, kThreads, 0, st>>>(grad_w, m);
    int b2 = (cycle_len + kThreads - 1) / kThreads;
    if (b2 > 4096) b2 = 4096;
    if (b2 < 1) b2 = 1;
    cycle_grad_kernel<<<b2, kThreads, 0, st>>>(cycle_edges, cycle_len, grad_lambda, grad_w, m);
}

// ---------------------------------------------------------- profiling --
namespace {
struct ProfPair {
    int cls;
    cudaEvent_t a, b;
};
bool g_prof_on = false;
std::vector<cudaEvent_t> g_prof_free;
std::vector<ProfPair> g_prof_done;
cudaEvent_t g_prof_open = nullptr;
double g_prof_ms[kProfCount];
long long g_prof_n[kProfCount];

cudaEvent_t prof_event() {
    if (!g_prof_free.empty()) {
        cudaEvent_t e = g_prof_free.back();
        g_prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

thread_local bool t_prof_paused = false;

bool prof_active() { return g_prof_on && !t_prof_paused; }

ProfilePause::ProfilePause() : prev(t_prof_paused) { t_prof_paused = true; }
ProfilePause::~ProfilePause() { t_prof_paused = prev; }

void prof_begin(int cls, cudaStream_t st) {
    (void)cls;
    if (!prof_active()) return;
    g_prof_open = prof_event();
    if (g_prof_open) cudaEventRecord(g_prof_open, st);
}

void prof_end(int cls, cudaStream_t st) {
    if (!prof_active() || !g_prof_open) return;
    cudaEvent_t b = prof_event();
    if (!b) return;
    cudaEventRecord(b, st);
    g_prof_done.push_back(ProfPair{cls, g_prof_open, b});
    g_prof_open = nullptr;
}

NvtxRange::NvtxRange(const char *name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

// Host-side fault injection for tests of the error paths: the environment
// variable OCM_FAULT names one failure that the entry points then report as
// if the runtime or the input checks had produced it, before any device work
// of that step ("launch": a kernel launch fails, OCM_ERR_CUDA; "validate":
// the CSR checks fail, OCM_ERR_BAD_CSR; "alloc": the loop graph cannot be
// instantiated, so the solve falls back to the host-driven loop).  No GPU
// fault is ever made.
bool injected_fault(const char *what) {
    const char *e = getenv("OCM_FAULT");
    return e != nullptr && strcmp(e, what) == 0;
}

static int persistent_grid() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1024;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return 1024;
    return sms * 8;   // 8 resident 256-thread CTAs per SM
}

static int map_err_bits(int err) {
    if (err & kErrTimeout) return OCM_ERR_TIMEOUT;
    if (err & (kErrInitPolicy | kErrTransit | kErrUnreached)) return OCM_ERR_INVALID_ARG;
    if (err & kErrRatioKey) return OCM_ERR_OVERFLOW;
    if (err & (kErrRowPtr | kErrCol)) return OCM_ERR_BAD_CSR;
    if (err & kErrNoOutEdge) return OCM_ERR_NO_OUT_EDGE;
    if (err & kErrWeightMin) return OCM_ERR_OVERFLOW;
    if (err & kErrSweep) return OCM_ERR_INTERNAL;
    if (err) return OCM_ERR_INTERNAL;
    return OCM_OK;
}

static int read_ctrl(const Ctrl *dev, Ctrl *host, cudaStream_t st) {
    if (cudaMemcpyAsync(host, dev, sizeof(Ctrl), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return OCM_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return OCM_ERR_CUDA;
    return OCM_OK;
}

// ------------------------------------------------------ iteration loop --
// One improvement step is: evaluate the current policy, sweep every vertex
// for a better out-edge, (batched: retire the graphs that stopped changing),
// then the control kernel below.  The step reads its iteration index from
// the control block, so the same launches serve a host-driven loop and the
// body of a CUDA graph WHILE node.

// Ends a step: stop on an error or when no vertex switched (Howard's
// termination test, Alg. 1), else advance the iteration index unless the
// cap is reached.  With use_cond the decision also sets the WHILE node's
// condition.
__global__ void loop_control_kernel(Ctrl *c, long long max_iters, int use_cond,
                                    cudaGraphConditionalHandle handle) {
    // the next step's cooperative launches count their barriers from zero
    for (int i = 0; i < 2; ++i) {
        c->bar[i].arrive = 0;
        for (int j = 0; j < 4; ++j) {
            c->bar[i].sum[j] = 0;
            c->bar[i].sum2[j] = 0;
        }
    }
    c->switched_total += c->switched;
    int more = 0;
    if (c->err == 0 && c->changed) {
        if ((long long)c->iter + 1 >= max_iters) {
            c->not_converged = 1;
        } else {
            c->iter += 1;
            more = 1;
        }
    }
    c->loop_more = more;
    if (use_cond) cudaGraphSetConditional(handle, more ? 1u : 0u);
}

// Everything a step's launches depend on.
struct StepArgs {
    const int32_t *row_ptr, *col_idx, *w;
    int n, m, sign, threads, stall;
    int kind, epl;            // sweep layout (OCM_SWEEP_TILES, _CLASSES or _WINDOW) and its lane load
    int win_hb;               // window sweep: the window starts this many vertices before the tile
    int band_blocks;          // class sweep: classification blocks per band of its task order
    long long N2, max_iters;
    Workspace ws;
    BatchState bs;
    bool batch;
    bool single;              // the paper's single-lambda form: rebuild after each evaluation
    bool local;               // the two-level evaluation (locality of the policy graph)
    bool no_bitmap;           // (test) the two-level evaluation without its bitmaps
    SingleWs sg;
    int cls_cnt[kClassSlots];
    int heavy_edges;
};

// Launches one step; returns the number of kernels, or -1.
static int launch_step(const StepArgs &a, int use_cond, cudaGraphConditionalHandle handle,
                       cudaStream_t st) {
    int le = launch_evaluate(a.n, a.N2, a.ws, a.stall, a.bs, st, a.local, a.no_bitmap);
    if (le < 0) return -1;
    if (a.single) {
        if (launch_connect(a.row_ptr, a.col_idx, a.w, a.sign, a.n, a.ws, a.sg, st) < 0) return -1;
        le += 1;
    }
    const int ks = (a.kind == OCM_SWEEP_TILES)
                       ? launch_sweep_tiles(a.row_ptr, a.col_idx, a.w, a.sign, a.n, a.m, a.epl,
                                            a.ws, a.bs, a.threads, st)
                   : (a.kind == OCM_SWEEP_WINDOW)
                       ? launch_sweep_window(a.row_ptr, a.col_idx, a.w, a.sign, a.n, a.epl,
                                             a.win_hb, a.ws, a.cls_cnt, a.heavy_edges, a.bs, st)
                       : launch_sweep(a.row_ptr, a.col_idx, a.w, a.sign, a.n, a.ws, a.cls_cnt,
                                      a.heavy_edges, a.bs, a.threads, a.band_blocks, st);
    if (ks < 0) return -1;
    int k = le + ks;
    if (a.batch) k += launch_batch_converge(a.bs, a.ws, st);
    loop_control_kernel<<<1, 1, 0, st>>>(a.ws.ctrl, a.max_iters, use_cond, handle);
    k += 1;
    if (cudaGetLastError() != cudaSuccess) return -1;
    return k;
}

namespace {

// Instantiated loop graphs, keyed by everything their kernel nodes bake in.
struct LoopKey {
    int dev;
    const void *row_ptr, *col_idx, *w, *ctrl, *vptr, *transit;
    int n, m, sign, threads, stall, G, kind, epl, single, heavy_edges, local, no_bitmap, win_hb,
        band_blocks;
    long long N2, max_iters;
    int cls_cnt[kClassSlots];
    bool operator==(const LoopKey &o) const {
        if (dev != o.dev || row_ptr != o.row_ptr || col_idx != o.col_idx || w != o.w ||
            ctrl != o.ctrl || vptr != o.vptr || transit != o.transit || n != o.n || m != o.m ||
            sign != o.sign || single != o.single || local != o.local ||
            no_bitmap != o.no_bitmap ||
            threads != o.threads || stall != o.stall || G != o.G || kind != o.kind ||
            win_hb != o.win_hb || band_blocks != o.band_blocks ||
            epl != o.epl || N2 != o.N2 || max_iters != o.max_iters || heavy_edges != o.heavy_edges)
            return false;
        for (int c = 0; c < kClassSlots; ++c)
            if (cls_cnt[c] != o.cls_cnt[c]) return false;
        return true;
    }
};

struct LoopEntry {
    bool valid;
    LoopKey key;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int kernels;              // kernels per step
    int busy;                 // launches in flight from callers that have not synchronised yet
    unsigned long long stamp; // last use, for eviction
};

constexpr int kLoopCache = 16;
std::mutex g_loop_mutex;
LoopEntry g_loops[kLoopCache];   // never destroyed: the runtime may be gone at exit
unsigned long long g_loop_clock = 0;

LoopKey make_key(const StepArgs &a) {
    LoopKey k;
    memset(&k, 0, sizeof k);
    cudaGetDevice(&k.dev);
    k.row_ptr = a.row_ptr;
    k.col_idx = a.col_idx;
    k.w = a.w;
    k.ctrl = a.ws.ctrl;
    k.vptr = a.bs.vptr;
    k.transit = a.ws.transit;
    k.n = a.n;
    k.m = a.m;
    k.kind = a.kind;
    k.epl = a.epl;
    k.win_hb = a.win_hb;
    k.band_blocks = a.band_blocks;
    k.sign = a.sign;
    k.threads = a.threads;
    k.stall = a.stall;
    k.G = a.bs.G;
    k.single = a.single ? 1 : 0;
    k.local = a.local ? 1 : 0;
    k.no_bitmap = a.no_bitmap ? 1 : 0;
    k.N2 = a.N2;
    k.max_iters = a.max_iters;
    for (int c = 0; c < kClassSlots; ++c) k.cls_cnt[c] = a.cls_cnt[c];
    k.heavy_edges = a.heavy_edges;
    return k;
}

// A graph holding one WHILE node whose body is one step, captured from the
// same launch code the host loop uses.
bool build_loop_graph(const StepArgs &a, LoopEntry *e) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    cudaStream_t cs = nullptr;
    bool ok = false;
    do {
        if (cudaGraphCreate(&g, 0) != cudaSuccess) break;
        cudaGraphConditionalHandle handle;
        // default value 1 at every launch: the body runs at least once
        if (cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault) !=
            cudaSuccess)
            break;
        cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
        p.conditional.handle = handle;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p) != cudaSuccess) break;
        cudaGraph_t body = p.conditional.phGraph_out[0];
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) break;
        if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed) != cudaSuccess)
            break;
        const int k = launch_step(a, 1, handle, cs);
        cudaGraph_t captured = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(cs, &captured);
        if (k < 0 || ec != cudaSuccess) break;
        if (cudaGraphInstantiate(&x, g, 0) != cudaSuccess) break;
        e->kernels = k;
        ok = true;
    } while (false);
    if (cs) cudaStreamDestroy(cs);
    if (!ok) {
        if (x) cudaGraphExecDestroy(x);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();   // a refused capture is not sticky; clear it
        return false;
    }
    e->graph = g;
    e->exec = x;
    return true;
}

// Cached (or newly built) loop graph for these arguments, marked busy; -1 if
// none can be had (every slot busy, or the build failed).
int acquire_loop(const StepArgs &a) {
    const LoopKey key = make_key(a);
    std::lock_guard<std::mutex> lock(g_loop_mutex);
    ++g_loop_clock;
    for (int i = 0; i < kLoopCache; ++i) {
        if (g_loops[i].valid && g_loops[i].key == key) {
            g_loops[i].busy += 1;
            g_loops[i].stamp = g_loop_clock;
            return i;
        }
    }
    int slot = -1;
    for (int i = 0; i < kLoopCache; ++i) {
        if (!g_loops[i].valid) {
            slot = i;
            break;
        }
        if (g_loops[i].busy == 0 && (slot < 0 || g_loops[i].stamp < g_loops[slot].stamp)) slot = i;
    }
    if (slot < 0) return -1;
    LoopEntry &e = g_loops[slot];
    if (e.valid) {
        // idle: every caller that launched it has synchronised its stream
        cudaGraphExecDestroy(e.exec);
        cudaGraphDestroy(e.graph);
        e.valid = false;
    }
    if (!build_loop_graph(a, &e)) return -1;
    e.valid = true;
    e.key = key;
    e.busy = 1;
    e.stamp = g_loop_clock;
    return slot;
}

void release_loop(int slot) {
    std::lock_guard<std::mutex> lock(g_loop_mutex);
    g_loops[slot].busy -= 1;
}

}  // namespace

}  // namespace ocm

using namespace ocm;

extern "C" {

size_t ocm_workspace_size(int32_t n, int32_t m) {
    if (n < 1 || m < 1) return 0;
    return carve_workspace(nullptr, n, m, nullptr);
}

const char *ocm_status_string(int status) {
    switch (status) {
        case OCM_OK: return "ok";
        case OCM_ERR_INVALID_ARG: return "invalid argument";
        case OCM_ERR_BAD_CSR: return "malformed CSR (row_ptr or col_idx)";
        case OCM_ERR_NO_OUT_EDGE: return "a vertex has no out-edge";
        case OCM_ERR_OVERFLOW: return "weights out of the exact range (INT32_MIN or 2 n^2 max|w| >= 2^62)";
        case OCM_ERR_NOT_CONVERGED: return "iteration cap reached";
        case OCM_ERR_TIMEOUT: return "a bounded device-side wait gave up";
        case OCM_ERR_WORKSPACE: return "workspace missing, too small or not 256-byte aligned";
        case OCM_ERR_CUDA: return "CUDA runtime error";
        case OCM_ERR_INTERNAL: return "internal consistency check failed";
        default: return "unknown status";
    }
}

int ocm_version(void) { return 112; }

int ocm_profile_enable(int on) {
    int prev = g_prof_on ? 1 : 0;
    g_prof_on = on != 0;
    return prev;
}

int ocm_profile_collect(double *ms_out, int64_t *launches_out) {
    for (const ProfPair &p : g_prof_done) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_prof_ms[p.cls] += ms;
            g_prof_n[p.cls] += 1;
        }
        g_prof_free.push_back(p.a);
        g_prof_free.push_back(p.b);
    }
    g_prof_done.clear();
    for (int c = 0; c < kProfCount; ++c) {
        if (ms_out) ms_out[c] = g_prof_ms[c];
        if (launches_out) launches_out[c] = g_prof_n[c];
        g_prof_ms[c] = 0.0;
        g_prof_n[c] = 0;
    }
    return kProfCount;
}

}  // extern "C"

namespace ocm {

// Outputs of one solve: a single graph (host scalars) or a batch (device arrays).
struct SolveOut {
    int64_t *num;
    int32_t *den;
    int32_t *cycle_len;
    int32_t *cycle_out;
};

// The whole solve; bs == nullptr for a single graph.
static int solve_impl(const int32_t *row_ptr, const int32_t *col_idx, const int32_t *w, int32_t n,
                      int32_t m, int mode, SolveOut out, void *workspace, size_t ws_bytes,
                      size_t need, void *stream, const ocm_options *opt, ocm_stats *stats,
                      BatchState *bs) {
    if (ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return OCM_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Workspace ws;
    carve_workspace(workspace, n, m, &ws);
    ws.transit = opt ? opt->transit : nullptr;   // optimal cycle ratio when set
    const bool ratio = ws.transit != nullptr;
    // the paper's single-lambda form (single graphs only): its extra state
    // follows the workspace
    const bool single = !bs && opt && (opt->flags & OCM_FLAG_SINGLE_LAMBDA);
    SingleWs sg{};
    if (single) carve_single(static_cast<char *>(workspace) + ocm_workspace_size(n, m), n, m, &sg);
    const int sign = (mode == OCM_MAX) ? 1 : -1;
    const int grid = persistent_grid();
    long long launches = 0;
    Ctrl h;
    BatchState none{};
    BatchState b = bs ? *bs : none;

    // Limit of every device-side wait: the caller's, else two seconds (10 ms
    // for the test-only stall, which can only run out).
    long long wait_ns = kDefaultWaitNs;
    if (opt && opt->wait_limit_ms > 0) wait_ns = (long long)opt->wait_limit_ms * 1000000LL;
    else if (opt && (opt->flags & OCM_FLAG_TEST_STALL)) wait_ns = kStallTestWaitNs;

    // 1. row_ptr (and the graph offsets) must be sane before any kernel trusts them
    NvtxRange r_all(bs ? "ocm_solve_batch" : "ocm_solve");
    if (injected_fault("launch")) return OCM_ERR_CUDA;
    if (injected_fault("validate")) return OCM_ERR_BAD_CSR;
    auto phase = [](const char *name) { nvtxRangePop(); nvtxRangePushA(name); };
    nvtxRangePushA("ocm:validate");
    struct PopOnExit { ~PopOnExit() { nvtxRangePop(); } } pop_phase;
    // the frontier sweep: not in the single-lambda form, whose rebuild writes
    // records after the record pass
    const int frontier =
        single ? 0 : (opt && (opt->flags & OCM_FLAG_TEST_FRONTIER)) ? 2 : 1;
    const int local_chunks = !opt                                         ? 1
                             : (opt->flags & OCM_FLAG_TEST_NO_LOCAL_CHUNKS) ? 0
                             : (opt->flags & OCM_FLAG_TEST_LOCAL_CHUNKS)    ? 2
                                                                           : 1;
    ctrl_init_kernel<<<1, 1, 0, st>>>(ws.ctrl, wait_ns, frontier, local_chunks);
    launch_check_row_ptr(row_ptr, n, m, ws.ctrl, st);
    launches += 2;
    if (bs) launches += launch_batch_prepare(n, m, b, ws, st);
    if (cudaGetLastError() != cudaSuccess) return OCM_ERR_CUDA;
    int rc = read_ctrl(ws.ctrl, &h, st);
    if (rc) return rc;
    if (h.err) return map_err_bits(h.err);

    phase("ocm:init_policy");
    // 2. degree classes of the improvement sweep (and the heavy vertices), then
    //    the initial policy (the paper's first pass from val = 0, lambda = 0),
    //    which also validates col_idx and w and measures max|w|
    // (the edge-tiled sweep has no cycle-ratio form)
    // (the window sweep is decided after the initial pass, which measures the
    // locality it relies on; it groups vertices by the same degree classes)
    const int req_kind = opt ? opt->sweep_kind : OCM_SWEEP_DEFAULT;
    int kind = (req_kind == OCM_SWEEP_TILES && !ratio) ? OCM_SWEEP_TILES : OCM_SWEEP_CLASSES;
    int epl = (opt && opt->edges_per_lane > 0) ? opt->edges_per_lane : kEdgesPerLane;
    if (epl > 64) epl = 64;
    if (kind == OCM_SWEEP_TILES) epl = epl <= 4 ? 4 : 8;
    const int sweep_threads = (opt && opt->sweep_threads > 0) ? opt->sweep_threads : kSweepThreads;
    // bands of the class sweep's task order (one band up to 2^22 vertices)
    const int band_blocks =
        (opt && (opt->flags & OCM_FLAG_TEST_SMALL_BANDS)) ? 1 : sweep_band_blocks(n);
    launches += launch_classify(row_ptr, n, kind == OCM_SWEEP_TILES ? kEdgesPerLane : epl,
                                band_blocks, ws, st);
    if (kind == OCM_SWEEP_TILES) launches += launch_tile_index(row_ptr, n, m, 32 * epl, ws, st);
    // the two-level evaluation serves single graphs whose edges mostly stay
    // inside the evaluation grid's block ranges (or when forced); the initial
    // pass counts those edges
    const int eval_flags = opt ? opt->flags & (OCM_FLAG_EVAL_LOCAL | OCM_FLAG_EVAL_GLOBAL) : 0;
    const bool local_ok = !bs && !ratio && !single && !(eval_flags & OCM_FLAG_EVAL_GLOBAL);
    int local_R = 0;
    if (local_ok) {
        const int blocks = evaluate_local_blocks(n);
        if (blocks <= 0) return OCM_ERR_CUDA;
        local_R = (n + blocks - 1) / blocks;
    }
    launch_init_policy(row_ptr, col_idx, w, sign, n, m, opt ? opt->init_policy : nullptr, ws,
                       bs ? &b : nullptr, st, local_R,
                       (req_kind == OCM_SWEEP_WINDOW && kind == OCM_SWEEP_CLASSES && !ratio) ? 1
                                                                                            : 0,
                       band_blocks);
    launches += 3;
    if (cudaGetLastError() != cudaSuccess) return OCM_ERR_CUDA;
    rc = read_ctrl(ws.ctrl, &h, st);
    if (rc) return rc;
    if (h.err) return map_err_bits(h.err);
    // Cycles never span graphs, so the largest cycle length (and denominator)
    // is bounded by the largest graph.  Exactness bound: 2 n_max^2 max|w| <
    // 2^62 keeps every value, key and cross product inside int64.  Cycle
    // ratio: values q*S - p*T and keys q*w - p*t + V are bounded by
    // 4 n_max^2 max|w| max t, and a cycle's time n_max max t must fit int32.
    const long long nmax = bs ? h.max_ng : n;
    {
        unsigned __int128 bound = (unsigned __int128)2 * (unsigned long long)nmax *
                                  (unsigned long long)nmax * (unsigned)h.maxabsw;
        if (ratio) bound *= 2 * (unsigned __int128)(unsigned)h.maxt;
        if (bound >= ((unsigned __int128)1 << 62)) return OCM_ERR_OVERFLOW;
        if (ratio && (unsigned long long)nmax * (unsigned)h.maxt > 0x7fffffffULL)
            return OCM_ERR_OVERFLOW;
    }
    const long long N2 = nmax * nmax;
    // the window sweep (asked for; the mean only): the window placement that
    // holds the most edges
    int win_hb = 0;
    if (kind == OCM_SWEEP_CLASSES && !ratio && req_kind == OCM_SWEEP_WINDOW) {
        int best = 0;
        for (int j = 1; j < kWinShapes; ++j)
            if (h.win_edges[j] > h.win_edges[best]) best = j;
        kind = OCM_SWEEP_WINDOW;
        win_hb = best * kWinTile;
    }
    const long long max_iters = (opt && opt->max_iters > 0) ? opt->max_iters : 4LL * n + 64;
    if (single) {
        // the backward search of the rebuild walks the transposed graph
        // (col_idx was validated above)
        launches += launch_csc(row_ptr, col_idx, n, m, sg.in_ptr, sg.in_src, sg.cursor, sg.bsum,
                               st);
        if (cudaGetLastError() != cudaSuccess) return OCM_ERR_CUDA;
    }

    phase("ocm:iterate");
    // 2b. batch: the small graphs, one thread block each for all their
    //     iterations (largest first); the union loop below skips them.  Not
    //     with transit times or per-vertex outputs, which the union path
    //     serves for every graph.
    if (bs) {
        const int small_n = opt ? opt->batch_small_vertices : 0;   // 0: automatic
        const bool outputs = opt && (opt->eta_num || opt->eta_den || opt->potential || opt->policy);
        if (small_n >= 0 && !ratio && !outputs) {
            const int k = launch_batch_small(row_ptr, col_idx, w, sign, small_n, n, max_iters,
                                             b.small_queue, ws, b, st);
            if (k < 0) return OCM_ERR_CUDA;
            launches += k;
        }
    }

    // 3. Howard iteration: evaluate the policy, sweep, stop when stable --
    //    as one launch of the cached loop graph, or driven from the host
    StepArgs sa;
    sa.row_ptr = row_ptr;
    sa.col_idx = col_idx;
    sa.w = w;
    sa.n = n;
    sa.m = m;
    sa.kind = kind;
    sa.epl = epl;
    sa.win_hb = win_hb;
    sa.band_blocks = band_blocks;
    sa.sign = sign;
    sa.threads = (sweep_threads == 64 || sweep_threads == 128 || sweep_threads == 256 ||
                  sweep_threads == 512) ? sweep_threads : kSweepThreads;
    sa.stall = (opt && (opt->flags & OCM_FLAG_TEST_STALL)) ? 1 : 0;
    sa.N2 = N2;
    sa.max_iters = max_iters;
    sa.ws = ws;
    sa.bs = b;
    sa.batch = bs != nullptr;
    sa.single = single;
    sa.local = local_ok && ((eval_flags & OCM_FLAG_EVAL_LOCAL) ||
                            (n >= kLocalEvalMinN &&
                             (double)h.local_edges >= kLocalEvalMinFraction * (double)m));
    sa.no_bitmap = opt && (opt->flags & OCM_FLAG_TEST_NO_BITMAP);
    sa.sg = sg;
    for (int c = 0; c < kClassSlots; ++c) sa.cls_cnt[c] = h.cls_cnt[c];
    sa.heavy_edges = (kind == OCM_SWEEP_TILES) ? 0 : h.heavy_edges;
    if ((single && prepare_connect() != 0) || prepare_evaluate(ratio) != 0 ||
        (sa.local && prepare_evaluate_local() != 0) ||
        (kind == OCM_SWEEP_TILES    ? prepare_sweep_tiles(epl, sa.threads)
         : kind == OCM_SWEEP_WINDOW ? prepare_sweep_window()
                                    : prepare_sweep_classes(sa.threads, ratio)) != 0)
        return OCM_ERR_CUDA;
    const bool host_loop = (opt && (opt->flags & OCM_FLAG_HOST_LOOP)) || prof_active();
    // (a failed instantiation of the loop graph falls back to the host loop)
    const int slot = (host_loop || injected_fault("alloc")) ? -1 : acquire_loop(sa);
    if (slot >= 0) {
        const cudaError_t e = cudaGraphLaunch(g_loops[slot].exec, st);
        rc = (e == cudaSuccess) ? read_ctrl(ws.ctrl, &h, st) : OCM_ERR_CUDA;
        const int per_step = g_loops[slot].kernels;
        release_loop(slot);
        if (rc) return rc;
        launches += (long long)per_step * (h.iter + 1);
    } else {
        for (;;) {
            const int k = launch_step(sa, 0, 0, st);
            if (k < 0) return OCM_ERR_CUDA;
            launches += k;
            rc = read_ctrl(ws.ctrl, &h, st);
            if (rc) return rc;
            if (!h.loop_more) break;
        }
    }
    if (h.err) return map_err_bits(h.err);
    if (h.not_converged) return OCM_ERR_NOT_CONVERGED;
    const long long it = h.iter;

    phase("ocm:extract");
    // 4. critical cycle(s) of the final policy
    int Lstar = 0;
    if (bs) {
        int bits = 0;
        while ((1LL << bits) <= nmax) ++bits;
        launches += launch_batch_finish(n, sign, bits, b, ws, out.num, out.den, out.cycle_len,
                                        out.cycle_out, grid, st);
    } else {
        Lstar = h.res_len;
        if (Lstar < 1 || Lstar > n) return OCM_ERR_INTERNAL;
        // (after the two-level evaluation: its block range size, for the
        // segment walk along the cycle)
        int local_R = 0;
        if (sa.local) {
            const int eb = evaluate_local_blocks(n);
            if (eb > 0) local_R = (n + eb - 1) / eb;
        }
        launches += launch_extract(n, Lstar, ws, out.cycle_out, grid, local_R, st);
    }
    if (opt && (opt->eta_num || opt->eta_den || opt->potential || opt->policy)) {
        launch_outputs(n, ws, opt->eta_num, opt->eta_den, opt->potential, opt->policy, st);
        launches += 1;
    }
    if (cudaGetLastError() != cudaSuccess) return OCM_ERR_CUDA;
    Ctrl fin;
    rc = read_ctrl(ws.ctrl, &fin, st);
    if (rc) return rc;
    if (fin.err) return map_err_bits(fin.err);
    if (!bs) {
        if (fin.cnt[0] != Lstar) return OCM_ERR_INTERNAL;
        *out.num = (int64_t)sign * (int64_t)h.res_num;
        *out.den = h.res_den;
        *out.cycle_len = Lstar;
    }
    if (stats) {
        stats->iterations = (int32_t)(it > fin.small_iters ? it : fin.small_iters);
        stats->cycles = h.res_cycles;
        stats->detect_rounds = fin.rounds_detect;
        stats->value_rounds = fin.rounds_value;
        stats->switched = h.switched_total;
        stats->launches = launches;
        stats->detect_items = fin.items_detect;
        stats->value_items = fin.items_value;
        stats->graph_loop = slot >= 0 ? 1 : 0;
        stats->rebuild_levels = fin.connect_levels;
        stats->batch_small_graphs = fin.small_total;
        stats->sweep_kind = kind;
    }
    return OCM_OK;
}

// Batch workspace: the single-graph layout for all N vertices, then the
// per-vertex graph ids and the per-graph records.
static size_t batch_extra(int G, int N, BatchState *bs, char *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        off = align_up(off, 256);
        void *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    BatchState b{};
    b.gid = static_cast<int *>(take(4 * (size_t)N));
    b.gbest = static_cast<unsigned long long *>(take(8 * (size_t)G));
    b.groot = static_cast<int *>(take(4 * (size_t)G));
    b.glen = static_cast<int *>(take(4 * (size_t)G));
    b.gfound = static_cast<int *>(take(4 * (size_t)G));
    b.gp = static_cast<long long *>(take(8 * (size_t)G));
    b.gq = static_cast<int *>(take(4 * (size_t)G));
    b.gconv = static_cast<int *>(take(4 * (size_t)G));
    b.gsw = static_cast<int *>(take(4 * (size_t)G));
    b.small_queue = static_cast<int *>(take(4 * (size_t)G));
    b.G = G;
    if (bs) *bs = b;
    return align_up(off, 256);
}

}  // namespace ocm

extern "C" {

size_t ocm_workspace_size_single(int32_t n, int32_t m) {
    if (n < 1 || m < 1) return 0;
    return carve_workspace(nullptr, n, m, nullptr) + carve_single(nullptr, n, m, nullptr);
}

int ocm_solve(const int32_t *row_ptr, const int32_t *col_idx, const int32_t *w, int32_t n,
              int32_t m, int mode, int64_t *num, int32_t *den, int32_t *cycle_out,
              int32_t *cycle_len, void *workspace, size_t ws_bytes, void *stream,
              const ocm_options *opt, ocm_stats *stats) {
    if (!row_ptr || !col_idx || !w || !num || !den || !cycle_out || !cycle_len) return OCM_ERR_INVALID_ARG;
    if (n < 1 || m < 1 || (mode != OCM_MAX && mode != OCM_MIN)) return OCM_ERR_INVALID_ARG;
    if (opt && (opt->flags & ~(OCM_FLAG_TEST_STALL | OCM_FLAG_HOST_LOOP | OCM_FLAG_SINGLE_LAMBDA |
                               OCM_FLAG_EVAL_LOCAL | OCM_FLAG_EVAL_GLOBAL |
                               OCM_FLAG_TEST_NO_BITMAP | OCM_FLAG_TEST_SMALL_BANDS |
                               OCM_FLAG_TEST_FRONTIER | OCM_FLAG_TEST_LOCAL_CHUNKS |
                               OCM_FLAG_TEST_NO_LOCAL_CHUNKS)))
        return OCM_ERR_INVALID_ARG;
    if (opt && (opt->flags & OCM_FLAG_EVAL_LOCAL) && (opt->flags & OCM_FLAG_EVAL_GLOBAL))
        return OCM_ERR_INVALID_ARG;
    if (opt && (opt->flags & OCM_FLAG_TEST_LOCAL_CHUNKS) &&
        (opt->flags & OCM_FLAG_TEST_NO_LOCAL_CHUNKS))
        return OCM_ERR_INVALID_ARG;
    const bool single = opt && (opt->flags & OCM_FLAG_SINGLE_LAMBDA);
    if (opt && (opt->sweep_kind < OCM_SWEEP_DEFAULT || opt->sweep_kind > OCM_SWEEP_WINDOW))
        return OCM_ERR_INVALID_ARG;
    if (!workspace) return OCM_ERR_WORKSPACE;
    SolveOut out{num, den, cycle_len, cycle_out};
    return solve_impl(row_ptr, col_idx, w, n, m, mode, out, workspace, ws_bytes,
                      single ? ocm_workspace_size_single(n, m) : ocm_workspace_size(n, m), stream,
                      opt, stats, nullptr);
}

size_t ocm_workspace_size_batch(int32_t G, int32_t N, int32_t M) {
    if (G < 1 || N < G || M < 1) return 0;
    return ocm_workspace_size(N, M) + batch_extra(G, N, nullptr, nullptr);
}

int ocm_solve_batch(const int32_t *graph_vptr, const int32_t *row_ptr, const int32_t *col_idx,
                    const int32_t *w, int32_t G, int32_t N, int32_t M, int mode, int64_t *num,
                    int32_t *den, int32_t *cycle_len, int32_t *cycle_out, void *workspace,
                    size_t ws_bytes, void *stream, const ocm_options *opt, ocm_stats *stats) {
    if (!graph_vptr || !row_ptr || !col_idx || !w || !num || !den || !cycle_len || !cycle_out)
        return OCM_ERR_INVALID_ARG;
    if (G < 1 || N < G || M < 1 || (mode != OCM_MAX && mode != OCM_MIN)) return OCM_ERR_INVALID_ARG;
    if (opt && (opt->flags & ~(OCM_FLAG_TEST_STALL | OCM_FLAG_HOST_LOOP | OCM_FLAG_TEST_SMALL_BANDS |
                               OCM_FLAG_TEST_FRONTIER)))
        return OCM_ERR_INVALID_ARG;
    if (opt && (opt->sweep_kind < OCM_SWEEP_DEFAULT || opt->sweep_kind > OCM_SWEEP_WINDOW))
        return OCM_ERR_INVALID_ARG;
    if (!workspace) return OCM_ERR_WORKSPACE;
    const size_t base = ocm_workspace_size(N, M);
    const size_t need = ocm_workspace_size_batch(G, N, M);
    if (ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return OCM_ERR_WORKSPACE;
    BatchState bs;
    batch_extra(G, N, &bs, static_cast<char *>(workspace) + base);
    bs.vptr = graph_vptr;
    SolveOut out{num, den, cycle_len, cycle_out};
    return solve_impl(row_ptr, col_idx, w, N, M, mode, out, workspace, ws_bytes, base, stream, opt,
                      stats, &bs);
}

int ocm_backward_batch(const int32_t *graph_vptr, const int32_t *cycle_out,
                       const int32_t *cycle_len, const float *grad_lambda, int32_t G, int32_t M,
                       float *grad_w, void *stream) {
    if (!graph_vptr || !cycle_out || !cycle_len || !grad_lambda || !grad_w) return OCM_ERR_INVALID_ARG;
    if (G < 1 || M < 1) return OCM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int blocks = (M + kThreads - 1) / kThreads;
    if (blocks > 8192) blocks = 8192;
    zero_float_kernel<<<blocks, kThreads, 0, st>>>(grad_w, M);
    int gb = (G * 32 + kThreads - 1) / kThreads;
    if (gb > 4096) gb = 4096;
    batch_cycle_grad_kernel<<<gb, kThreads, 0, st>>>(graph_vptr, cycle_out, cycle_len, grad_lambda,
                                                     G, grad_w, M);
    if (cudaGetLastError() != cudaSuccess) return OCM_ERR_CUDA;
    return OCM_OK;
}

int ocm_backward_ratio(const int32_t *cycle_edges, int32_t cycle_len, const int32_t *transit,
                       const float *grad_lambda, int32_t m, float *grad_w, void *stream) {
    if (!cycle_edges || !transit || !grad_lambda || !grad_w) return OCM_ERR_INVALID_ARG;
    if (m < 1 || cycle_len < 1 || cycle_len > m) return OCM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int blocks = (m + kThreads - 1) / kThreads;
    if (blocks > 8192) blocks = 8192;
    zero_float_kernel<<<blocks, kThreads, 0, st>>>(grad_w, m);
    cycle_grad_ratio_kernel<<<1, kThreads, 0, st>>>(cycle_edges, cycle_len, transit, grad_lambda,
                                                    grad_w, m);
    if (cudaGetLastError() != cudaSuccess) return OCM_ERR_CUDA;
    return OCM_OK;
}

int ocm_backward(const int32_t *cycle_edges, int32_t cycle_len, const float *grad_lambda,
                 int32_t m, float *grad_w, void *stream) {
    if (!cycle_edges || !grad_lambda || !grad_w) return OCM_ERR_INVALID_ARG;
    if (m < 1 || cycle_len < 1 || cycle_len > m) return OCM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    launch_backward(cycle_edges, cycle_len, grad_lambda, m, grad_w, st);
    if (cudaGetLastError() != cudaSuccess) return OCM_ERR_CUDA;
    return OCM_OK;
}

}  // extern "C"
