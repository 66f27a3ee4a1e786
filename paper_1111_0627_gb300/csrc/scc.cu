// scc.cu -- strongly connected components on the GPU, and the optimal cycle
// mean of every component that holds a cycle, solved as one batch.
//
// The paper prepends an SCC decomposition to its solver (Sec. 3.3): by
// Prop. 2.2 the optimal cycle mean of a graph is the optimum over its
// components, every cycle lies inside one component, and the components can
// be solved concurrently as regions.  Here the decomposition is a
// forward-backward search with trimming over colour classes:
//   trim      a vertex with no active out-neighbour or no active in-neighbour
//             of its own class lies on no cycle of the class: it is a
//             component by itself;
//   pivot     every class picks its largest active vertex;
//   FW / BW   breadth-first searches from the pivots along out-edges and
//             along in-edges (a transposed CSR built once), inside the class;
//   split     FW and BW reached: the pivot's component; FW only, BW only,
//             neither: three new classes (every component lies wholly in one).
// One cooperative launch runs an iteration (its BFS levels separated by the
// bounded grid barrier); the host repeats iterations until no vertex is
// active.  Each component is labelled by its smallest vertex, so the labels
// do not depend on the order in which components are found.
//
// The per-component solve relabels the vertices of the components that hold a
// cycle so that each component is a contiguous range in increasing vertex
// order (a stable radix sort by label), keeps only the edges inside
// components, and hands the result to the batched solver: each component is
// solved exactly as its induced subgraph with its vertices in their original
// order would be.
#include <climits>
#include <cstring>

#include "common.cuh"
#include "grid_sync.cuh"

namespace ocm {

constexpr int kSccThreads = 1024;   // one block per SM: fewer arrivals at each grid barrier
constexpr int kSortThreads = 512;
constexpr int kScanBlock = 1024;
constexpr int kTrimRounds = 8;
constexpr int kActive = 1, kFw = 2, kBw = 4;
// A frontier vertex with more edges than this in the search direction goes to
// a heavy frontier, whose vertices are expanded by the whole grid together.
constexpr int kSccHeavy = 2048;

// Workspace of the decomposition, carved from one caller buffer.
struct SccWs {
    int *in_ptr;     // [n+1] CSC offsets
    int *in_src;     // [m] source vertex of each in-edge
    int *cursor;     // [n] CSC scatter cursors
    int *bsum;       // [n / kScanBlock + 1] block sums of the scans
    int *color;      // [n] colour class (3p + k after a split at pivot p; 3n at first)
    int *flags;      // [n] kActive | kFw | kBw
    int *piv;        // [3n + 1] pivot of each class
    int *minv;       // [n] smallest vertex of the component found from pivot p
    int *q[4];       // [n] BFS frontiers: forward 0/1, backward 2/3
    int *hq[4];      // [m / kSccHeavy + 2] heavy frontiers, the same order
    Ctrl *ctrl;
};

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

static size_t carve_scc(void *base, int n, int m, SccWs *ws) {
    char *b = static_cast<char *>(base);
    size_t off = 0;
    const size_t N = (size_t)n, M = (size_t)m;
    auto take = [&](size_t bytes) -> void * {
        off = align256(off);
        void *p = b ? b + off : nullptr;
        off += bytes;
        return p;
    };
    SccWs w{};
    w.in_ptr = static_cast<int *>(take(4 * (N + 1)));
    w.in_src = static_cast<int *>(take(4 * (M > 0 ? M : 1)));
    w.cursor = static_cast<int *>(take(4 * N));
    w.bsum = static_cast<int *>(take(4 * (N / kScanBlock + 2)));
    w.color = static_cast<int *>(take(4 * N));
    w.flags = static_cast<int *>(take(4 * N));
    w.piv = static_cast<int *>(take(4 * (3 * N + 1)));
    w.minv = static_cast<int *>(take(4 * N));
    for (int i = 0; i < 4; ++i) w.q[i] = static_cast<int *>(take(4 * N));
    for (int i = 0; i < 4; ++i) w.hq[i] = static_cast<int *>(take(4 * (M / kSccHeavy + 2)));
    w.ctrl = static_cast<Ctrl *>(take(sizeof(Ctrl)));
    if (ws) *ws = w;
    return align256(off);
}

// ------------------------------------------------------------ device scan --
// In-place inclusive scan of a[0..len) in three launches: per-block scans
// with block totals, one block scanning the totals, and the carry-in.
__global__ void __launch_bounds__(kScanBlock) scan_blocks_kernel(int *a, int len, int *bsum) {
    __shared__ int s_warp[32];
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = i < len ? a[i] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int wv = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wv, o);
            if (lane >= o) wv += y;
        }
        s_warp[lane] = wv;
    }
    __syncthreads();
    if (warp > 0) x += s_warp[warp - 1];
    if (i < len) a[i] = x;
    if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = x;
}

__global__ void __launch_bounds__(kScanBlock) scan_totals_kernel(int *bsum, int nb) {
    // exclusive scan of the block totals by one block, kScanBlock at a time
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += kScanBlock) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? bsum[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int wv = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wv, o);
                if (lane >= o) wv += y;
            }
            s_warp[lane] = wv;
        }
        __syncthreads();
        const int incl = x + (warp > 0 ? s_warp[warp - 1] : 0);
        if (i < nb) bsum[i] = s_carry + incl - v;
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) s_carry += incl;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanBlock) scan_carry_kernel(int *a, int len, const int *bsum) {
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    if (i < len && blockIdx.x > 0) a[i] += bsum[blockIdx.x];
}

static void inclusive_scan(int *a, int len, int *bsum, cudaStream_t st) {
    if (len <= 0) return;
    const int nb = (len + kScanBlock - 1) / kScanBlock;
    scan_blocks_kernel<<<nb, kScanBlock, 0, st>>>(a, len, bsum);
    scan_totals_kernel<<<1, kScanBlock, 0, st>>>(bsum, nb);
    scan_carry_kernel<<<nb, kScanBlock, 0, st>>>(a, len, bsum);
}

// ------------------------------------------------------ setup and CSC ----
__global__ void __launch_bounds__(kThreads)
scc_check_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col, int n, int m,
                 Ctrl *c) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
        const int a = row_ptr[v];
        if ((v == 0 && a != 0) || (v == n && a != m)) atomicOr(&c->err, kErrRowPtr);
        if (v < n) {
            const int b = row_ptr[v + 1];
            if (b < a || a < 0 || b > m) atomicOr(&c->err, kErrRowPtr);
        }
    }
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride)
        if ((unsigned)col[e] >= (unsigned)n) atomicOr(&c->err, kErrCol);
}

__global__ void __launch_bounds__(kThreads)
scc_init_kernel(int n, SccWs s, int *scc) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
        s.in_ptr[v] = 0;
        if (v < n) {
            s.cursor[v] = 0;
            s.flags[v] = kActive;
            s.color[v] = 3 * n;
            scc[v] = -1;
        }
    }
}

// In-degrees, warp-uniform over 32 consecutive edges: the lanes that share a
// target add their count with one atomic (a vertex with a million in-edges
// would otherwise serialise a million atomics on one address).
__global__ void __launch_bounds__(kThreads)
csc_count_kernel(const int *__restrict__ col, int m, int *in_ptr) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < m;
         base += warps * 32) {
        const int e = base + lane;
        const int x = e < m ? col[e] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, x);
        if (x >= 0 && lane == __ffs(peers) - 1) atomicAdd(&in_ptr[x + 1], __popc(peers));
    }
}

// Largest u in [lo, hi] with row_ptr[u] <= e (row_ptr[lo] <= e assumed).
static __device__ __forceinline__ int source_of(const int *__restrict__ row_ptr, int e, int lo,
                                                int hi) {
    while (lo < hi) {
        const int mid = lo + ((hi - lo + 1) >> 1);
        if (__ldg(&row_ptr[mid]) <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Edge-parallel: each warp takes 32 consecutive edges, finds the sources of
// its first and last edge over the whole row_ptr, and every lane then finds
// its own source between those two (a vertex with millions of edges is spread
// over many warps instead of one thread).
__global__ void __launch_bounds__(kThreads)
csc_scatter_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col, int n, int m,
                   const int *__restrict__ in_ptr, int *in_src, int *cursor) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < m;
         base += warps * 32) {
        const int last = min(base + 31, m - 1);
        int lo = 0, hi = 0;
        if (lane == 0) lo = source_of(row_ptr, base, 0, n - 1);
        if (lane == 1) hi = source_of(row_ptr, last, 0, n - 1);
        lo = __shfl_sync(0xffffffffu, lo, 0);
        hi = __shfl_sync(0xffffffffu, hi, 1);
        const int e = base + lane;
        const int x = e < m ? col[e] : -1;
        // lanes sharing a target claim their slots with one atomic
        const unsigned peers = __match_any_sync(0xffffffffu, x);
        const int first = __ffs(peers) - 1;
        int pos = 0;
        if (x >= 0 && lane == first) pos = atomicAdd(&cursor[x], __popc(peers));
        pos = __shfl_sync(0xffffffffu, pos, first) + __popc(peers & ((1u << lane) - 1u));
        if (x >= 0) in_src[in_ptr[x] + pos] = source_of(row_ptr, e, lo, hi);
    }
}

__global__ void __launch_bounds__(kThreads)
csc_zero_kernel(int n, int *in_ptr, int *cursor) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
        in_ptr[v] = 0;
        if (v < n) cursor[v] = 0;
    }
}

// Transposed CSR of a graph (in-edges by target; sources in no particular
// order within a row) for the backward searches.  bsum needs n / 1024 + 2
// ints, cursor n.  Returns the number of kernels launched.
int launch_csc(const int *row_ptr, const int *col, int n, int m, int *in_ptr, int *in_src,
               int *cursor, int *bsum, cudaStream_t st) {
    int blocks = (n + kThreads - 1) / kThreads;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    int eb = (m + kThreads - 1) / kThreads;
    if (eb > 8192) eb = 8192;
    if (eb < 1) eb = 1;
    csc_zero_kernel<<<blocks, kThreads, 0, st>>>(n, in_ptr, cursor);
    if (m > 0) csc_count_kernel<<<eb, kThreads, 0, st>>>(col, m, in_ptr);
    inclusive_scan(in_ptr + 1, n, bsum, st);
    if (m > 0) csc_scatter_kernel<<<eb, kThreads, 0, st>>>(row_ptr, col, n, m, in_ptr, in_src, cursor);
    return 6;
}

// largest out- or in-degree (after the CSC is built)
__global__ void __launch_bounds__(kThreads)
max_degree_kernel(const int *__restrict__ row_ptr, const int *__restrict__ in_ptr, int n,
                  Ctrl *c) {
    const int stride = gridDim.x * blockDim.x;
    int d = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        d = max(d, max(row_ptr[v + 1] - row_ptr[v], in_ptr[v + 1] - in_ptr[v]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d = max(d, __shfl_xor_sync(0xffffffffu, d, o));
    if ((threadIdx.x & 31) == 0 && d) atomicMax(&c->maxt, d);
}

// -------------------------------------------------------- one iteration --
// atomicMax / atomicMin on slot[key] by every lane with pred, combined first
// among the lanes of the warp that share the key (one atomic per distinct key
// per warp): all vertices of a large class meet on one pivot slot.
static __device__ __forceinline__ void warp_atomic_max(int *slot, bool pred, int key, int val,
                                                       int lane) {
    const unsigned act = __ballot_sync(0xffffffffu, pred);
    if (!act) return;
    const unsigned peers = __match_any_sync(0xffffffffu, pred ? key : INT_MIN);
    const int mine = pred ? val : INT_MIN;
    int m = mine;
    // reduce over the peer group (every lane takes part in every shuffle)
    for (int src = 0; src < 32; ++src) {
        const int o = __shfl_sync(0xffffffffu, mine, src);
        if ((peers >> src) & 1u) m = max(m, o);
    }
    if (pred && (__ffs(peers) - 1) == lane) atomicMax(&slot[key], m);
}

static __device__ __forceinline__ void warp_atomic_min(int *slot, bool pred, int key, int val,
                                                       int lane) {
    const unsigned act = __ballot_sync(0xffffffffu, pred);
    if (!act) return;
    const unsigned peers = __match_any_sync(0xffffffffu, pred ? key : INT_MIN);
    const int mine = pred ? val : INT_MAX;
    int m = mine;
    for (int src = 0; src < 32; ++src) {
        const int o = __shfl_sync(0xffffffffu, mine, src);
        if ((peers >> src) & 1u) m = min(m, o);
    }
    if (pred && (__ffs(peers) - 1) == lane) atomicMin(&slot[key], m);
}
// Appends item to a global frontier (warp-aggregated atomic on its counter).
static __device__ __forceinline__ void frontier_append(int *q, int *cnt, bool pred, int item,
                                                       int lane) {
    const int pos = warp_append(cnt, pred, lane);
    if (pred) q[pos] = item;
}

// LG = lanes serving one frontier vertex in the searches (8, 16 or 32),
// chosen from the largest degree so that wide vertices do not serialise a
// small group and narrow ones do not idle a whole warp.
template <int LG>
__global__ void __launch_bounds__(kSccThreads, 1)
scc_iteration_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col, int n,
                     SccWs s, int *scc) {
    grid_sync_start();
    Ctrl *c = s.ctrl;
    const unsigned nb = gridDim.x;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;

    if (leader) {
        for (int k = 0; k < 3; ++k) {
            c->cnt[k] = 0;
            c->pending[k] = 0;
            c->hcnt[0][k] = 0;
            c->hcnt[1][k] = 0;
        }
    }
    // 1. trimming: no active out- or in-neighbour in the own class
    for (int round = 0; round < kTrimRounds; ++round) {
        int removed = 0;
        for (int v = gtid; v < n; v += stride) {
            if (!(s.flags[v] & kActive)) continue;
            const int cv = s.color[v];
            bool out_ok = false, in_ok = false;
            for (int e = row_ptr[v]; e < row_ptr[v + 1] && !out_ok; ++e) {
                const int x = col[e];
                out_ok = (s.flags[x] & kActive) && s.color[x] == cv;
            }
            for (int e = s.in_ptr[v]; out_ok && e < s.in_ptr[v + 1] && !in_ok; ++e) {
                const int u = s.in_src[e];
                in_ok = (s.flags[u] & kActive) && s.color[u] == cv;
            }
            if (!out_ok || !in_ok) {
                scc[v] = v;
                s.flags[v] = 0;
                ++removed;
            }
        }
        bool ok;
        const int total = grid_sum_barrier(c, nb, removed, &ok);
        if (!ok) return;
        if (total == 0) break;
    }
    // 2. one pivot per class: its largest active vertex
    for (int v = gtid; v < n; v += stride)
        if (s.flags[v] & kActive) s.piv[s.color[v]] = -1;
    if (!grid_barrier(c, nb)) return;
    for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const int v = base + threadIdx.x;
        const bool act = v < n && (s.flags[v] & kActive);
        warp_atomic_max(s.piv, act, act ? s.color[v] : 0, v, lane);
    }
    if (!grid_barrier(c, nb)) return;
    for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const int v = base + threadIdx.x;
        const bool pv = v < n && (s.flags[v] & kActive) && s.piv[s.color[v]] == v;
        bool hf = false, hb = false;
        if (pv) {
            s.minv[v] = INT_MAX;
            s.flags[v] = kActive | kFw | kBw;
            hf = row_ptr[v + 1] - row_ptr[v] > kSccHeavy;
            hb = s.in_ptr[v + 1] - s.in_ptr[v] > kSccHeavy;
        }
        frontier_append(s.q[0], &c->cnt[0], pv && !hf, v, lane);
        frontier_append(s.hq[0], &c->hcnt[0][0], pv && hf, v, lane);
        frontier_append(s.q[2], &c->pending[0], pv && !hb, v, lane);
        frontier_append(s.hq[2], &c->hcnt[1][0], pv && hb, v, lane);
    }
    if (!grid_barrier(c, nb)) return;
    // 3. forward and backward searches inside the classes, level by level;
    //    counters rotate over three slots so that a reset never meets a read
    for (int lvl = 0;; ++lvl) {
        const int cur = lvl % 3, nxt = (lvl + 1) % 3, old = (lvl + 2) % 3;
        const int nf = load_volatile(&c->cnt[cur]);
        const int nbk = load_volatile(&c->pending[cur]);
        const int nhf = load_volatile(&c->hcnt[0][cur]);
        const int nhb = load_volatile(&c->hcnt[1][cur]);
        if (leader) {
            c->cnt[old] = 0;
            c->pending[old] = 0;
            c->hcnt[0][old] = 0;
            c->hcnt[1][old] = 0;
        }
        const int *qf = s.q[lvl & 1], *qb = s.q[2 + (lvl & 1)];
        int *qf2 = s.q[(lvl + 1) & 1], *qb2 = s.q[2 + ((lvl + 1) & 1)];
        const int *hqf = s.hq[lvl & 1], *hqb = s.hq[2 + (lvl & 1)];
        int *hqf2 = s.hq[(lvl + 1) & 1], *hqb2 = s.hq[2 + ((lvl + 1) & 1)];
        int added = 0;
        // a newly reached vertex joins the next heavy frontier of its search
        // direction when it has more than kSccHeavy edges in that direction
        auto push = [&](bool fwd, bool take, int x) {
            bool heavy = false;
            if (take)
                heavy = (fwd ? row_ptr[x + 1] - row_ptr[x] : s.in_ptr[x + 1] - s.in_ptr[x]) >
                        kSccHeavy;
            frontier_append(fwd ? qf2 : qb2, fwd ? &c->cnt[nxt] : &c->pending[nxt],
                            take && !heavy, x, lane);
            frontier_append(fwd ? hqf2 : hqb2, &c->hcnt[fwd ? 0 : 1][nxt], take && heavy, x,
                            lane);
        };
        // groups of LG lanes per frontier vertex (32 / LG vertices per warp
        // task, forward tasks first, then backward ones); a group strides
        // over its vertex's edges
        constexpr int kPer = 32 / LG;
        const int warp_id = gtid >> 5, nwarps = stride >> 5;
        const int grp = lane / LG, sub = lane % LG;
        const int ntf = (nf + kPer - 1) / kPer, ntb = (nbk + kPer - 1) / kPer;
        for (int task = warp_id; task < ntf + ntb; task += nwarps) {
            const bool fwd = task < ntf;
            const int i = (fwd ? task : task - ntf) * kPer + grp;
            const int bit = fwd ? kFw : kBw;
            const int *adj = fwd ? col : s.in_src;
            int e = 0, e1 = 0, cu = 0;
            if (i < (fwd ? nf : nbk)) {
                const int u = fwd ? qf[i] : qb[i];
                cu = s.color[u];
                e = (fwd ? row_ptr[u] : s.in_ptr[u]) + sub;
                e1 = fwd ? row_ptr[u + 1] : s.in_ptr[u + 1];
            }
            for (;;) {
                const bool more = e < e1;
                if (!__any_sync(0xffffffffu, more)) break;
                bool take = false;
                int x = 0;
                if (more) {
                    x = adj[e];
                    e += LG;
                    const int f = s.flags[x];
                    if ((f & kActive) && !(f & bit) && s.color[x] == cu)
                        take = !(atomicOr(&s.flags[x], bit) & bit);
                }
                push(fwd, take, x);
                added += take;
            }
        }
        // heavy frontier vertices: every warp of the grid takes a strided
        // share of each one's edges
        for (int j = 0; j < nhf + nhb; ++j) {
            const bool fwd = j < nhf;
            const int u = fwd ? hqf[j] : hqb[j - nhf];
            const int bit = fwd ? kFw : kBw;
            const int *adj = fwd ? col : s.in_src;
            const int cu = s.color[u];
            int e = (fwd ? row_ptr[u] : s.in_ptr[u]) + gtid;
            const int e1 = fwd ? row_ptr[u + 1] : s.in_ptr[u + 1];
            for (;;) {
                const bool more = e < e1;
                if (!__any_sync(0xffffffffu, more)) break;
                bool take = false;
                int x = 0;
                if (more) {
                    x = adj[e];
                    e += stride;
                    const int f = s.flags[x];
                    if ((f & kActive) && !(f & bit) && s.color[x] == cu)
                        take = !(atomicOr(&s.flags[x], bit) & bit);
                }
                push(fwd, take, x);
                added += take;
            }
        }
        bool ok;
        const int total = grid_sum_barrier(c, nb, added, &ok);
        if (!ok) return;
        if (leader) c->rounds_detect += 1;
        if (total == 0) break;
        if (lvl > n) {   // a search cannot have more levels than vertices
            if (leader) atomicOr(&c->err, kErrDetect);
            return;
        }
    }
    // 4. split: reached both ways = the pivot's component
    for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const int v = base + threadIdx.x;
        const int f = v < n ? s.flags[v] : 0;
        const bool in = (f & kActive) && (f & kFw) && (f & kBw);
        warp_atomic_min(s.minv, in, in ? s.piv[s.color[v]] : 0, v, lane);
    }
    if (!grid_barrier(c, nb)) return;
    int still = 0;
    for (int v = gtid; v < n; v += stride) {
        const int f = s.flags[v];
        if (!(f & kActive)) continue;
        const int p = s.piv[s.color[v]];
        if ((f & kFw) && (f & kBw)) {
            scc[v] = s.minv[p];
            s.flags[v] = 0;
        } else {
            s.color[v] = 3 * p + ((f & kFw) ? 1 : (f & kBw) ? 2 : 0);
            s.flags[v] = kActive;
            ++still;
        }
    }
    bool ok;
    const int left = grid_sum_barrier(c, nb, still, &ok);
    if (!ok) return;
    if (leader) c->nrep = left;
}

__global__ void __launch_bounds__(kThreads)
scc_count_kernel(const int *__restrict__ scc, int n, Ctrl *c) {
    const int stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const int v = base + threadIdx.x;
        warp_append(&c->ncand, v < n && scc[v] == v, lane);
    }
}

__global__ void scc_ctrl_init_kernel(Ctrl *c) {
    Ctrl z;
    memset(&z, 0, sizeof z);
    z.bad_index = INT_MAX;
    z.wait_ns = kDefaultWaitNs;
    *c = z;
}

template <int LG>
static int scc_grid() {
    static int cached_dev = -1, cached = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev == cached_dev && cached > 0) return cached;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scc_iteration_kernel<LG>,
                                                      kSccThreads, 0) != cudaSuccess ||
        per_sm < 1)
        return 0;
    cached_dev = dev;
    cached = sms * per_sm;
    return cached;
}

static int read_scc_ctrl(const Ctrl *dev, Ctrl *host, cudaStream_t st) {
    if (cudaMemcpyAsync(host, dev, sizeof(Ctrl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return OCM_ERR_CUDA;
    return OCM_OK;
}

static int scc_err(int err) {
    if (err & kErrTimeout) return OCM_ERR_TIMEOUT;
    if (err & (kErrRowPtr | kErrCol)) return OCM_ERR_BAD_CSR;
    return err ? OCM_ERR_INTERNAL : OCM_OK;
}

// The whole decomposition; *levels receives the BFS levels summed over the
// iterations and *iters the iterations (either may be null).
int scc_decompose(const int *row_ptr, const int *col, int n, int m, int *scc, int *num_scc,
                  void *workspace, cudaStream_t st, long long *launches, int *iters,
                  int *levels) {
    SccWs s;
    carve_scc(workspace, n, m, &s);
    Ctrl h;
    long long k = 0;
    int blocks = (n + kThreads - 1) / kThreads;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    scc_ctrl_init_kernel<<<1, 1, 0, st>>>(s.ctrl);
    scc_check_kernel<<<blocks, kThreads, 0, st>>>(row_ptr, col, n, m, s.ctrl);
    k += 2;
    if (cudaGetLastError() != cudaSuccess) return OCM_ERR_CUDA;
    int rc = read_scc_ctrl(s.ctrl, &h, st);
    if (rc) return rc;
    if (h.err) return scc_err(h.err);
    scc_init_kernel<<<blocks, kThreads, 0, st>>>(n, s, scc);
    launch_csc(row_ptr, col, n, m, s.in_ptr, s.in_src, s.cursor, s.bsum, st);
    max_degree_kernel<<<blocks, kThreads, 0, st>>>(row_ptr, s.in_ptr, n, s.ctrl);
    k += 7;
    if (cudaGetLastError() != cudaSuccess) return OCM_ERR_CUDA;
    rc = read_scc_ctrl(s.ctrl, &h, st);
    if (rc) return rc;
    // lanes per frontier vertex: about half the largest degree, 8 to 32
    const int lg = h.maxt > 32 ? 32 : h.maxt > 16 ? 16 : 8;
    const int grid = lg == 32 ? scc_grid<32>() : lg == 16 ? scc_grid<16>() : scc_grid<8>();
    if (grid <= 0) return OCM_ERR_CUDA;
    int g = (n + kSccThreads - 1) / kSccThreads;
    if (g > grid) g = grid;
    int it = 0;
    for (;; ++it) {
        if (it > n) return OCM_ERR_NOT_CONVERGED;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(g);
        cfg.blockDim = dim3(kSccThreads);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        // the grid barrier counts arrivals from zero in every launch
        if (cudaMemsetAsync(&s.ctrl->bar[0], 0, sizeof(GridBar), st) != cudaSuccess)
            return OCM_ERR_CUDA;
        const cudaError_t le =
            lg == 32 ? cudaLaunchKernelEx(&cfg, scc_iteration_kernel<32>, row_ptr, col, n, s, scc)
            : lg == 16 ? cudaLaunchKernelEx(&cfg, scc_iteration_kernel<16>, row_ptr, col, n, s, scc)
                       : cudaLaunchKernelEx(&cfg, scc_iteration_kernel<8>, row_ptr, col, n, s, scc);
        if (le != cudaSuccess) return OCM_ERR_CUDA;
        ++k;
        rc = read_scc_ctrl(s.ctrl, &h, st);
        if (rc) return rc;
        if (h.err) return scc_err(h.err);
        if (h.nrep == 0) break;
    }
    scc_count_kernel<<<blocks, kThreads, 0, st>>>(scc, n, s.ctrl);
    ++k;
    if (cudaGetLastError() != cudaSuccess) return OCM_ERR_CUDA;
    rc = read_scc_ctrl(s.ctrl, &h, st);
    if (rc) return rc;
    if (num_scc) *num_scc = h.ncand;
    if (launches) *launches += k;
    if (iters) *iters = it + 1;
    if (levels) *levels = h.rounds_detect;
    return OCM_OK;
}

size_t scc_workspace_size(int n, int m) { return carve_scc(nullptr, n, m, nullptr); }

}  // namespace ocm

using namespace ocm;

extern "C" {

size_t ocm_workspace_size_scc(int32_t n, int32_t m) {
    if (n < 1 || m < 0) return 0;
    return scc_workspace_size(n, m);
}

int ocm_scc(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int32_t m, int32_t *scc,
            int32_t *num_scc, void *workspace, size_t ws_bytes, void *stream) {
    if (!row_ptr || !scc || !num_scc || (m > 0 && !col_idx)) return OCM_ERR_INVALID_ARG;
    if (n < 1 || m < 0 || n > (INT_MAX - 2) / 3) return OCM_ERR_INVALID_ARG;
    if (!workspace || ws_bytes < scc_workspace_size(n, m) ||
        (reinterpret_cast<uintptr_t>(workspace) & 255u))
        return OCM_ERR_WORKSPACE;
    NvtxRange range("ocm_scc");
    if (injected_fault("launch")) return OCM_ERR_CUDA;
    int count = 0;
    const int rc = scc_decompose(row_ptr, col_idx, n, m, scc, &count, workspace,
                                 static_cast<cudaStream_t>(stream), nullptr, nullptr, nullptr);
    if (rc == OCM_OK) *num_scc = count;
    return rc;
}

}  // extern "C"

namespace ocm {

// ------------------------------------------- per-component solve ------------
// Stable LSD radix sort of (key, id) pairs, 8-bit digits, across a
// cooperative grid: per pass, per-block digit histograms, one exclusive scan
// in (digit, block) order by block 0, then a stable scatter (warps of a
// block in turn; lanes with equal digits ranked by a match mask).  Passes
// whose digit is the same for every key are skipped.  keys are non-negative.
// On return the sorted pairs are in (k0, i0) if the number of executed
// passes is even, else in (k1, i1); *which reports it (block 0, thread 0).
__global__ void __launch_bounds__(kSortThreads, 1)
sort_pairs_kernel(int len, int *k0, int *i0, int *k1, int *i1, int *hist, Ctrl *c) {
    __shared__ int s_off[256];
    __shared__ int s_warp[32];
    __shared__ int s_skip;
    grid_sync_start();
    const unsigned nb = gridDim.x;
    const int G = (int)gridDim.x;
    const int chunk = (len + G - 1) / G;
    const int c0 = min(len, (int)blockIdx.x * chunk), c1 = min(len, c0 + chunk);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (int)(blockDim.x >> 5);
    int *ka = k0, *ia = i0, *kb = k1, *ib = i1;
    int swaps = 0;
    for (int pass = 0; pass < 4; ++pass) {
        const int sh = 8 * pass;
        int *h = hist + (pass & 1) * 256 * G;
        if (threadIdx.x < 256) s_off[threadIdx.x] = 0;
        __syncthreads();
        for (int i = c0 + (int)threadIdx.x; i < c1; i += blockDim.x)
            atomicAdd(&s_off[(ka[i] >> sh) & 255], 1);
        __syncthreads();
        if (threadIdx.x < 256) h[threadIdx.x * G + blockIdx.x] = s_off[threadIdx.x];
        if (!grid_barrier(c, nb)) return;
        if (blockIdx.x == 0) {
            const int total = 256 * G;
            const int per = (total + (int)blockDim.x - 1) / (int)blockDim.x;
            const int b0 = min(total, (int)threadIdx.x * per), b1 = min(total, b0 + per);
            int sum = 0;
            for (int i = b0; i < b1; ++i) sum += h[i];
            // block-wide exclusive scan of the per-thread sums
            int x = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_warp[warp] = x;
            __syncthreads();
            if (warp == 0) {
                int wv = lane < nwarps ? s_warp[lane] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, wv, o);
                    if (lane >= o) wv += y;
                }
                s_warp[lane] = wv;
            }
            __syncthreads();
            int run = x - sum + (warp > 0 ? s_warp[warp - 1] : 0);
            for (int i = b0; i < b1; ++i) {
                const int v = h[i];
                h[i] = run;
                run += v;
            }
        }
        if (!grid_barrier(c, nb)) return;
        if (threadIdx.x == 0) s_skip = 0;
        __syncthreads();
        if (threadIdx.x < 256) {
            const int lo = h[threadIdx.x * G];
            const int hi = threadIdx.x < 255 ? h[(threadIdx.x + 1) * G] : len;
            if (hi - lo == len) s_skip = 1;
            s_off[threadIdx.x] = h[threadIdx.x * G + blockIdx.x];
        }
        __syncthreads();
        if (s_skip) continue;   // the same decision in every block
        for (int t0 = c0; t0 < c1; t0 += blockDim.x) {
            const int i = t0 + (int)threadIdx.x;
            const bool valid = i < c1;
            const int k = valid ? ka[i] : 0;
            const int id = valid ? ia[i] : 0;
            const int dg = valid ? ((k >> sh) & 255) : 256 + lane;
            const unsigned peers = __match_any_sync(0xffffffffu, dg);
            const int r = __popc(peers & ((1u << lane) - 1u));
            for (int wv = 0; wv < nwarps; ++wv) {
                int base = 0;
                if (warp == wv && valid) base = s_off[dg];
                __syncwarp();
                if (warp == wv && valid) {
                    kb[base + r] = k;
                    ib[base + r] = id;
                    if (r == 0) s_off[dg] = base + __popc(peers);
                }
                __syncthreads();
            }
        }
        int *t = ka;
        ka = kb;
        kb = t;
        t = ia;
        ia = ib;
        ib = t;
        ++swaps;
        if (!grid_barrier(c, nb)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) c->iter = swaps & 1;
}

// Workspace of the per-component solve, after the decomposition's.
struct CompWs {
    int *ideg;      // [n] edges of v that stay inside its component
    int *cyclic;    // [n] by label: the component holds a cycle
    int *sel;       // [n + 1] selection flags, then their inclusive scan
    int *key[2];    // [n] sort keys (labels)
    int *ids[2];    // [n] sort values (vertices)
    int *hist;      // [2 * 256 * blocks] radix histograms
    int *newid;     // [n] position of a vertex in the component order
    int *vptr;      // [n + 1] first position of each component (+ end)
    int *rp2;       // [n + 1] CSR of the components' induced subgraphs
    int *col2;      // [m]
    int *w2;        // [m]
    int *emap;      // [m] original edge of each kept edge
    int *eflag;     // [m] edge stays inside its component, then the inclusive scan of that
    int *ebsum;     // [m / 1024 + 2] block sums of that scan
    int *cyc2;      // [n] cycles in kept-edge indices
    void *batch_ws; // batched solve
    size_t batch_bytes;
};

static size_t carve_comp(void *base, int n, int m, int hist_blocks, CompWs *ws) {
    char *b = static_cast<char *>(base);
    size_t off = scc_workspace_size(n, m);
    const size_t N = (size_t)n, M = (size_t)(m > 0 ? m : 1);
    auto take = [&](size_t bytes) -> void * {
        off = align256(off);
        void *p = b ? b + off : nullptr;
        off += bytes;
        return p;
    };
    CompWs w{};
    w.ideg = static_cast<int *>(take(4 * N));
    w.cyclic = static_cast<int *>(take(4 * N));
    w.sel = static_cast<int *>(take(4 * (N + 1)));
    for (int i = 0; i < 2; ++i) {
        w.key[i] = static_cast<int *>(take(4 * N));
        w.ids[i] = static_cast<int *>(take(4 * N));
    }
    w.hist = static_cast<int *>(take(4 * 2 * 256 * (size_t)hist_blocks));
    w.newid = static_cast<int *>(take(4 * N));
    w.vptr = static_cast<int *>(take(4 * (N + 1)));
    w.rp2 = static_cast<int *>(take(4 * (N + 1)));
    w.col2 = static_cast<int *>(take(4 * M));
    w.w2 = static_cast<int *>(take(4 * M));
    w.emap = static_cast<int *>(take(4 * M));
    w.eflag = static_cast<int *>(take(4 * M));
    w.ebsum = static_cast<int *>(take(4 * (M / kScanBlock + 2)));
    w.cyc2 = static_cast<int *>(take(4 * N));
    w.batch_bytes = ocm_workspace_size_batch(n, n, m > 0 ? m : 1);
    w.batch_ws = take(w.batch_bytes);
    if (ws) *ws = w;
    return align256(off);
}

constexpr int kMaxSortBlocks = 1024;   // histogram capacity of the component sort

// The edges that stay inside their component (edge-parallel: warps of 32
// consecutive edges, sources as in csc_scatter_kernel); their inclusive scan
// then gives every vertex its internal degree and every internal edge its
// place among its vertex's internal edges, without a per-vertex edge loop.
__global__ void __launch_bounds__(kThreads)
comp_flag_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col,
                 const int *__restrict__ scc, int n, int m, CompWs cw) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < m;
         base += warps * 32) {
        const int last = min(base + 31, m - 1);
        int lo = 0, hi = 0;
        if (lane == 0) lo = source_of(row_ptr, base, 0, n - 1);
        if (lane == 1) hi = source_of(row_ptr, last, 0, n - 1);
        lo = __shfl_sync(0xffffffffu, lo, 0);
        hi = __shfl_sync(0xffffffffu, hi, 1);
        const int e = base + lane;
        if (e < m) {
            const int u = source_of(row_ptr, e, lo, hi);
            cw.eflag[e] = scc[col[e]] == scc[u] ? 1 : 0;
        }
    }
}

// internal degree of every vertex; components with an internal edge hold a cycle
__global__ void __launch_bounds__(kThreads)
comp_degree_kernel(const int *__restrict__ row_ptr, const int *__restrict__ scc, int n,
                   CompWs cw) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int a = row_ptr[v], b = row_ptr[v + 1];
        const int d = b > a ? cw.eflag[b - 1] - (a > 0 ? cw.eflag[a - 1] : 0) : 0;
        cw.ideg[v] = d;
        if (d) cw.cyclic[scc[v]] = 1;
    }
}

__global__ void __launch_bounds__(kThreads)
comp_zero_kernel(int n, CompWs cw) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) cw.cyclic[v] = 0;
}

__global__ void __launch_bounds__(kThreads)
comp_select_kernel(const int *__restrict__ scc, int n, CompWs cw) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        cw.sel[v] = cw.cyclic[scc[v]] ? 1 : 0;
}

// stable compaction (vertex order) of the selected vertices: key = label
__global__ void __launch_bounds__(kThreads)
comp_compact_kernel(const int *__restrict__ scc, int n, CompWs cw) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int before = v > 0 ? cw.sel[v - 1] : 0;   // inclusive scan
        if (cw.sel[v] != before) {
            cw.key[0][before] = scc[v];
            cw.ids[0][before] = v;
        }
    }
}

// positions of the sorted vertices, component starts, kept-degree per position
__global__ void __launch_bounds__(kThreads)
comp_order_kernel(int len, const int *__restrict__ skey, const int *__restrict__ sid, CompWs cw) {
    const int stride = gridDim.x * blockDim.x;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < len; k += stride) {
        const int v = sid[k];
        cw.newid[v] = k;
        cw.rp2[k + 1] = cw.ideg[v];
        cw.sel[k] = (k == 0 || skey[k] != skey[k - 1]) ? 1 : 0;
    }
}

__global__ void __launch_bounds__(kThreads)
comp_vptr_kernel(int len, CompWs cw) {
    const int stride = gridDim.x * blockDim.x;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < len; k += stride) {
        const int before = k > 0 ? cw.sel[k - 1] : 0;
        if (cw.sel[k] != before) cw.vptr[before] = k;
        if (k == len - 1) cw.vptr[cw.sel[k]] = len;
    }
}

__global__ void __launch_bounds__(kThreads)
comp_edges_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col,
                  const int *__restrict__ w, int n, int m, CompWs cw) {
    // edge-parallel like comp_flag_kernel; an internal edge's place is its
    // vertex's first kept position plus the internal edges before it
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < m;
         base += warps * 32) {
        const int last = min(base + 31, m - 1);
        int lo = 0, hi = 0;
        if (lane == 0) lo = source_of(row_ptr, base, 0, n - 1);
        if (lane == 1) hi = source_of(row_ptr, last, 0, n - 1);
        lo = __shfl_sync(0xffffffffu, lo, 0);
        hi = __shfl_sync(0xffffffffu, hi, 1);
        const int e = base + lane;
        if (e < m) {
            const int incl = cw.eflag[e];
            if (incl - (e > 0 ? cw.eflag[e - 1] : 0)) {
                const int u = source_of(row_ptr, e, lo, hi);
                const int a = row_ptr[u];
                const int pos = cw.rp2[cw.newid[u]] + incl - 1 - (a > 0 ? cw.eflag[a - 1] : 0);
                cw.col2[pos] = cw.newid[col[e]];
                cw.w2[pos] = w[e];
                cw.emap[pos] = e;
            }
        }
    }
}

// one warp per component: its cycle in original edge indices, its root, offset
__global__ void __launch_bounds__(kThreads)
comp_results_kernel(int G, const int *__restrict__ sid, CompWs cw,
                    const int *__restrict__ clen, int *comp_root, int *comp_off,
                    int *cycle_out) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G; g += warps) {
        const int start = cw.vptr[g];
        if (lane == 0) {
            comp_root[g] = sid[start];
            comp_off[g] = start;
            if (g == G - 1) comp_off[G] = cw.vptr[G];
        }
        const int L = clen[g];
        for (int j = lane; j < L; j += 32) cycle_out[start + j] = cw.emap[cw.cyc2[start + j]];
    }
}

static int sort_grid() {
    static int cached_dev = -1, cached = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev == cached_dev && cached > 0) return cached;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sort_pairs_kernel, kSortThreads,
                                                      0) != cudaSuccess ||
        per_sm < 1)
        return 0;
    cached_dev = dev;
    cached = sms * per_sm < kMaxSortBlocks ? sms * per_sm : kMaxSortBlocks;
    return cached;
}

static int read_int(const int *dev, int *host, cudaStream_t st) {
    if (cudaMemcpyAsync(host, dev, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return OCM_ERR_CUDA;
    return OCM_OK;
}

size_t comp_workspace_size(int n, int m) { return carve_comp(nullptr, n, m, kMaxSortBlocks, nullptr); }

}  // namespace ocm

extern "C" {

size_t ocm_workspace_size_solve_scc(int32_t n, int32_t m) {
    if (n < 1 || m < 0 || n > (INT_MAX - 2) / 3) return 0;
    return comp_workspace_size(n, m);
}

int ocm_solve_scc(const int32_t *row_ptr, const int32_t *col_idx, const int32_t *w, int32_t n,
                  int32_t m, int mode, int32_t *scc, int32_t *num_comp, int32_t *comp_root,
                  int32_t *comp_off, int64_t *num, int32_t *den, int32_t *cycle_len,
                  int32_t *cycle_out, void *workspace, size_t ws_bytes, void *stream,
                  const ocm_options *opt, ocm_stats *stats) {
    if (!row_ptr || !scc || !num_comp || !comp_root || !comp_off || !num || !den ||
        !cycle_len || !cycle_out || (m > 0 && (!col_idx || !w)))
        return OCM_ERR_INVALID_ARG;
    if (n < 1 || m < 0 || n > (INT_MAX - 2) / 3 || (mode != OCM_MAX && mode != OCM_MIN))
        return OCM_ERR_INVALID_ARG;
    if (opt && (opt->init_policy || opt->transit || (opt->flags & OCM_FLAG_TEST_STALL)))
        return OCM_ERR_INVALID_ARG;
    NvtxRange range("ocm_solve_scc");
    if (injected_fault("launch")) return OCM_ERR_CUDA;
    if (!workspace || ws_bytes < comp_workspace_size(n, m) ||
        (reinterpret_cast<uintptr_t>(workspace) & 255u))
        return OCM_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CompWs cw;
    carve_comp(workspace, n, m, kMaxSortBlocks, &cw);
    SccWs sw;
    carve_scc(workspace, n, m, &sw);
    long long launches = 0;
    int nscc = 0, iters = 0, levels = 0;
    int rc = scc_decompose(row_ptr, col_idx, n, m, scc, &nscc, workspace, st, &launches, &iters,
                           &levels);
    if (rc) return rc;
    int blocks = (n + kThreads - 1) / kThreads;
    if (blocks > 4096) blocks = 4096;
    comp_zero_kernel<<<blocks, kThreads, 0, st>>>(n, cw);
    int eb = (m + kThreads - 1) / kThreads;
    if (eb > 8192) eb = 8192;
    if (eb < 1) eb = 1;
    if (m > 0) {
        comp_flag_kernel<<<eb, kThreads, 0, st>>>(row_ptr, col_idx, scc, n, m, cw);
        inclusive_scan(cw.eflag, m, cw.ebsum, st);
        comp_degree_kernel<<<blocks, kThreads, 0, st>>>(row_ptr, scc, n, cw);
        launches += 5;
    }
    comp_select_kernel<<<blocks, kThreads, 0, st>>>(scc, n, cw);
    inclusive_scan(cw.sel, n, sw.bsum, st);
    comp_compact_kernel<<<blocks, kThreads, 0, st>>>(scc, n, cw);
    launches += 6;
    if (cudaGetLastError() != cudaSuccess) return OCM_ERR_CUDA;
    int len = 0;
    rc = read_int(cw.sel + (n - 1), &len, st);
    if (rc) return rc;
    if (len == 0) {   // acyclic: no component holds a cycle
        *num_comp = 0;
        if (stats) {
            memset(stats, 0, sizeof *stats);
            stats->launches = launches;
        }
        return OCM_OK;
    }
    // stable sort of the selected vertices by label: components become
    // contiguous, each in increasing vertex order
    const int sg = sort_grid();
    if (sg <= 0) return OCM_ERR_CUDA;
    int g = (len + kSortThreads - 1) / kSortThreads;
    if (g > sg) g = sg;
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(g);
        cfg.blockDim = dim3(kSortThreads);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        scc_ctrl_init_kernel<<<1, 1, 0, st>>>(sw.ctrl);
        if (cudaLaunchKernelEx(&cfg, sort_pairs_kernel, len, cw.key[0], cw.ids[0], cw.key[1],
                               cw.ids[1], cw.hist, sw.ctrl) != cudaSuccess)
            return OCM_ERR_CUDA;
        launches += 2;
    }
    Ctrl h;
    rc = read_scc_ctrl(sw.ctrl, &h, st);
    if (rc) return rc;
    if (h.err) return scc_err(h.err);
    const int *skey = cw.key[h.iter], *sid = cw.ids[h.iter];
    int lb = (len + kThreads - 1) / kThreads;
    if (lb > 4096) lb = 4096;
    comp_order_kernel<<<lb, kThreads, 0, st>>>(len, skey, sid, cw);
    inclusive_scan(cw.sel, len, sw.bsum, st);
    comp_vptr_kernel<<<lb, kThreads, 0, st>>>(len, cw);
    // rp2[0] = 0, rp2[k+1] = kept degree of position k -> inclusive scan
    if (cudaMemsetAsync(cw.rp2, 0, sizeof(int), st) != cudaSuccess) return OCM_ERR_CUDA;
    inclusive_scan(cw.rp2 + 1, len, sw.bsum, st);
    if (m > 0) comp_edges_kernel<<<eb, kThreads, 0, st>>>(row_ptr, col_idx, w, n, m, cw);
    launches += 9;
    if (cudaGetLastError() != cudaSuccess) return OCM_ERR_CUDA;
    int G = 0, M2 = 0;
    rc = read_int(cw.sel + (len - 1), &G, st);
    if (rc) return rc;
    rc = read_int(cw.rp2 + len, &M2, st);
    if (rc) return rc;
    ocm_stats bst;
    memset(&bst, 0, sizeof bst);
    rc = ocm_solve_batch(cw.vptr, cw.rp2, cw.col2, cw.w2, G, len, M2, mode, num, den, cycle_len,
                         cw.cyc2, cw.batch_ws, cw.batch_bytes, stream, opt, &bst);
    if (rc) return rc;
    int gb = (G * 32 + kThreads - 1) / kThreads;
    if (gb > 4096) gb = 4096;
    comp_results_kernel<<<gb, kThreads, 0, st>>>(G, sid, cw, cycle_len, comp_root, comp_off,
                                                 cycle_out);
    launches += 1;
    if (cudaGetLastError() != cudaSuccess) return OCM_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return OCM_ERR_CUDA;
    *num_comp = G;
    if (stats) {
        *stats = bst;
        stats->launches = bst.launches + launches;
    }
    return OCM_OK;
}

}  // extern "C"
