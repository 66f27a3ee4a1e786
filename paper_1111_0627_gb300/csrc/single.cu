// single.cu -- the paper's own form of the policy iteration (Alg. 1 as
// written; Alg. 2's markMinComponent, connectGpi and valuePropagate): one
// lambda per iteration, the mean of the chosen policy cycle, and every other
// policy cycle broken so that all vertices reach the chosen one.
//
// The solver's default iteration keeps one mean per policy cycle (multichain)
// and needs no rebuild; with OCM_FLAG_SINGLE_LAMBDA the step becomes
//   evaluate -> connect (this file) -> sweep -> control,
// where connect, one cooperative launch, does the rebuild and the value
// propagation of Alg. 1 at once:
//   level 0   the component of the chosen cycle (the evaluation's best: the
//             largest mean, then the smallest root) keeps its policy and its
//             values -- markMinComponent;
//   level k   every vertex not yet connected with an out-edge into level
//             k-1 takes its smallest-index out-edge into the vertices
//             connected at levels < k -- connectGpi; the paper leaves that
//             choice open, the smallest index makes it deterministic.  A
//             level of more than n/64 vertices (there are at most 64) is
//             found by passes over all vertices -- pulling (every unconnected
//             vertex scans its out-edges) when fewer vertices are left than
//             level k-1 holds, else pushing (level k-1 marks its in-neighbours
//             over the transposed graph, plain stores, then every marked
//             vertex picks its edge) -- and a smaller one through compact
//             lists (atomic claims and appends), so small levels cost no pass
//             over the graph; a heavy vertex (more than kHeavyEdges
//             out-edges) is left out of the per-vertex edge scans and its
//             edges are scanned by the whole grid in chunks instead, and a
//             pushing vertex with more than kInHeavy in-edges is listed and
//             its in-edges spread over a block (over the grid above
//             kInHeavyGrid);
//   values    a vertex connected at level k gets its path sums from its new
//             successor, final since level k-1: (len, S) = (len(t) + 1,
//             S(t) + s*w(e)) and V = q*S - p*len relative to the chosen
//             cycle's smallest vertex -- valuePropagate along the new edges.
// Both state buffers of the value jumping receive the final state, so the
// next evaluation treats a rebuilt vertex like any vertex the sweep did not
// touch.  The levels are separated by the bounded grid barrier.
#include <climits>

#include "common.cuh"
#include "grid_sync.cuh"

namespace ocm {

constexpr int kConnectThreads = 1024;   // one block per SM: few arrivals per barrier
constexpr int kConnectLanes = 8;        // lanes serving one frontier vertex
constexpr int kBarConnect = 1;          // this kernel's GridBar in the control block
constexpr int kInHeavy = 4096;          // in-edges above which a push is spread over a block
constexpr int kInHeavyGrid = 65536;     // ... and above which over the whole grid

size_t carve_single(void *base, int n, int m, SingleWs *sw) {
    char *b = static_cast<char *>(base);
    size_t off = 0;
    const size_t N = (size_t)n, M = (size_t)m;
    auto take = [&](size_t bytes) -> void * {
        off = (off + 255) / 256 * 256;
        void *p = b ? b + off : nullptr;
        off += bytes;
        return p;
    };
    SingleWs w{};
    w.in_ptr = static_cast<int *>(take(4 * (N + 1)));
    w.in_src = static_cast<int *>(take(4 * M));
    w.cursor = static_cast<int *>(take(4 * N));
    w.bsum = static_cast<int *>(take(4 * (N / 1024 + 2)));
    w.lev = static_cast<int *>(take(4 * N));
    w.fr[0] = static_cast<int *>(take(4 * N));
    w.fr[1] = static_cast<int *>(take(4 * N));
    if (sw) *sw = w;
    return (off + 255) / 256 * 256;
}

static __device__ __forceinline__ void append(int *q, int *cnt, bool pred, int item, int lane) {
    const int pos = warp_append(cnt, pred, lane);
    if (pred) q[pos] = item;
}

// The heavy vertices (listed by the classify step, their edges numbered in
// one sequence by heavy_off) whose level is `want` look for their smallest
// out-edge into levels < k: one warp per chunk of kHeavyChunk entries of the
// sequence, four edges per lane in flight, the chunk's first hit lowering
// pick[i] (atomicMin; a chunk above an edge already found is skipped).  No
// level below k changes while this runs, and a vertex that joins level k
// concurrently fails the test either way, so the picks are the smallest
// qualifying edges whatever the order of the chunks.
static __device__ __forceinline__ void heavy_scan(int want, int k, const int *__restrict__ row_ptr,
                                                  const int *__restrict__ col, const Workspace &ws,
                                                  const SingleWs &sg, int *pick, int H,
                                                  const int *hv, int total, int warp_id,
                                                  int nwarps, int lane) {
    const int nchunks = (total + kHeavyChunk - 1) / kHeavyChunk;
    for (int ch = warp_id; ch < nchunks; ch += nwarps) {
        const int g0 = ch * kHeavyChunk, g1 = min(g0 + kHeavyChunk, total);
        int lo = 0, hi = H;   // the heavy vertex holding entry g0
        while (hi - lo > 1) {
            const int mid = lo + ((hi - lo) >> 1);
            if (ws.heavy_off[mid] <= g0) lo = mid; else hi = mid;
        }
        // at most two heavy vertices meet in a chunk: each has more edges
        for (int i = lo; i < H && ws.heavy_off[i] < g1; ++i) {
            const int v = hv[i];
            if (sg.lev[v] != want) continue;   // stable during the scan: warp-uniform
            const int a = max(g0, ws.heavy_off[i]), b = min(g1, ws.heavy_off[i + 1]);
            const int base = row_ptr[v] - ws.heavy_off[i];
            int known = 0;
            if (lane == 0) known = load_volatile(&pick[i]);
            known = __shfl_sync(0xffffffffu, known, 0);
            if (known < base + a) continue;
            int best = INT_MAX;
            for (int g = a + lane; g < b && best == INT_MAX; g += 128) {
                int l[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) l[j] = g + 32 * j < b ? sg.lev[col[base + g + 32 * j]] : -1;
#pragma unroll
                for (int j = 3; j >= 0; --j)
                    if (l[j] >= 0 && l[j] < k) best = base + g + 32 * j;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
            if (lane == 0 && best != INT_MAX) atomicMin(&pick[i], best);
        }
    }
}


// Vertex u joins level k through edge e: its policy, its final path sums
// (both buffers of the value jumping) and its record for the sweep, all
// relative to the chosen cycle (root rstar, mean P/Q, rank RK).
static __device__ __forceinline__ void take_edge(int u, int e, int k, int rstar, long long P,
                                                 long long Q, int RK, bool ratio, int sign,
                                                 const int *__restrict__ col,
                                                 const int *__restrict__ w, const Workspace &ws,
                                                 const SingleWs &sg) {
    const int t = col[e];
    const int wv = sign * w[e];
    ws.pi[u] = e;
    ws.succ[u] = t;
    ws.wpi[u] = wv;
    const JLS st = ws.jls[0][t];
    const JLS su{~rstar, st.len + 1, st.S + (long long)wv};
    ws.jls[0][u] = su;
    ws.jls[1][u] = su;
    long long T = su.len;
    if (ratio) {
        const int tr = ws.transit[e];
        ws.tpi[u] = tr;
        T = ws.jt[0][t] + tr;
        ws.jt[0][u] = T;
        ws.jt[1][u] = T;
        ws.recp[u] = P;
    }
    Rec r;
    r.V = Q * su.S - P * T;
    r.rank = RK;
    r.q = (int)Q;
    ws.rec[u] = r;
    // level k is numbered at once: the edge tests above take levels < k only
    sg.lev[u] = k;
}

__global__ void __launch_bounds__(kConnectThreads, 1)
connect_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col,
               const int *__restrict__ w, int sign, int n, Workspace ws, SingleWs sg) {
    grid_sync_start();
    Ctrl *c = ws.ctrl;
    const unsigned nb = gridDim.x;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const bool leader = gtid == 0;
    // the evaluation before this launch finished (or stopped on an error)
    // before any block started, so every block takes the same branch here
    if (c->err) return;
    const unsigned long long bb = c->best;
    const int rstar = 0x7fffffff - (int)(unsigned)(bb & 0xffffffffu);
    if (bb == 0 || rstar < 0 || rstar >= n) {
        if (leader) atomicOr(&c->err, kErrConnect);
        return;
    }
    const int istar = ws.cid_of_root[rstar];
    const long long P = ws.cyc_p[istar];
    const long long Q = ws.cyc_q[istar];
    const int RK = ws.cyc_rank[istar];
    const bool ratio = ws.transit != nullptr;
    // the frontier counters are first used after the barrier ending level 0
    if (leader) {
        for (int j = 0; j < 3; ++j) {
            c->fcnt[j] = 0;
            c->hcnt[0][j] = 0;   // listed pushing vertices with many in-edges
        }
    }

    // heavy vertices: their picks, then the list of pushing vertices with
    // many in-edges, live in the CSC scatter cursors, free once the
    // transposed graph is built
    const int H = c->cls_cnt[kClasses];
    const int *hv = ws.cls_list + c->cls_off[kClasses];
    const int htotal = c->heavy_edges;
    int *pick = sg.cursor;
    int *hin = sg.cursor + H;
    const int hcap = n - H;   // a vertex that finds the list full is walked where it is met

    // level 0: the vertices whose policy path ends on the chosen cycle
    int mine = 0, hmine = 0;
    for (int v = gtid; v < n; v += stride) {
        const bool in0 = (~ws.jls[0][v].J == rstar);
        sg.lev[v] = in0 ? 0 : -1;
        mine += !in0;
    }
    for (int i = gtid; i < H; i += stride) {
        pick[i] = INT_MAX;
        hmine += ~ws.jls[0][hv[i]].J != rstar;
    }
    bool ok;
    // vertices still unconnected, heavy ones among them
    int hleft = 0;
    int left = grid_sum_barrier_impl<true>(c, nb, mine, hmine, &hleft, &ok, kWaitFromCtrl,
                                           kBarConnect);
    if (!ok) return;
    // the heavy vertices at level `want` take the edges heavy_scan found
    // (and reset their picks); the sum of takes ends the phase
    auto heavy_take = [&](int want, int k, bool must) -> int {
        int took = 0;
        for (int i = gtid; i < H; i += stride) {
            const int v = hv[i];
            const int e = pick[i];
            pick[i] = INT_MAX;
            if (sg.lev[v] != want) continue;
            if (e != INT_MAX) {
                take_edge(v, e, k, rstar, P, Q, RK, ratio, sign, col, w, ws, sg);
                ++took;
            } else if (must) {
                atomicOr(&c->err, kErrConnect);   // a marked vertex has the edge
            }
        }
        return grid_sum_barrier(c, nb, took, &ok, kWaitFromCtrl, kBarConnect);
    };
    // the listed pushing vertices hin[0, nh): each one's in-edges spread over
    // one block (blocks take the list round-robin) or, above kInHeavyGrid,
    // over the whole grid; the loops run on block- or grid-uniform bounds so
    // that whole warps append.  claim: the list form (CAS claims, appended to
    // Fn, counted in added / hadded); else the pass form (plain marks).
    auto spread_push = [&](int nh, bool claim, int *Fn, int *cnt, int &added, int &hadded) {
        for (int j = 0; j < nh; ++j) {
            const int f = hin[j];
            const int e0 = sg.in_ptr[f], e1 = sg.in_ptr[f + 1];
            const bool grid = e1 - e0 > kInHeavyGrid;
            if (!grid && j % (int)gridDim.x != (int)blockIdx.x) continue;
            const int t0 = grid ? gtid : (int)threadIdx.x;
            const int step = grid ? stride : (int)blockDim.x;
            for (int base = e0; base < e1; base += step) {
                const int e = base + t0;
                bool take = false;
                int u = 0;
                if (e < e1) {
                    u = sg.in_src[e];
                    if (sg.lev[u] == -1) {
                        if (claim)
                            take = atomicCAS(&sg.lev[u], -1, -2) == -1;
                        else
                            sg.lev[u] = -2;
                    }
                }
                if (claim) {
                    append(Fn, cnt, take, u, lane);
                    added += take;
                    if (take && H > 0) hadded += row_ptr[u + 1] - row_ptr[u] > kHeavyEdges;
                }
            }
        }
    };
    constexpr int kPer = 32 / kConnectLanes;
    const int warp_id = gtid >> 5, nwarps = stride >> 5;
    const int grp = lane / kConnectLanes, sub = lane % kConnectLanes;
    int levels = 0;
    int nf = n - left;        // size of level k-1 (level 0 first)
    bool have_list = false;   // level k-1 is listed in fr[(k-1) & 1]
    for (int k = 1; left > 0; ++k) {
        if (k > n) {   // a search cannot have more levels than vertices
            if (leader) atomicOr(&c->err, kErrConnect);
            return;
        }
        int *F = sg.fr[(k - 1) & 1];
        int *Fn = sg.fr[k & 1];
        // counters rotate over three slots: the one reset here was last
        // appended to two levels ago and is next appended to at level k+1
        if (leader) {
            c->fcnt[(k + 1) % 3] = 0;
            c->hcnt[0][(k + 1) % 3] = 0;
        }
        int *hcount = &c->hcnt[0][k % 3];
        // A level of more than n/64 vertices is handled by passes over all
        // vertices (at most 64 such levels: the levels are disjoint), a
        // smaller one through a compact list.
        const bool big = (long long)nf * 64 > (long long)n;
        int found = 0;
        if (big) {
            // passes over all vertices, one thread per vertex, edges four at
            // a time (independent loads in flight).  pull: the unconnected
            // vertices look for an out-edge into levels < k (when fewer are
            // left than level k-1 holds); push: (a) level k-1 marks its
            // unconnected in-neighbours (-2, plain stores: every writer
            // writes the same), (b) the marked vertices pick their edge as in
            // the pull.
            const bool pull = left <= nf;
            if (!pull) {
                for (int v = gtid; v < n; v += stride) {
                    if (sg.lev[v] != k - 1) continue;
                    const int e0 = sg.in_ptr[v], e1 = sg.in_ptr[v + 1];
                    if (e1 - e0 > kInHeavy) {   // spread_push
                        const int pos = atomicAdd(hcount, 1);
                        if (pos < hcap) {
                            hin[pos] = v;
                            continue;
                        }
                    }
                    for (int e = e0; e < e1; e += 4) {
                        int u[4], l[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) u[j] = e + j < e1 ? sg.in_src[e + j] : -1;
#pragma unroll
                        for (int j = 0; j < 4; ++j) l[j] = u[j] >= 0 ? sg.lev[u[j]] : 0;
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (l[j] == -1) sg.lev[u[j]] = -2;
                    }
                }
                if (!grid_barrier(c, nb, kWaitFromCtrl, kBarConnect)) return;
                const int nh = min(load_volatile(hcount), hcap);
                if (nh > 0) {
                    int unused = 0, unused2 = 0;
                    spread_push(nh, false, nullptr, nullptr, unused, unused2);
                    if (!grid_barrier(c, nb, kWaitFromCtrl, kBarConnect)) return;
                }
            }
            const int want = pull ? -1 : -2;
            for (int u = gtid; u < n; u += stride) {
                if (sg.lev[u] != want) continue;
                const int e0 = row_ptr[u], e1 = row_ptr[u + 1];
                if (e1 - e0 > kHeavyEdges) continue;   // heavy_scan
                int pk = -1;
                for (int e = e0; e < e1 && pk < 0; e += 4) {
                    int l[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) l[j] = e + j < e1 ? sg.lev[col[e + j]] : -1;
#pragma unroll
                    for (int j = 3; j >= 0; --j)
                        if (l[j] >= 0 && l[j] < k) pk = e + j;   // the smallest index wins
                }
                if (pk >= 0) {
                    take_edge(u, pk, k, rstar, P, Q, RK, ratio, sign, col, w, ws, sg);
                    ++found;
                } else if (!pull) {
                    atomicOr(&c->err, kErrConnect);   // a marked vertex has the edge
                }
            }
            if (hleft > 0)
                heavy_scan(want, k, row_ptr, col, ws, sg, pick, H, hv, htotal, warp_id, nwarps,
                           lane);
            nf = grid_sum_barrier(c, nb, found, &ok, kWaitFromCtrl, kBarConnect);
            if (!ok) return;
            if (hleft > 0) {
                const int took = heavy_take(want, k, !pull);
                if (!ok) return;
                nf += took;
                hleft -= took;
            }
            have_list = false;
        } else {
            // push through lists: list level k-1 first if a pass made it
            if (!have_list) {
                for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
                    const int v = base + threadIdx.x;
                    append(F, &c->fcnt[(k - 1) % 3], v < n && sg.lev[v] == k - 1, v, lane);
                }
                if (!grid_barrier(c, nb, kWaitFromCtrl, kBarConnect)) return;
            }
            // (a) the unconnected in-neighbours of level k-1 are reached ...
            int added = 0, hadded = 0;
            const int ntask = (nf + kPer - 1) / kPer;
            for (int task = warp_id; task < ntask; task += nwarps) {
                const int i = task * kPer + grp;
                int e = 0, e1 = 0, f = -1;
                if (i < nf) {
                    f = F[i];
                    e = sg.in_ptr[f] + sub;
                    e1 = sg.in_ptr[f + 1];
                }
                // a vertex with many in-edges goes to spread_push
                const bool spread = f >= 0 && e1 - (e - sub) > kInHeavy;
                int pos = 0;
                if (spread && sub == 0) pos = atomicAdd(hcount, 1);
                pos = __shfl_sync(0xffffffffu, pos, grp * kConnectLanes);
                if (spread && pos < hcap) {
                    if (sub == 0) hin[pos] = f;
                    e1 = e;
                }
                for (;;) {
                    const bool more = e < e1;
                    if (!__any_sync(0xffffffffu, more)) break;
                    bool take = false;
                    int u = 0;
                    if (more) {
                        u = sg.in_src[e];
                        e += kConnectLanes;
                        if (sg.lev[u] == -1) take = atomicCAS(&sg.lev[u], -1, -2) == -1;
                    }
                    append(Fn, &c->fcnt[k % 3], take, u, lane);
                    added += take;
                    // (the degree loads only where heavy vertices exist)
                    if (take && H > 0) hadded += row_ptr[u + 1] - row_ptr[u] > kHeavyEdges;
                }
            }
            int hreached = 0;
            int reached = grid_sum_barrier_impl<true>(c, nb, added, hadded, &hreached, &ok,
                                                      kWaitFromCtrl, kBarConnect);
            if (!ok) return;
            const int nh = min(load_volatile(hcount), hcap);
            if (nh > 0) {
                int added2 = 0, hadded2 = 0, hreached2 = 0;
                spread_push(nh, true, Fn, &c->fcnt[k % 3], added2, hadded2);
                reached += grid_sum_barrier_impl<true>(c, nb, added2, hadded2, &hreached2, &ok,
                                                       kWaitFromCtrl, kBarConnect);
                if (!ok) return;
                hreached += hreached2;
            }
            // ... (b) and each takes its smallest out-edge into levels < k
            const int ntask2 = (reached + kPer - 1) / kPer;
            for (int task = warp_id; task < ntask2; task += nwarps) {
                const int i = task * kPer + grp;
                int u = -1, e = 0, e1 = 0;
                if (i < reached) {
                    u = Fn[i];
                    e = row_ptr[u] + sub;
                    e1 = row_ptr[u + 1];
                    if (e1 - (e - sub) > kHeavyEdges) {   // heavy_scan
                        u = -1;
                        e1 = e;
                    }
                }
                int pk = INT_MAX;
                for (; e < e1; e += kConnectLanes) {
                    const int l = sg.lev[col[e]];
                    if (l >= 0 && l < k) {
                        pk = e;
                        break;
                    }
                }
#pragma unroll
                for (int o = kConnectLanes / 2; o > 0; o >>= 1)
                    pk = min(pk, __shfl_xor_sync(0xffffffffu, pk, o));
                if (u >= 0 && sub == 0) {
                    if (pk == INT_MAX)
                        atomicOr(&c->err, kErrConnect);
                    else
                        take_edge(u, pk, k, rstar, P, Q, RK, ratio, sign, col, w, ws, sg);
                }
            }
            if (hreached > 0)
                heavy_scan(-2, k, row_ptr, col, ws, sg, pick, H, hv, htotal, warp_id, nwarps,
                           lane);
            if (!grid_barrier(c, nb, kWaitFromCtrl, kBarConnect)) return;
            if (hreached > 0) {
                heavy_take(-2, k, true);
                if (!ok) return;
                hleft -= hreached;
            }
            nf = reached;
            have_list = true;
        }
        if (nf == 0) break;   // the rest cannot reach the chosen cycle
        left -= nf;
        ++levels;
    }
    if (leader) {
        if (left > 0) atomicOr(&c->err, kErrUnreached);
        c->connect_levels += levels;
        c->nrep = 1;   // the chosen cycle is now the only one
    }
}

static int connect_grid() {
    static int cached_dev = -1, cached = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev == cached_dev && cached > 0) return cached;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, connect_kernel, kConnectThreads,
                                                      0) != cudaSuccess ||
        per_sm < 1)
        return 0;
    cached_dev = dev;
    cached = sms * per_sm;
    return cached;
}

int prepare_connect() { return connect_grid() > 0 ? 0 : -1; }

int launch_connect(const int *row_ptr, const int *col, const int *w, int sign, int n,
                   Workspace ws, SingleWs sw, cudaStream_t st) {
    int blocks = connect_grid();
    if (blocks <= 0) return -1;
    const int need = (n + kConnectThreads - 1) / kConnectThreads;
    if (need < blocks) blocks = need;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kConnectThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    prof_begin(kProfEvaluate, st);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, connect_kernel, row_ptr, col, w, sign, n, ws, sw);
    prof_end(kProfEvaluate, st);
    return e == cudaSuccess ? 1 : -1;
}

}  // namespace ocm
