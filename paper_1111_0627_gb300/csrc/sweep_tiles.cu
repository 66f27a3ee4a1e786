// sweep_tiles.cu -- the improvement sweep (Alg. 1's pass over all vertices,
// Alg. 2 SPFPassIter) as one pass over the CSR edge array in fixed tiles.
//
// The sweep is a streaming pass: 8 bytes of col_idx and w per edge, one
// 16-byte record gather per edge (rec[t] = V(t), rank(t), q_t), and a little
// per-vertex state.  Cutting the edge array into equal, aligned tiles of
// ET = 32 * K edges (K edges per lane) makes every load of col_idx and w a
// 16-byte vector load, gives every warp the same amount of work whatever the
// degree distribution, and visits the targets in CSR order, so the records a
// tile gathers are the ones its neighbours gather too (good L2 reuse when
// targets are local, as in BFS-numbered state spaces).
//
// Per tile, a warp:
//   1. copies row_ptr[v+1] and pi[v] of the tile's vertices into shared
//      memory (the tile's first vertex comes from tile_v, built once per solve);
//   2. lets every lane scan its K consecutive edges, keeping the best candidate
//      (rank, key, -e) of the vertex it is in and, when it meets the vertex's
//      current policy edge pi[v], that edge's key; vertices whose edges begin
//      and end inside the lane are decided on the spot;
//   3. joins vertices that cross lane boundaries with a segmented suffix scan
//      over the lanes (5 shuffle steps); the lane holding a vertex's first
//      edge decides it;
//   4. records the partial result of the (at most one) vertex that runs past
//      the tile's end, and of the vertex that entered from the previous tile.
// A small fix-up kernel then decides the vertices that span tiles, combining
// the per-tile partials in edge order.  A vertex switches only on a strict
// improvement over its current policy edge (Alg. 1: strict ">"), exactly as
// in the degree-class sweep, so both give the same policy.
#include <climits>

#include "common.cuh"

namespace ocm {

// Key of a vertex's current policy edge; rank INT_MIN = not seen yet.
struct CurKey {
    int rank;
    long long key;
};

__device__ __forceinline__ Cand no_cand() { return Cand{INT_MIN, INT_MAX, LLONG_MIN}; }

// Decides vertex v: switch to its best edge b if that strictly improves on
// the current edge's key c.  colp / wp hold col_idx and w of edges from
// `base` on (a tile staged in shared memory, or the global arrays with base
// 0).  Returns 1 on a switch.
static __device__ __forceinline__ int decide(int v, const Cand &b, const CurKey &c,
                                             const int *colp, const int *wp, int base, int sign,
                                             int next_eval, const Workspace &ws,
                                             const BatchState &bs) {
    // batched: a graph that stopped changing keeps its policy (its records
    // are frozen, so nothing can improve there; the tiles that lie wholly
    // inside it are skipped, so its partials may be stale)
    if (bs.G && bs.gconv[bs.gid[v]]) return 0;
    if (c.rank == INT_MIN) {   // pi[v] is always one of v's edges
        atomicOr(&ws.ctrl->err, kErrSweep);
        return 0;
    }
    if (!(b.rank > c.rank || (b.rank == c.rank && b.key > c.key))) return 0;
    ws.pi[v] = b.e;
    ws.succ[v] = colp[b.e - base];
    ws.wpi[v] = sign * wp[b.e - base];
    ws.sw_iter[v] = next_eval;
    if (bs.G) {
        const int g = bs.gid[v];
        if (bs.gsw[g] != next_eval) bs.gsw[g] = next_eval;
    }
    return 1;
}

static __device__ __forceinline__ Cand shfl_down_cand(const Cand &a, int d) {
    Cand o;
    o.rank = __shfl_down_sync(0xffffffffu, a.rank, d);
    o.e = __shfl_down_sync(0xffffffffu, a.e, d);
    o.key = __shfl_down_sync(0xffffffffu, a.key, d);
    return o;
}

static __device__ __forceinline__ CurKey shfl_down_cur(const CurKey &a, int d) {
    CurKey o;
    o.rank = __shfl_down_sync(0xffffffffu, a.rank, d);
    o.key = __shfl_down_sync(0xffffffffu, a.key, d);
    return o;
}

// tile_v[t] = the vertex owning edge t * ET (every vertex has an out-edge, so
// the tiles that start inside [row_ptr[v], row_ptr[v+1]) are exactly v's).
__global__ void __launch_bounds__(kThreads)
tile_index_kernel(const int *__restrict__ row_ptr, int n, int et, int tiles, int *tile_v) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const long long a = __ldg(&row_ptr[v]), b = __ldg(&row_ptr[v + 1]);
        long long t = (a + et - 1) / et;
        const long long t_end = (b + et - 1) / et;
        for (; t < t_end && t < tiles; ++t) tile_v[t] = v;
    }
}

int launch_tile_index(const int *row_ptr, int n, int m, int tile_edges, Workspace ws,
                      cudaStream_t st) {
    const int tiles = (int)(((long long)m + tile_edges - 1) / tile_edges);
    int blocks = (n + kThreads - 1) / kThreads;
    if (blocks > 4096) blocks = 4096;
    prof_begin(kProfInit, st);
    tile_index_kernel<<<blocks, kThreads, 0, st>>>(row_ptr, n, tile_edges, tiles, ws.tile_v);
    prof_end(kProfInit, st);
    return 1;
}

// ---- asynchronous global -> shared copies (cp.async), per lane
static __device__ __forceinline__ unsigned smem_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
static __device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}
static __device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}
static __device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
static __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared-memory stages of one warp: the edge arrays of three tiles (the one
// being computed and two in flight), and for two tiles the gathered records
// and row_ptr / pi of their vertices.
template <int K>
struct __align__(16) TileStages {
    static constexpr int ET = 32 * K;
    int4 rec[2][ET];
    int col[3][ET];
    int w[3][ET];
    int rp[2][ET + 4];   // row_ptr[vb .. ve+1]
    int pi[2][ET + 4];   // pi[vb .. ve]
};

template <int K>
__global__ void __launch_bounds__(256)
improve_tiles_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col,
                     const int *__restrict__ w, int sign, int n, int m, int tiles, int vec,
                     Workspace ws, BatchState bs) {
    constexpr int ET = 32 * K;
    extern __shared__ int4 s_stage[];
    __shared__ int s_sw;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    if (tid == 0) s_sw = 0;
    if (blockIdx.x == 0 && tid == 0) publish_result(ws, n);
    __syncthreads();
    TileStages<K> &S = reinterpret_cast<TileStages<K> *>(s_stage)[tid >> 5];
    const int next_eval = ws.ctrl->iter + 1;   // switched vertices are dirty for it
    const int4 *rec = reinterpret_cast<const int4 *>(ws.rec);
    const int gw = (blockIdx.x * blockDim.x + tid) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;

    // stage A: the tile's col_idx and w (16-byte copies when aligned and full)
    auto issue_edges = [&](int t, int slot) {
        const int e0 = t * ET;
        const int e_end = (m - e0 < ET) ? m : e0 + ET;
        if (lane * K >= e_end - e0) return;
        const int ea = e0 + lane * K;
        const int cnt = min(K, e_end - ea);
        if (vec && cnt == K) {
#pragma unroll
            for (int k = 0; k < K; k += 4) {
                cp_async16(&S.col[slot][lane * K + k], col + ea + k);
                cp_async16(&S.w[slot][lane * K + k], w + ea + k);
            }
        } else {
            for (int k = 0; k < cnt; ++k) {
                cp_async4(&S.col[slot][lane * K + k], col + ea + k);
                cp_async4(&S.w[slot][lane * K + k], w + ea + k);
            }
        }
    };
    // stage B: the records of the tile's targets, and row_ptr / pi of its vertices
    auto issue_gather = [&](int t, int slot_a, int slot_b, int vb, int ve) {
        const int e0 = t * ET;
        const int e_end = (m - e0 < ET) ? m : e0 + ET;
        if (lane * K < e_end - e0) {
            const int cnt = min(K, e_end - e0 - lane * K);
            for (int k = 0; k < cnt; ++k)
                cp_async16(&S.rec[slot_b][lane * K + k], rec + S.col[slot_a][lane * K + k]);
        }
        const int nv = ve - vb + 1;
        for (int i = lane; i <= nv; i += 32) cp_async4(&S.rp[slot_b][i], row_ptr + vb + i);
        for (int i = lane; i < nv; i += 32) cp_async4(&S.pi[slot_b][i], ws.pi + vb + i);
    };
    auto first_vertex = [&](int t) { return __ldg(&ws.tile_v[t]); };
    auto last_vertex = [&](int t) { return (t + 1 < tiles) ? __ldg(&ws.tile_v[t + 1]) : n - 1; };

    // prologue: edges of the first two tiles, records of the first
    int vb0 = 0, ve0 = 0, vb1 = 0, ve1 = 0, vb2 = 0, ve2 = 0;
    if (gw < tiles) {
        issue_edges(gw, 0);
        vb0 = first_vertex(gw);
        ve0 = last_vertex(gw);
    }
    cp_async_commit();
    if (gw + nw < tiles) {
        issue_edges(gw + nw, 1);
        vb1 = first_vertex(gw + nw);
        ve1 = last_vertex(gw + nw);
    }
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();
    if (gw < tiles) issue_gather(gw, 0, 0, vb0, ve0);
    cp_async_commit();

    int switched = 0;
    int j = 0;
    for (int t = gw; t < tiles; t += nw, ++j) {
        const int sa = j % 3, sb = j & 1;
        // ---- keep two tiles in flight
        const int t1 = t + nw, t2 = t + 2 * nw;
        if (t2 < tiles) {
            issue_edges(t2, (j + 2) % 3);
            vb2 = first_vertex(t2);
            ve2 = last_vertex(t2);
        }
        cp_async_commit();
        cp_async_wait<2>();   // edges of t1 have landed
        __syncwarp();
        if (t1 < tiles) issue_gather(t1, (j + 1) % 3, (j + 1) & 1, vb1, ve1);
        cp_async_commit();
        cp_async_wait<2>();   // records of t have landed
        __syncwarp();

        // ---- compute tile t from shared memory
        const int e0 = t * ET;
        const int e_end = (m - e0 < ET) ? m : e0 + ET;
        const int vb = vb0, ve = ve0;
        bool skip = false;
        if (bs.G) {
            // batched: a tile inside one converged graph has nothing to do
            const int g0 = bs.gid[vb];
            skip = g0 == bs.gid[ve] && bs.gconv[g0];
        }
        if (skip) {
            if (lane == 0) {
                ws.tile_pend[t] = -1;
                ws.tile_fopen[t] = 0;
            }
        } else {
            const int *rp = S.rp[sb];        // rp[i] = row_ptr[vb + i]
            const int *sp = S.pi[sb];
            const int *tcol = S.col[sa];
            const int *tw = S.w[sa];
            const int4 *trec = S.rec[sb];
            const int nv = ve - vb + 1;
            const int head0 = rp[0];
            const bool live = lane * K < e_end - e0;
            const int ea = live ? e0 + lane * K : e0;
            const int cnt = live ? min(K, e_end - ea) : 0;
            int i = 0;   // index (from vb) of the vertex owning edge ea
            if (live) {
                int lo = 0, hi = nv - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (rp[mid + 1] > ea) hi = mid; else lo = mid + 1;
                }
                i = lo;
            }
            const int i0 = i;
            const bool f_head = live && rp[i] == ea;
            int seg_end = live ? rp[i + 1] : 0;
            int seg_pi = live ? sp[i] : -1;
            Cand best = no_cand();
            CurKey cur{INT_MIN, 0};
            Cand fbest = best;       // the lane's first vertex, once it is closed
            CurKey fcur = cur;
            bool multi = false;      // the lane has seen a vertex boundary
            for (int k = 0; k < cnt; ++k) {
                const int e = ea + k;
                if (e >= seg_end) {   // the vertex at i ends before e
                    if (!multi) {
                        fbest = best;
                        fcur = cur;
                        multi = true;
                    } else {          // begun and ended in this lane
                        switched += decide(vb + i, best, cur, tcol, tw, e0, sign,
                                           next_eval, ws, bs);
                    }
                    ++i;
                    seg_end = rp[i + 1];
                    seg_pi = sp[i];
                    best = no_cand();
                    cur = CurKey{INT_MIN, 0};
                }
                const int4 r = trec[lane * K + k];
                const long long V = ((long long)(unsigned)r.x) | ((long long)r.y << 32);
                const Cand c{r.z, e, (long long)r.w * (long long)(sign * tw[lane * K + k]) + V};
                if (better(c, best)) best = c;
                if (e == seg_pi) cur = CurKey{c.rank, c.key};
            }
            const bool l_open = live && seg_end > ea + cnt;   // the last vertex goes on
            bool f_closed = true;
            if (!multi) {
                fbest = best;
                fcur = cur;
                f_closed = !l_open;
            }
            if (multi && !l_open)
                switched += decide(vb + i, best, cur, tcol, tw, e0, sign, next_eval, ws, bs);
            if (f_head && f_closed)
                switched += decide(vb + i0, fbest, fcur, tcol, tw, e0, sign, next_eval, ws,
                                   bs);

            // vertices crossing lanes: suffix scan of the first-vertex
            // partials; "open" = the vertex continues past the covered lanes
            Cand sbst = fbest;
            CurKey scur = fcur;
            int so = f_closed ? 0 : 1;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const Cand ob = shfl_down_cand(sbst, d);
                const CurKey oc = shfl_down_cur(scur, d);
                const int oo = __shfl_down_sync(0xffffffffu, so, d);
                if (lane + d < 32 && so) {
                    if (better(ob, sbst)) sbst = ob;
                    if (oc.rank != INT_MIN) scur = oc;
                    so = oo;
                }
            }
            const Cand nb = shfl_down_cand(sbst, 1);
            const CurKey nc = shfl_down_cur(scur, 1);
            const int no = __shfl_down_sync(0xffffffffu, so, 1);
            int pend = 0;
            if (l_open && (multi || f_head)) {   // this lane holds the vertex's first edge
                Cand b = best;
                CurKey c = cur;
                bool off = true;                 // lane 31: runs into the next tile
                if (lane < 31) {
                    if (better(nb, b)) b = nb;
                    if (nc.rank != INT_MIN) c = nc;
                    off = no != 0;
                }
                if (!off) {
                    switched += decide(vb + i, b, c, tcol, tw, e0, sign, next_eval, ws, bs);
                } else {
                    ws.tile_last[t] = TilePart{b.rank, b.e, b.key, c.rank, 0, c.key};
                    ws.tile_pend[t] = vb + i;
                    pend = 1;
                }
            }
            // the tile's summary for the fix-up
            if (__ballot_sync(0xffffffffu, pend) == 0 && lane == 0) ws.tile_pend[t] = -1;
            if (lane == 0) {
                if (head0 < e0)
                    ws.tile_first[t] = TilePart{sbst.rank, sbst.e, sbst.key, scur.rank, 0, scur.key};
                ws.tile_fopen[t] = (head0 < e0) ? so : 0;
            }
        }
        __syncwarp();   // this tile's stages are refilled from the next iteration on
        vb0 = vb1;
        ve0 = ve1;
        vb1 = vb2;
        ve1 = ve2;
    }
    cp_async_wait<0>();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) switched += __shfl_xor_sync(0xffffffffu, switched, o);
    if (lane == 0 && switched) atomicAdd(&s_sw, switched);
    __syncthreads();
    if (tid == 0 && s_sw) {
        atomicAdd(&ws.ctrl->switched, s_sw);
        ws.ctrl->changed = 1;
    }
}

// Vertices whose edges span tiles: starting from the partial of the tile
// holding the first edge, add the partials of the following tiles while the
// vertex goes on, 32 tiles per step (one per lane), then decide.
__global__ void __launch_bounds__(kThreads)
improve_fixup_kernel(const int *__restrict__ col, const int *__restrict__ w, int sign, int tiles,
                     Workspace ws, BatchState bs) {
    __shared__ int s_sw;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    if (tid == 0) s_sw = 0;
    __syncthreads();
    const int next_eval = ws.ctrl->iter + 1;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int switched = 0;
    for (int base = ((blockIdx.x * blockDim.x + tid) >> 5) * 32; base < tiles; base += nw * 32) {
        const int t = base + lane;
        const int v = (t < tiles) ? ws.tile_pend[t] : -1;
        unsigned todo = __ballot_sync(0xffffffffu, v >= 0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int tt = base + src;
            const int vv = __shfl_sync(0xffffffffu, v, src);
            const TilePart L = ws.tile_last[tt];
            Cand b{L.rank, L.e, L.key};
            CurKey c{L.crank, L.ckey};
            for (int u0 = tt + 1; u0 < tiles; u0 += 32) {
                const int u = u0 + lane;
                Cand pb = no_cand();
                CurKey pc{INT_MIN, 0};
                int open = 0;
                if (u < tiles) {
                    const TilePart F = ws.tile_first[u];
                    pb = Cand{F.rank, F.e, F.key};
                    pc = CurKey{F.crank, F.ckey};
                    open = ws.tile_fopen[u];
                }
                // tiles up to and including the first one where the vertex ends
                const unsigned stop = __ballot_sync(0xffffffffu, u >= tiles || !open);
                const int last = stop ? __ffs(stop) - 1 : 31;
                const bool take = lane <= last && u < tiles;
                if (!take) {
                    pb = no_cand();
                    pc = CurKey{INT_MIN, 0};
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    Cand ob;
                    ob.rank = __shfl_xor_sync(0xffffffffu, pb.rank, o);
                    ob.e = __shfl_xor_sync(0xffffffffu, pb.e, o);
                    ob.key = __shfl_xor_sync(0xffffffffu, pb.key, o);
                    const int ocr = __shfl_xor_sync(0xffffffffu, pc.rank, o);
                    const long long ock = __shfl_xor_sync(0xffffffffu, pc.key, o);
                    if (better(ob, pb)) pb = ob;
                    if (ocr != INT_MIN) pc = CurKey{ocr, ock};
                }
                if (better(pb, b)) b = pb;
                if (pc.rank != INT_MIN) c = pc;
                if (stop) break;
            }
            if (lane == 0) switched += decide(vv, b, c, col, w, 0, sign, next_eval, ws, bs);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) switched += __shfl_xor_sync(0xffffffffu, switched, o);
    if (lane == 0 && switched) atomicAdd(&s_sw, switched);
    __syncthreads();
    if (tid == 0 && s_sw) {
        atomicAdd(&ws.ctrl->switched, s_sw);
        ws.ctrl->changed = 1;
    }
}

namespace {

// Co-resident blocks of the tiled sweep for (K, block size) on the current
// device, with the shared-memory opt-in done once per device.  Host-side
// configuration only: it runs before any launch is captured into a graph.
template <int K>
int tiles_grid(int threads) {
    static int cached_dev[3] = {-1, -1, -1}, cached_blocks[3] = {0, 0, 0};
    static int optin_dev = -1;
    const int slot = threads == 64 ? 0 : threads == 128 ? 1 : 2;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (optin_dev != dev) {
        // the largest block (256 threads), so no later call lowers the limit
        if (cudaFuncSetAttribute(improve_tiles_kernel<K>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(8 * sizeof(TileStages<K>))) != cudaSuccess)
            return 0;
        optin_dev = dev;
    }
    if (cached_dev[slot] != dev) {
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, improve_tiles_kernel<K>, threads,
                (size_t)(threads / 32) * sizeof(TileStages<K>)) != cudaSuccess ||
            sms <= 0 || per_sm <= 0)
            return 0;
        cached_blocks[slot] = sms * per_sm;
        cached_dev[slot] = dev;
    }
    return cached_blocks[slot];
}

int tiles_threads(int threads) { return threads <= 64 ? 64 : threads <= 128 ? 128 : 256; }

template <int K>
int launch_tiles_k(const int *row_ptr, const int *col, const int *w, int sign, int n, int m,
                   Workspace ws, BatchState bs, int threads, cudaStream_t st) {
    constexpr int ET = 32 * K;
    const int tiles = (int)(((long long)m + ET - 1) / ET);
    const size_t smem = (size_t)(threads / 32) * sizeof(TileStages<K>);
    const int grid = tiles_grid<K>(threads);
    if (grid <= 0) return -1;
    const int wpb = threads / 32;
    int blocks = (tiles + wpb - 1) / wpb;
    if (blocks > grid) blocks = grid;
    const int vec = ((reinterpret_cast<uintptr_t>(col) | reinterpret_cast<uintptr_t>(w)) & 15u) ? 0 : 1;
    prof_begin(kProfSweep, st);
    improve_tiles_kernel<K><<<blocks, threads, smem, st>>>(row_ptr, col, w, sign, n, m, tiles, vec,
                                                           ws, bs);
    int fb = (tiles + kThreads - 1) / kThreads;   // one warp per 32 tiles
    if (fb > 2048) fb = 2048;
    improve_fixup_kernel<<<fb, kThreads, 0, st>>>(col, w, sign, tiles, ws, bs);
    prof_end(kProfSweep, st);
    return 2;
}

}  // namespace

// Host-side configuration of the tiled sweep (see tiles_grid); 0 on success.
int prepare_sweep_tiles(int edges_per_lane, int threads) {
    threads = tiles_threads(threads);
    const int g = (edges_per_lane <= 4) ? tiles_grid<4>(threads) : tiles_grid<8>(threads);
    return g > 0 ? 0 : -1;
}

int launch_sweep_tiles(const int *row_ptr, const int *col, const int *w, int sign, int n, int m,
                       int edges_per_lane, Workspace ws, BatchState bs, int threads,
                       cudaStream_t st) {
    // each warp stages three tiles in shared memory, so blocks stay small:
    // 64, 128 or 256 threads (a requested 512 runs as 256)
    threads = tiles_threads(threads);
    if (edges_per_lane <= 4) return launch_tiles_k<4>(row_ptr, col, w, sign, n, m, ws, bs, threads, st);
    return launch_tiles_k<8>(row_ptr, col, w, sign, n, m, ws, bs, threads, st);
}

}  // namespace ocm
