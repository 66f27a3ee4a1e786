// batch_small.cu -- the batched form's persistent per-graph solver.
//
// The regions of Sec. 3.3 are independent; for the small ones a whole Howard
// iteration (Alg. 1: evaluate the policy, improve it, stop when stable) fits
// one thread block.  A persistent grid of blocks pops graph tasks from a queue
// ordered by decreasing size (a log2 bucket per size class, the largest
// first, so the longest tasks start first), and every block runs all
// iterations of its graph with block barriers only: no grid barrier and no
// launch per iteration.  Each graph converges on its own (the paper's per-
// region "work" flag becomes the end of the block's loop) and leaves its
// answer in the per-graph records of the batch; the larger graphs go through
// the disjoint-union path of batch.cu / evaluate.cu / sweep.cu, which skips
// the graphs solved here.
//
// Every step computes what the union path computes, with the same order and
// tie rules (cycle root = smallest vertex, V = q*S - p*len, improvement key
// q_t*s*w(e) + V(t) compared within equal mean rank, strict switching, ties to
// the smaller edge index), so every graph follows the trajectory the oracle
// follows for that graph alone.  State lives in the batch workspace at the
// graph's own vertex range (and its cycle records at the same offsets), where
// it stays in L1/L2 while the block works on it.
#include <climits>

#include "common.cuh"
#include "grid_sync.cuh"

namespace ocm {

constexpr int kSmallThreads = 1024;
constexpr int kSU = 4;   // vertices per thread per pass of a jump round (64 registers)
constexpr int kSmallBuckets = 32;
// Shared-memory words for the leaf bitmaps of one graph (two bitmap words and
// a prefix word per 32 vertices: graphs up to 512K vertices are trimmed).
constexpr int kSmallBitmapWords = 49152;

// Size buckets of the queue: floor(log2(n_g)), largest first.
static __device__ __forceinline__ int size_bucket(int n) { return 31 - __clz(n); }

static __device__ __forceinline__ bool small_eligible(const BatchState &bs,
                                                      const int *__restrict__ row_ptr, int g,
                                                      int max_n, int *n_out) {
    const int a = bs.vptr[g], b = bs.vptr[g + 1];
    const int n = b - a;
    const long long m = (long long)row_ptr[b] - row_ptr[a];
    *n_out = n;
    return n <= max_n && m <= 16LL * max_n;
}

__global__ void __launch_bounds__(kThreads)
small_count_kernel(const int *__restrict__ row_ptr, BatchState bs, int max_n, Ctrl *c) {
    __shared__ int s_cnt[kSmallBuckets];
    if (threadIdx.x < kSmallBuckets) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < bs.G; g += gridDim.x * blockDim.x) {
        int n;
        if (small_eligible(bs, row_ptr, g, max_n, &n)) atomicAdd(&s_cnt[size_bucket(n)], 1);
    }
    __syncthreads();
    if (threadIdx.x < kSmallBuckets && s_cnt[threadIdx.x])
        atomicAdd(&c->small_bucket[threadIdx.x], s_cnt[threadIdx.x]);
}

// Queue positions: bucket b (larger b first) starts after all larger buckets;
// within a bucket the order is that of the atomics (it decides only which
// block solves which graph, never a result).
__global__ void __launch_bounds__(kThreads)
small_fill_kernel(const int *__restrict__ row_ptr, BatchState bs, int max_n, Ctrl *c,
                  int *queue) {
    __shared__ int s_start[kSmallBuckets];
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = kSmallBuckets - 1; b >= 0; --b) {
            s_start[b] = run;
            run += c->small_bucket[b];
        }
        if (blockIdx.x == 0) c->small_total = run;
    }
    __syncthreads();
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < bs.G; g += gridDim.x * blockDim.x) {
        int n;
        if (small_eligible(bs, row_ptr, g, max_n, &n)) {
            const int b = size_bucket(n);
            queue[s_start[b] + atomicAdd(&c->small_cursor[b], 1)] = g;
        }
    }
}

// Block-wide sum (all threads call it).
static __device__ __forceinline__ int block_sum(int x, int *s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = x;
    __syncthreads();
    int t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_red[k];
    __syncthreads();
    return t;
}

// Inclusive sum over the block (all threads call it).
static __device__ __forceinline__ int block_scan_incl(int x, int *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int wv = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wv, o);
            if (lane >= o) wv += y;
        }
        s_warp[lane] = wv;
    }
    __syncthreads();
    const int r = x + (warp > 0 ? s_warp[warp - 1] : 0);
    __syncthreads();
    return r;
}

// Policy evaluation of graph [v0, v1) inside one block, the steps of
// evaluate_kernel over every vertex that is no leaf in every round (no
// worklists: a graph's state stays in L1/L2 while its block works on it, and
// a dense pass costs less than keeping lists): cycle detection by doubling
// with window minima, resolved vertices holding J = ~root; then value
// propagation with (len, S) until the root, which is terminal.  On return
// every vertex has its root (rep), its final (~root, len, S) in jls[0], its
// record {V, rank, q}; the cycle records sit at [v0, v0 + K) and the packed
// best (rank, INT_MAX - root) in *s_best.  Returns false on an error
// (recorded in the control block).
static __device__ bool small_evaluate(int v0, int v1, const Workspace &ws, int *s_red, int *s_k,
                                      unsigned long long *s_best, unsigned *bits, int nwords,
                                      unsigned *dirty, int *n_dirty) {
    const int n = v1 - v0;
    int lg = 0;
    while ((1 << lg) < n) ++lg;
    Ctrl *c = ws.ctrl;
    const int Wt = blockDim.x;
    // Vertices nobody points to (leaves), and those whose predecessors are
    // all leaves, lie on no cycle and no other vertex jumps to them: when the
    // graph's bitmaps fit in shared memory the others are renumbered densely
    // (rank in the "has a predecessor that is no leaf" bitmap) and the jump
    // rounds run on that dense space; the leaves take their successor's final
    // state at the end.
    const int nw = (n + 31) / 32;
    const bool trim = nwords > 0 && 3 * nw <= nwords;
    unsigned *keepb = bits + nw, *pref = bits + 2 * nw;
    int nk = n;
    if (trim) {
        for (int i = threadIdx.x; i < 2 * nw; i += Wt) bits[i] = 0u;
        __syncthreads();
        for (int v = v0 + (int)threadIdx.x; v < v1; v += Wt) {
            const int l = ws.succ[v] - v0;
            atomicOr(&bits[l >> 5], 1u << (l & 31));
        }
        __syncthreads();
        for (int v = v0 + (int)threadIdx.x; v < v1; v += Wt) {
            const int lv = v - v0;
            if ((bits[lv >> 5] >> (lv & 31)) & 1u) {
                const int l = ws.succ[v] - v0;
                atomicOr(&keepb[l >> 5], 1u << (l & 31));
            }
        }
        __syncthreads();
        const int per = (nw + Wt - 1) / Wt;
        const int w0 = min(nw, (int)threadIdx.x * per), w1 = min(nw, w0 + per);
        int sum = 0;
        for (int i = w0; i < w1; ++i) sum += __popc(keepb[i]);
        __shared__ int s_warp[32];
        __shared__ int s_total;
        const int incl = block_scan_incl(sum, s_warp);
        int run = incl - sum;
        for (int i = w0; i < w1; ++i) {
            pref[i] = (unsigned)run;
            run += __popc(keepb[i]);
        }
        if (threadIdx.x == Wt - 1) s_total = incl;
        __syncthreads();
        nk = s_total;
    }
    auto dense = [&](int v) -> int {
        const int l = v - v0;
        return trim ? (int)pref[l >> 5] + __popc(keepb[l >> 5] & ((1u << (l & 31)) - 1u)) : l;
    };
    auto kept = [&](int v) -> bool {
        const int l = v - v0;
        return !trim || ((keepb[l >> 5] >> (l & 31)) & 1u);
    };
    auto leaf1 = [&](int v) -> bool {
        const int l = v - v0;
        return trim && !((bits[l >> 5] >> (l & 31)) & 1u);
    };
    int *orig = ws.aprev + v0;    // dense index -> vertex
    int *ap = ws.list[0] + v0;    // previous window minimum, per dense index
    // ---- cycle detection on the dense space (window minima of vertex ids)
    JM *X = ws.jm[0] + v0, *Y = ws.jm[1] + v0;
    for (int v = v0 + (int)threadIdx.x; v < v1; v += Wt) {
        if (!kept(v)) continue;
        const int d = dense(v);
        orig[d] = v;
        X[d] = JM{dense(ws.succ[v]), v};
    }
    __syncthreads();
    for (int r = 0;; ++r) {
        int pend = 0;
        for (int base = (int)threadIdx.x; base < nk; base += kSU * Wt) {
            JM sj[kSU], tj[kSU];
#pragma unroll
            for (int u = 0; u < kSU; ++u) {
                const int d = base + u * Wt;
                sj[u] = d < nk ? X[d] : JM{-1, 0};
            }
#pragma unroll
            for (int u = 0; u < kSU; ++u)
                if (sj[u].J >= 0) tj[u] = X[sj[u].J];
#pragma unroll
            for (int u = 0; u < kSU; ++u) {
                const int d = base + u * Wt;
                if (d >= nk) continue;
                if (sj[u].J < 0) { Y[d] = sj[u]; continue; }
                int root = -1;
                if (tj[u].J < 0) root = ~tj[u].J;
                else if (r > 0 && tj[u].M == ap[d]) root = tj[u].M;
                if (root >= 0) { Y[d] = JM{~root, 0}; ws.rep[orig[d]] = root; }
                else { Y[d] = JM{tj[u].J, min(sj[u].M, tj[u].M)}; ap[d] = tj[u].M; ++pend; }
            }
        }
        JM *tmp = X; X = Y; Y = tmp;
        if (block_sum(pend, s_red) == 0) break;
        if (r + 1 > lg + 4) { if (threadIdx.x == 0) atomicOr(&c->err, kErrDetect); return false; }
    }
    // ---- values on the dense space, the root terminal (final J = ~root)
    JLS *A = ws.jls[1] + v0, *B = reinterpret_cast<JLS *>(ws.scratch16) + v0;
    for (int d = (int)threadIdx.x; d < nk; d += Wt) {
        const int v = orig[d];
        const int root = ws.rep[v];
        JLS st;
        if (root == v) {
            st = JLS{~v, 0, 0};
        } else {
            const int sv = ws.succ[v];
            st = ws.rep[sv] == sv ? JLS{~sv, 1, (long long)ws.wpi[v]}
                                  : JLS{dense(sv), 1, (long long)ws.wpi[v]};
        }
        A[d] = st;
    }
    __syncthreads();
    for (int r = 0;; ++r) {
        int pend = 0;
        for (int base = (int)threadIdx.x; base < nk; base += kSU * Wt) {
            JLS sj[kSU], tj[kSU];
#pragma unroll
            for (int u = 0; u < kSU; ++u) { const int d = base + u * Wt; sj[u] = d < nk ? A[d] : JLS{-1, 0, 0}; }
#pragma unroll
            for (int u = 0; u < kSU; ++u) if (sj[u].J >= 0) tj[u] = A[sj[u].J];
#pragma unroll
            for (int u = 0; u < kSU; ++u) {
                const int d = base + u * Wt;
                if (d >= nk) continue;
                if (sj[u].J < 0) { B[d] = sj[u]; continue; }
                const JLS nu{tj[u].J, sj[u].len + tj[u].len, sj[u].S + tj[u].S};
                B[d] = nu; pend += nu.J >= 0;
            }
        }
        JLS *tmp = A; A = B; B = tmp;
        if (block_sum(pend, s_red) == 0) break;
        if (r + 1 > lg + 3) { if (threadIdx.x == 0) atomicOr(&c->err, kErrValue); return false; }
    }
    // final states at the vertices' own indices (jls[0], which the extraction
    // reads), then the leaves: second level first, from their successors
    for (int d = (int)threadIdx.x; d < nk; d += Wt) ws.jls[0][orig[d]] = A[d];
    __syncthreads();
    for (int pass = 0; pass < 2 && trim; ++pass) {
        for (int v = v0 + (int)threadIdx.x; v < v1; v += Wt) {
            if (kept(v) || leaf1(v) != (pass == 1)) continue;
            const JLS f = ws.jls[0][ws.succ[v]];
            ws.jls[0][v] = JLS{f.J, f.len + 1, f.S + (long long)ws.wpi[v]};
            ws.rep[v] = ~f.J;
        }
        __syncthreads();
    }
    const unsigned W = blockDim.x;
    A = ws.jls[0];
    // ---- cycles: mean W/L reduced, exact key, rank among this graph's cycles
    if (threadIdx.x == 0) {
        *s_k = 0;
        *s_best = 0;
    }
    __syncthreads();
    const long long N2 = (long long)n * n;
    for (int v = v0 + (int)threadIdx.x; v < v1; v += W) {
        if (ws.rep[v] != v) continue;
        const int x = ws.succ[v];
        const JLS st = A[x];
        const long long Wc = (long long)ws.wpi[v] + st.S;
        const long long L = 1 + (long long)st.len;
        const long long g = gcd_ll(Wc, L);
        const int i = v0 + atomicAdd(s_k, 1);
        ws.cyc_root[i] = v;
        ws.cyc_p[i] = Wc / g;
        ws.cyc_q[i] = (int)(L / g);
        ws.cyc_L[i] = (int)L;
        ws.cyc_key[i] = mean_key(Wc / g, L / g, N2);
        ws.cid_of_root[v] = i;
    }
    __syncthreads();
    const int K = *s_k;
    for (int i = v0 + (int)threadIdx.x; i < v0 + K; i += W) {
        const long long key = ws.cyc_key[i];
        int rank = 0;
        for (int j = v0; j < v0 + K; ++j) rank += ws.cyc_key[j] < key;
        ws.cyc_rank[i] = rank;
        const unsigned long long packed =
            ((unsigned long long)(unsigned)rank << 32) | (unsigned)(INT_MAX - ws.cyc_root[i]);
        atomicMax(s_best, packed);
    }
    __syncthreads();
    // ---- materialise the records the sweep gathers (with dirty != nullptr,
    //      marking those that change: the next sweep looks only at vertices
    //      with a changed target)
    if (dirty) {
        for (int i = threadIdx.x; i < (n + 31) / 32; i += W) dirty[i] = 0u;
        __syncthreads();
    }
    int changed = 0;
    for (int v = v0 + (int)threadIdx.x; v < v1; v += W) {
        const JLS st = A[v];
        const int i = ws.cid_of_root[~st.J];
        const long long p = ws.cyc_p[i];
        const int q = ws.cyc_q[i];
        Rec rec;
        rec.V = (long long)q * st.S - p * (long long)st.len;
        rec.rank = ws.cyc_rank[i];
        rec.q = q;
        if (dirty) {
            const Rec old = ws.rec[v];
            if (old.V != rec.V || old.rank != rec.rank || old.q != rec.q) {
                atomicOr(&dirty[(v - v0) >> 5], 1u << ((v - v0) & 31));
                ++changed;
            }
        }
        ws.rec[v] = rec;
    }
    if (dirty) *n_dirty = block_sum(changed, s_red);   // (its barriers end the pass)
    else __syncthreads();
    return true;
}

// Switch decision of vertex v given the best candidate and the candidate of
// its current policy edge (strict improvement, Alg. 1).
static __device__ __forceinline__ int small_switch(int v, const Cand &best,
                                                   const Cand &own, const int *__restrict__ col,
                                                   const int *__restrict__ w, int sign,
                                                   const Workspace &ws) {
    if (own.e == INT_MAX) {
        atomicOr(&ws.ctrl->err, kErrSweep);
        return 0;
    }
    if (best.rank > own.rank || (best.rank == own.rank && best.key > own.key)) {
        ws.pi[v] = best.e;
        ws.succ[v] = col[best.e];
        ws.wpi[v] = sign * w[best.e];
        return 1;
    }
    return 0;
}

static __device__ __forceinline__ Cand small_cand(const int *__restrict__ col,
                                                  const int *__restrict__ w, int sign,
                                                  const Workspace &ws, int e) {
    const Rec r = ws.rec[col[e]];
    return Cand{r.rank, e, (long long)r.q * (long long)(sign * w[e]) + r.V};
}

// One improvement sweep of graph [v0, v1) (the candidate order of
// improve_kernel): a thread per vertex of out-degree <= 32, a warp per vertex
// with more (lanes stride its edges, shuffles combine); returns the number of
// switches.
static __device__ __forceinline__ bool target_changed(const unsigned *dirty, int v0, int t) {
    return (dirty[(t - v0) >> 5] >> ((t - v0) & 31)) & 1u;
}

// dirty != nullptr: the frontier form -- a vertex none of whose targets'
// records changed in the last evaluation would choose as in the last sweep,
// and is skipped.
static __device__ int small_sweep(int v0, int v1, const int *__restrict__ row_ptr,
                                  const int *__restrict__ col, const int *__restrict__ w,
                                  int sign, const Workspace &ws, int *s_red,
                                  const unsigned *dirty) {
    int sw = 0;
    bool heavy_seen = false;
    for (int v = v0 + (int)threadIdx.x; v < v1; v += blockDim.x) {
        const int a = row_ptr[v], b = row_ptr[v + 1];
        if (b - a > 32) {
            heavy_seen = true;
            continue;
        }
        if (dirty) {
            bool any = false;
            for (int e = a; e < b && !any; ++e) any = target_changed(dirty, v0, col[e]);
            if (!any) continue;
        }
        const int pv = ws.pi[v];
        Cand best{INT_MIN, INT_MAX, LLONG_MIN};
        Cand own{INT_MIN, INT_MAX, LLONG_MIN};
        for (int e = a; e < b; ++e) {
            const Cand x = small_cand(col, w, sign, ws, e);
            if (e == pv) own = x;
            if (better(x, best)) best = x;
        }
        sw += small_switch(v, best, own, col, w, sign, ws);
    }
    if (__syncthreads_or(heavy_seen)) {
        const int lane = threadIdx.x & 31;
        const int nw = blockDim.x >> 5;
        for (int v = v0 + (int)(threadIdx.x >> 5); v < v1; v += nw) {
            const int a = row_ptr[v], b = row_ptr[v + 1];
            if (b - a <= 32) continue;   // the same decision in every lane
            if (dirty) {
                bool any = false;
                for (int e = a + lane; e < b && !any; e += 32)
                    any = target_changed(dirty, v0, col[e]);
                if (!__any_sync(0xffffffffu, any)) continue;
            }
            const int pv = ws.pi[v];
            Cand best{INT_MIN, INT_MAX, LLONG_MIN};
            Cand own{INT_MIN, INT_MAX, LLONG_MIN};
            for (int e = a + lane; e < b; e += 32) {
                const Cand x = small_cand(col, w, sign, ws, e);
                if (e == pv) own = x;
                if (better(x, best)) best = x;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                Cand y;
                y.rank = __shfl_xor_sync(0xffffffffu, best.rank, o);
                y.e = __shfl_xor_sync(0xffffffffu, best.e, o);
                y.key = __shfl_xor_sync(0xffffffffu, best.key, o);
                if (better(y, best)) best = y;
                Cand z;
                z.rank = __shfl_xor_sync(0xffffffffu, own.rank, o);
                z.e = __shfl_xor_sync(0xffffffffu, own.e, o);
                z.key = __shfl_xor_sync(0xffffffffu, own.key, o);
                if (z.e != INT_MAX) own = z;   // one lane met the policy edge
            }
            if (lane == 0) sw += small_switch(v, best, own, col, w, sign, ws);
        }
    }
    return block_sum(sw, s_red);
}

__global__ void __launch_bounds__(kSmallThreads, 1)
small_graph_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col,
                   const int *__restrict__ w, int sign, const int *__restrict__ queue,
                   long long max_iters, int nwords, Workspace ws, BatchState bs) {
    extern __shared__ unsigned s_bits[];
    __shared__ int s_red[kSmallThreads / 32];
    __shared__ int s_task, s_k, s_stop;
    __shared__ unsigned long long s_best;
    Ctrl *c = ws.ctrl;
    const int total = c->small_total;
    for (;;) {
        if (threadIdx.x == 0) s_task = atomicAdd(&c->small_head, 1);
        __syncthreads();
        const int qi = s_task;
        __syncthreads();
        if (qi >= total) break;
        const int g = queue[qi];
        const int v0 = bs.vptr[g], v1 = bs.vptr[g + 1];
        long long it = 0;
        bool ok = true;
        // the frontier form: once the last sweep switched fewer than n/8
        // vertices, the record pass marks the records it changes (a bitmap in
        // shared memory after the leaf bitmaps, when both fit), and the sweep
        // looks only at vertices with a changed target when fewer than n/4
        // changed
        const int ng = v1 - v0;
        unsigned *dirty_bits = 4 * ((ng + 31) / 32) <= nwords ? s_bits + 3 * ((ng + 31) / 32)
                                                              : nullptr;
        int last_sw = ng;
        for (;;) {
            unsigned *mark = (dirty_bits && it > 0 && last_sw < (ng >> 3)) ? dirty_bits : nullptr;
            int n_dirty = ng;
            if (!small_evaluate(v0, v1, ws, s_red, &s_k, &s_best, s_bits, nwords, mark,
                                &n_dirty)) {
                ok = false;
                break;
            }
            const int sw = small_sweep(v0, v1, row_ptr, col, w, sign, ws, s_red,
                                       (mark && n_dirty < (ng >> 2)) ? mark : nullptr);
            last_sw = sw;
            if (sw == 0) break;
            if (++it >= max_iters) {
                if (threadIdx.x == 0) c->not_converged = 1;
                ok = false;
                break;
            }
        }
        if (threadIdx.x == 0) {
            if (ok) {
                const unsigned long long packed = s_best;
                const int root = INT_MAX - (int)(unsigned)(packed & 0xffffffffu);
                const int i = ws.cid_of_root[root];
                bs.gbest[g] = packed;
                bs.groot[g] = root;
                bs.glen[g] = ws.cyc_L[i];
                bs.gp[g] = ws.cyc_p[i];
                bs.gq[g] = ws.cyc_q[i];
                bs.gconv[g] = 1;
                atomicMax(&c->small_iters, (int)it);
            }
        }
        // an error anywhere fails the whole call: stop (the same decision in
        // every thread of the block)
        if (threadIdx.x == 0) s_stop = (load_volatile(&c->err) != 0) || load_volatile(&c->not_converged);
        __syncthreads();
        if (s_stop) break;
    }
}

// Builds the queue of graphs with at most max_n vertices (and at most 16 max_n
// edges) and solves them, one block per graph at a time; returns the number
// of kernel launches, or -1.  max_n == 0 picks the size limit from the batch:
// a graph goes to a block of its own unless it holds more than four times the
// batch's vertices per resident block (a few huge graphs are faster on the
// whole grid, the rest of the batch is not worth a launch per iteration), and
// never below kBatchSmallDefault.
int launch_batch_small(const int *row_ptr, const int *col, const int *w, int sign, int max_n,
                       long long N, long long max_iters, int *queue, Workspace ws, BatchState bs,
                       cudaStream_t st) {
    static int cached_dev = -1, cached_blocks = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (dev != cached_dev) {
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return -1;
        if (cudaFuncSetAttribute(small_graph_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmallBitmapWords * 4) != cudaSuccess)
            return -1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, small_graph_kernel,
                                                          kSmallThreads,
                                                          kSmallBitmapWords * 4) != cudaSuccess ||
            per_sm < 1)
            return -1;
        cached_blocks = sms * per_sm;
        cached_dev = dev;
    }
    if (max_n == 0) {
        const long long auto_n = 4 * N / cached_blocks;
        max_n = (int)(auto_n > INT_MAX / 16 ? INT_MAX / 16
                                            : (auto_n < kBatchSmallDefault ? kBatchSmallDefault
                                                                           : auto_n));
    }
    int gb = (bs.G + kThreads - 1) / kThreads;
    if (gb > 1024) gb = 1024;
    prof_begin(kProfEvaluate, st);
    small_count_kernel<<<gb, kThreads, 0, st>>>(row_ptr, bs, max_n, ws.ctrl);
    small_fill_kernel<<<gb, kThreads, 0, st>>>(row_ptr, bs, max_n, ws.ctrl, queue);
    small_graph_kernel<<<cached_blocks, kSmallThreads, kSmallBitmapWords * 4, st>>>(
        row_ptr, col, w, sign, queue, max_iters, kSmallBitmapWords, ws, bs);
    prof_end(kProfEvaluate, st);
    return cudaGetLastError() == cudaSuccess ? 3 : -1;
}

}  // namespace ocm
