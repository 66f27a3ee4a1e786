// sweep.cu -- the improvement sweep of Howard's algorithm (Alg. 1, the pass
// over all vertices; Alg. 2 SPFPassIter) and the initial policy.
//
// For every vertex v and every out-edge e = (v, t) the sweep forms the key
//     (rank(t), q_t * s*w(e) + V(t))
// where rank(t) orders the mean eta(t) of the policy cycle t reaches, q_t is
// that mean's denominator and V(t) the value of t scaled by q_t.  Within one
// rank all targets share (p, q), so comparing q*w + V is comparing the
// improvement key q*w - p + V of multichain policy iteration.  The best edge
// is the lexicographic maximum of (rank, key, -e); v switches to it only on a
// strict improvement over its current policy edge (Alg. 1: strict ">"), so
// ties keep the incumbent and the iteration terminates.
//
// Layout: vertices are grouped once per solve by degree class; a vertex of
// class c is served by a group of 2^c lanes that stride over its edges with
// coalesced loads, gather each target's 16-byte record (V, rank, q), and
// reduce by warp shuffles -- no shared memory and no block barriers, so the
// warps of an SM keep many independent loads in flight.  A vertex with more
// than kHeavyEdges out-edges takes the heavy path instead (chunks of its
// edges, one block each, combined per vertex).  The initial policy (no
// records yet) runs in the same lane groups and also validates the input,
// with the same heavy path for heavy vertices.
#include "common.cuh"

namespace ocm {

// Lexicographic best (rank, key, -edge) over the 32 lanes of a warp.
static __device__ __forceinline__ Cand warp_best(Cand b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Cand other;
        other.rank = __shfl_xor_sync(0xffffffffu, b.rank, o);
        other.e = __shfl_xor_sync(0xffffffffu, b.e, o);
        other.key = __shfl_xor_sync(0xffffffffu, b.key, o);
        if (better(other, b)) b = other;
    }
    return b;
}

// Best candidate of heavy vertex i over its chunks' partial results, by the
// whole block (kHeavyThreads threads); the result is valid in thread 0.
static __device__ __forceinline__ Cand heavy_combine(const Workspace &ws, int i, Cand *s_w) {
    const int a = ws.heavy_off[i], b = ws.heavy_off[i + 1];
    Cand best{INT_MIN, INT_MAX, LLONG_MIN};
    for (int c = a / kHeavyChunk + (int)threadIdx.x; c <= (b - 1) / kHeavyChunk;
         c += blockDim.x) {
        const Cand x = ws.heavy_part[2 * c + ((long long)c * kHeavyChunk >= a ? 0 : 1)];
        if (better(x, best)) best = x;
    }
    best = warp_best(best);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x < 32) {
        Cand x = threadIdx.x < kHeavyThreads / 32 ? s_w[threadIdx.x]
                                                  : Cand{INT_MIN, INT_MAX, LLONG_MIN};
        best = warp_best(x);
    }
    __syncthreads();   // s_w is reused for the next vertex
    return best;
}

__global__ void __launch_bounds__(kThreads)
check_row_ptr_kernel(const int *__restrict__ row_ptr, int n, int m, Ctrl *ctrl) {
    int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
        int a = row_ptr[v];
        if (v == 0 && a != 0) {
            atomicOr(&ctrl->err, kErrRowPtr);
            atomicMin(&ctrl->bad_index, 0);
        }
        if (v == n) {
            if (a != m) {
                atomicOr(&ctrl->err, kErrRowPtr);
                atomicMin(&ctrl->bad_index, n);
            }
        } else {
            int b = row_ptr[v + 1];
            if (b < a || a < 0 || b > m) {
                atomicOr(&ctrl->err, kErrRowPtr);
                atomicMin(&ctrl->bad_index, v);
            } else if (b == a) {
                atomicOr(&ctrl->err, kErrNoOutEdge);
                atomicMin(&ctrl->bad_index, v);
            }
        }
    }
}

void launch_check_row_ptr(const int *row_ptr, int n, int m, Ctrl *ctrl, cudaStream_t st) {
    int blocks = (n + 1 + kThreads - 1) / kThreads;
    if (blocks > 4096) blocks = 4096;
    prof_begin(kProfInit, st);
    check_row_ptr_kernel<<<blocks, kThreads, 0, st>>>(row_ptr, n, m, ctrl);
    prof_end(kProfInit, st);
}

// With local_R > 0 the pass also counts the edges whose target lies in the
// block range (local_R consecutive vertices) of their source, the locality
// measure that chooses the two-level evaluation, and clears that
// evaluation's root stamps (heavy vertices' edges are not counted).
//
// Initial policy (Alg. 1's first pass from val = 0, lambda = 0): the heaviest
// out-edge in the s*w sense, ties to the smallest edge index (for the cycle
// ratio too: with lambda = 0 the key w(e) - lambda t(e) is w(e)) -- or, for a
// warm start, the caller's policy (init != nullptr), which must name an
// out-edge of each vertex.  The same pass validates col_idx, w and the
// transit times and measures max|w| and max t for the exactness bound.
//
// Layout: the lane groups and band-major task order of the degree-class
// sweep (improve_kernel below), so the edge loads are coalesced.
__global__ void __launch_bounds__(kSweepMaxThreads, 3)
init_policy_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col,
                   const int *__restrict__ w, int sign, int n, const int *__restrict__ gid,
                   const int *__restrict__ init, int local_R, int count_win, int groups,
                   Workspace ws) {
    constexpr int kWarps = kSweepMaxThreads / 32;
    __shared__ int s_maxw[kWarps];
    __shared__ int s_maxt[kWarps];
    __shared__ unsigned long long s_local[kWarps];
    __shared__ unsigned s_win[kWarps][kWinShapes];
    unsigned long long local = 0;
    unsigned win[kWinShapes] = {};   // edges inside each window shape (window sweep)
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int stride = gridDim.x * blockDim.x;
    const int *__restrict__ tt = ws.transit;
    int maxabs = 0, maxt = 0;
    if (local_R)
        for (int v = blockIdx.x * blockDim.x + tid; v < n; v += stride) ws.root_mark[v] = 0;
    const int4 *__restrict__ grp_tab = ws.band_grp;
    const int total = grp_tab[groups].x;
    const int warps = stride >> 5;
    int p = 0;
    int4 grp = grp_tab[0];
    int next_start = groups > 1 ? grp_tab[1].x : total;
    for (int task = (blockIdx.x * blockDim.x + tid) >> 5; task < total; task += warps) {
        while (task >= next_start) {   // (the same steps in every lane)
            ++p;
            grp = grp_tab[p];
            next_start = p + 1 < groups ? grp_tab[p + 1].x : total;
        }
        const int c = grp.w;
        const int g = 1 << c;
        const int sub = lane & (g - 1);
        const int idx = (task - grp.x) * (32 >> c) + (lane >> c);
        const bool valid = idx < grp.z;
        const int v = valid ? ws.cls_list[grp.y + idx] : 0;
        Cand best{INT_MIN, INT_MAX, LLONG_MIN};
        int a = 0, b = 0;
        int tmin = INT_MAX, tmax = INT_MIN;   // this lane's targets
        if (valid) {
            a = __ldg(&row_ptr[v]);
            b = __ldg(&row_ptr[v + 1]);
            // v's block range of the two-level evaluation, as bounds
            const unsigned r_lo = local_R ? (unsigned)(v / local_R) * (unsigned)local_R : 0u;
            const unsigned r_len = (unsigned)local_R;
            const int my_g = gid ? gid[v] : 0;
            // (the lane's best as (key, edge): every key has rank 0 here, and
            // the lane meets its edges in increasing order, so a strictly larger
            // key is the only way to replace the incumbent)
            int best_k = INT_MIN, best_e = INT_MAX;
            for (int e = a + sub; e < b; e += g) {
                const int t = __ldg(&col[e]);
                int x = __ldg(&w[e]);
                if ((unsigned)t >= (unsigned)n || (gid && gid[t] != my_g)) {
                    // out of range, or (batched) an edge between different graphs
                    atomicOr(&ws.ctrl->err, kErrCol);
                    atomicMin(&ws.ctrl->bad_index, e);
                }
                if (x == INT_MIN) {
                    atomicOr(&ws.ctrl->err, kErrWeightMin);
                    atomicMin(&ws.ctrl->bad_index, e);
                    x = 0;
                }
                maxabs = max(maxabs, x < 0 ? -x : x);
                tmin = min(tmin, t);
                tmax = max(tmax, t);
                if (local_R) local += (unsigned)t - r_lo < r_len;
                if (count_win) {
#pragma unroll
                    for (int j = 0; j < kWinShapes; ++j)
                        win[j] += (unsigned)(t - v + j * kWinTile) < (unsigned)kWinHalo;
                }
                if (tt) {
                    const int te = __ldg(&tt[e]);
                    if (te < 1) {
                        atomicOr(&ws.ctrl->err, kErrTransit);
                        atomicMin(&ws.ctrl->bad_index, e);
                    }
                    maxt = max(maxt, te);
                }
                const int k = sign * x;
                if (k > best_k || best_e == INT_MAX) {
                    best_k = k;
                    best_e = e;
                }
            }
            if (best_e != INT_MAX) best = Cand{0, best_e, (long long)best_k};
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            if (o < g) {
                Cand other;
                other.rank = __shfl_xor_sync(0xffffffffu, best.rank, o);
                other.e = __shfl_xor_sync(0xffffffffu, best.e, o);
                other.key = __shfl_xor_sync(0xffffffffu, best.key, o);
                if (better(other, best)) best = other;
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            if (o < g) {
                tmin = min(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
                tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
            }
        }
        {
            // the range of target blocks of v's block (the frontier sweep): one
            // update per warp when all its vertices lie in one block (a plain
            // read first: most updates widen nothing)
            const bool ok = valid && sub == 0 && tmin <= tmax && (unsigned)tmin < (unsigned)n &&
                            (unsigned)tmax < (unsigned)n;
            const int blk = ok ? v / kClassifyBlock : -1;
            const unsigned okm = __ballot_sync(0xffffffffu, ok);
            const int blk0 = okm ? __shfl_sync(0xffffffffu, blk, __ffs(okm) - 1) : -1;
            const bool one = __all_sync(0xffffffffu, !ok || blk == blk0);
            int lo = ok ? tmin / kDirtyBlock : INT_MAX, hi = ok ? tmax / kDirtyBlock : INT_MIN;
            if (one) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
                }
            }
            if (ok && (!one || lane == __ffs(okm) - 1)) {
                int2 *bt = &ws.blk_tgt[blk];
                const int2 cur = *bt;
                if (lo < cur.x) atomicMin(&bt->x, lo);
                if (hi > cur.y) atomicMax(&bt->y, hi);
            }
        }
        if (valid && sub == 0) {
            int be = best.e;
            if (init) {
                const int e = __ldg(&init[v]);
                if (e >= a && e < b) {
                    be = e;
                } else {
                    atomicOr(&ws.ctrl->err, kErrInitPolicy);
                    atomicMin(&ws.ctrl->bad_index, v);
                }
            }
            const int t = __ldg(&col[be]);
            const int x = __ldg(&w[be]);
            ws.pi[v] = be;
            ws.succ[v] = ((unsigned)t < (unsigned)n) ? t : 0;
            ws.wpi[v] = sign * (x == INT_MIN ? 0 : x);
            if (tt) ws.tpi[v] = __ldg(&tt[be]);
            ws.sw_iter[v] = 0;   // the first evaluation treats every vertex as changed
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        maxabs = max(maxabs, __shfl_xor_sync(0xffffffffu, maxabs, o));
        maxt = max(maxt, __shfl_xor_sync(0xffffffffu, maxt, o));
        local += __shfl_xor_sync(0xffffffffu, local, o);
#pragma unroll
        for (int j = 0; j < kWinShapes; ++j) win[j] += __shfl_xor_sync(0xffffffffu, win[j], o);
    }
    if (lane == 0) {
        s_maxw[tid >> 5] = maxabs;
        s_maxt[tid >> 5] = maxt;
        s_local[tid >> 5] = local;
#pragma unroll
        for (int j = 0; j < kWinShapes; ++j) s_win[tid >> 5][j] = win[j];
    }
    __syncthreads();
    if (tid < 32) {
        const int nw = blockDim.x >> 5;
        int x = tid < nw ? s_maxw[tid] : 0;
        int y = tid < nw ? s_maxt[tid] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
            y = max(y, __shfl_xor_sync(0xffffffffu, y, o));
        }
        if (tid == 0) {
            atomicMax(&ws.ctrl->maxabsw, x);
            if (tt) atomicMax(&ws.ctrl->maxt, y);
            if (local_R) {
                unsigned long long sum = 0;
                for (int k = 0; k < nw; ++k) sum += s_local[k];
                if (sum) atomicAdd(reinterpret_cast<unsigned long long *>(&ws.ctrl->local_edges),
                                   sum);
            }
            for (int j = 0; j < kWinShapes && count_win; ++j) {
                unsigned long long sum = 0;
                for (int k = 0; k < nw; ++k) sum += s_win[k][j];
                if (sum) atomicAdd(reinterpret_cast<unsigned long long *>(&ws.ctrl->win_edges[j]),
                                   sum);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Degree classes.  A vertex of out-degree d is served by a group of 2^c lanes,
// c the smallest class with d <= kEdgesPerLane * 2^c (capped at 32 lanes), so
// every lane handles a few edges and the lanes of a warp finish together even
// when degrees are skewed.  The partition is computed once per solve (the
// graph does not change), stable within each class, in three passes:
// per-block counts, one exclusive scan, and a scatter.

__global__ void __launch_bounds__(kClassifyBlock)
classify_count_kernel(const int *__restrict__ row_ptr, int n, int nb, int epl, Workspace ws) {
    __shared__ int s_cnt[kClassSlots];
    if (threadIdx.x < kClassSlots) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int v = blockIdx.x * kClassifyBlock + threadIdx.x;
    if (v < n) atomicAdd(&s_cnt[degree_class(__ldg(&row_ptr[v + 1]) - __ldg(&row_ptr[v]), epl)], 1);
    __syncthreads();
    if (threadIdx.x < kClassSlots) ws.cls_hist[threadIdx.x * nb + blockIdx.x] = s_cnt[threadIdx.x];
    if (threadIdx.x == 0) ws.blk_tgt[blockIdx.x] = make_int2(INT_MAX, INT_MIN);   // (initial pass)
}

// One block: exclusive scan of the class-major histogram (class c, block b at
// c * nb + b), so every (class, block) pair gets its first list position.
__global__ void __launch_bounds__(1024) classify_scan_kernel(int nb, Workspace ws) {
    // (warp w scans the contiguous piece [w * per, (w + 1) * per) in strips
    // of 32 consecutive entries: the pieces' sums first, then, offset by a
    // scan of those sums, the prefixes)
    __shared__ int s_warp[32];
    __shared__ int s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int total = kClassSlots * nb;
    const int per = ((total + nwarps - 1) / nwarps + 31) & ~31;
    const int i0 = min(total, warp * per), i1 = min(total, i0 + per);
    int sum = 0;
    for (int i = i0 + lane; i < i1; i += 32) sum += ws.cls_hist[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) s_warp[warp] = sum;
    __syncthreads();
    if (warp == 0) {
        int wv = lane < nwarps ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wv, o);
            if (lane >= o) wv += y;
        }
        s_warp[lane] = wv;   // inclusive
    }
    __syncthreads();
    int run = warp > 0 ? s_warp[warp - 1] : 0;   // the piece's offset
    for (int base = i0; base < i1; base += 32) {   // (warp-uniform trip count)
        const int i = base + lane;
        const int x = i < i1 ? ws.cls_hist[i] : 0;
        int incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (i < i1) {
            const int excl = run + incl - x;
            ws.cls_hist[i] = excl;
            if (i % nb == 0) ws.ctrl->cls_off[i / nb] = excl;
        }
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (threadIdx.x == 0) s_total = s_warp[nwarps - 1];
    __syncthreads();
    if (threadIdx.x < kClassSlots) {
        const int c = threadIdx.x;
        const int next = (c + 1 < kClassSlots) ? ws.ctrl->cls_off[c + 1] : s_total;
        ws.ctrl->cls_cnt[c] = next - ws.ctrl->cls_off[c];
    }
}

__global__ void __launch_bounds__(kClassifyBlock)
classify_scatter_kernel(const int *__restrict__ row_ptr, int n, int nb, int epl, Workspace ws) {
    __shared__ int s_wcnt[kClassifyBlock / 32][kClassSlots];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int v = blockIdx.x * kClassifyBlock + threadIdx.x;
    const int c = (v < n) ? degree_class(__ldg(&row_ptr[v + 1]) - __ldg(&row_ptr[v]), epl) : -1;
    int my_rank = 0;
#pragma unroll
    for (int k = 0; k < kClassSlots; ++k) {
        const unsigned m = __ballot_sync(0xffffffffu, c == k);
        if (c == k) my_rank = __popc(m & ((1u << lane) - 1u));
        if (lane == 0) s_wcnt[warp][k] = __popc(m);
    }
    __syncthreads();
    if (c >= 0) {
        int before = 0;
        for (int q = 0; q < warp; ++q) before += s_wcnt[q][c];
        ws.cls_list[ws.cls_hist[c * nb + blockIdx.x] + before + my_rank] = v;
    }
}

// One block: the heavy vertices (the last class, in increasing vertex order)
// get their offsets in the heavy edge sequence, an exclusive scan of their
// out-degrees; the total goes to the control block.
__global__ void __launch_bounds__(1024) heavy_prep_kernel(const int *__restrict__ row_ptr,
                                                          Workspace ws) {
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    const int H = ws.ctrl->cls_cnt[kClasses];
    const int *hv = ws.cls_list + ws.ctrl->cls_off[kClasses];
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < H; base += 1024) {
        const int i = base + threadIdx.x;
        const int x = i < H ? __ldg(&row_ptr[hv[i] + 1]) - __ldg(&row_ptr[hv[i]]) : 0;
        int incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((threadIdx.x & 31) >= o) incl += y;
        }
        if ((threadIdx.x & 31) == 31) s_warp[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x < 32) {
            int wv = s_warp[threadIdx.x];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wv, o);
                if (threadIdx.x >= o) wv += y;
            }
            s_warp[threadIdx.x] = wv;
        }
        __syncthreads();
        const int warp_prefix = (threadIdx.x >= 32) ? s_warp[(threadIdx.x >> 5) - 1] : 0;
        if (i < H) ws.heavy_off[i] = s_carry + warp_prefix + incl - x;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry += warp_prefix + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ws.heavy_off[H] = s_carry;
        ws.ctrl->heavy_edges = s_carry;
    }
}

// One block: the sweep's (band, class) task groups in band-major order.  The
// class-c vertices of band b are the class-list entries from block b * B of
// the classification (B classification blocks a band) up to block
// (b + 1) * B (the class list is in vertex order within a class); a group of
// k entries takes ceil(k * 2^c / 32) warp tasks.
__global__ void __launch_bounds__(1024) band_tasks_kernel(int n, int nb, int B, Workspace ws) {
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    const int groups = sweep_groups(n, B);
    const Ctrl *c = ws.ctrl;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < groups; base += 1024) {
        const int i = base + threadIdx.x;
        int4 grp = make_int4(0, 0, 0, 0);
        int x = 0;
        if (i < groups) {
            const int b = i / kClasses, q = i % kClasses;
            const int first = ws.cls_hist[q * nb + b * B];
            const int last = (b + 1) * B < nb ? ws.cls_hist[q * nb + (b + 1) * B]
                                               : c->cls_off[q] + c->cls_cnt[q];
            grp = make_int4(0, first, last - first, q);
            x = (int)((((long long)(last - first) << q) + 31) >> 5);
        }
        int incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((threadIdx.x & 31) >= o) incl += y;
        }
        if ((threadIdx.x & 31) == 31) s_warp[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x < 32) {
            int wv = s_warp[threadIdx.x];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wv, o);
                if (threadIdx.x >= o) wv += y;
            }
            s_warp[threadIdx.x] = wv;
        }
        __syncthreads();
        const int warp_prefix = (threadIdx.x >= 32) ? s_warp[(threadIdx.x >> 5) - 1] : 0;
        if (i < groups) {
            grp.x = s_carry + warp_prefix + incl - x;
            ws.band_grp[i] = grp;
        }
        __syncthreads();
        if (threadIdx.x == 1023) s_carry += warp_prefix + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) ws.band_grp[groups] = make_int4(s_carry, 0, 0, 0);
}

int launch_classify(const int *row_ptr, int n, int epl, int band_blocks, Workspace ws,
                    cudaStream_t st) {
    const int nb = (n + kClassifyBlock - 1) / kClassifyBlock;
    prof_begin(kProfInit, st);
    classify_count_kernel<<<nb, kClassifyBlock, 0, st>>>(row_ptr, n, nb, epl, ws);
    classify_scan_kernel<<<1, 1024, 0, st>>>(nb, ws);
    classify_scatter_kernel<<<nb, kClassifyBlock, 0, st>>>(row_ptr, n, nb, epl, ws);
    heavy_prep_kernel<<<1, 1024, 0, st>>>(row_ptr, ws);
    band_tasks_kernel<<<1, 1024, 0, st>>>(n, nb, band_blocks, ws);
    prof_end(kProfInit, st);
    return 5;
}

// ---------------------------------------------------------------------------
// Improvement sweep.  Work is cut into warp tasks: a task of class c covers
// 32 / 2^c consecutive entries of the class list, one lane group per vertex.
// The lanes of a group stride over the vertex's edges (coalesced), gather the
// 16-byte record of every target, keep the lexicographic best (rank, key,
// -edge), and combine by shuffles inside the group.  The current policy edge
// is one of the vertex's edges, so the lane that meets it keeps its candidate
// (no second gather for the record of succ(v)); after the butterfly every lane
// holds the best, and that lane switches only on strict improvement in
// (rank, key).  A persistent grid walks the tasks band by band (all classes
// of a band of kSweepBand vertices, then the next band: the band's records
// are gathered from L2 in every class pass, not again from HBM); each warp
// keeps a cursor on the (band, class) groups, which its grid-stride steps
// advance by a few groups at most (BANDED; a graph that is one band takes
// its class of a task from the launch's per-class task offsets instead).
// Switches are counted in registers and published with one atomic per block
// (same-address atomics per warp would serialise the whole sweep).
struct ClassGrid {
    int task_off[kClasses + 1];  // first warp task of each class; [kClasses] = total
    int band_blocks;             // classification blocks per band of the task order
};

// Candidate of edge e.  Cycle ratio (RATIO): the key also subtracts
// p_t * t(e), the target's ratio numerator times the edge's transit time;
// for the mean t(e) = 1 and p_t is the same for every target of equal rank,
// so the term is dropped.
template <bool RATIO>
static __device__ __forceinline__ Cand edge_cand(const int *__restrict__ col,
                                                 const int *__restrict__ w, const int4 *rec,
                                                 const Workspace &ws, int sign, int e) {
    const int t = __ldg(&col[e]);
    const int x = __ldg(&w[e]);
    const int4 r = __ldg(&rec[t]);
    const long long V = ((long long)(unsigned)r.x) | ((long long)r.y << 32);
    long long key = (long long)r.w * (long long)(sign * x) + V;
    if (RATIO) key -= __ldg(&ws.recp[t]) * (long long)__ldg(&ws.transit[e]);
    return Cand{r.z, e, key};
}

// Whether some block of band b (of B classification blocks) has edges that
// reach a block with a changed record.
static __device__ __forceinline__ bool band_reaches_change(const Workspace &ws, int b, int B,
                                                           int n) {
    const int nbk = (n + kClassifyBlock - 1) / kClassifyBlock;
    const int b0 = b * B, b1 = min(b0 + B, nbk) - 1;
    for (int wd = b0 >> 5; wd <= (b1 >> 5); ++wd) {
        unsigned bits = ws.need_blk[wd];
        if (wd == (b0 >> 5)) bits &= ~0u << (b0 & 31);
        if (wd == (b1 >> 5)) bits &= ~0u >> (31 - (b1 & 31));
        if (bits) return true;
    }
    return false;
}

// FRONTIER: the instance for the frontier form; both instances are launched
// every step and the one whose form the control block does not ask for
// returns at once (the choice is made on the device, inside the loop graph).
template <bool RATIO, bool BANDED, bool FRONTIER>
__global__ void __launch_bounds__(kSweepMaxThreads, 3)   // 40 registers: 48 warps per SM
improve_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col,
               const int *__restrict__ w, int sign, int n_vertices, int groups, ClassGrid cg,
               Workspace ws, BatchState bs) {
    // the frontier form: the record pass marked the records it changed, and
    // few changed (or the test flag asks for it)
    const bool frontier =
        ws.ctrl->dirty_on &&
        (ws.ctrl->frontier == 2 || ws.ctrl->dirty_cnt < ((long long)n_vertices >> kFrontierDirtyShift));
    if (frontier != FRONTIER) return;
    __shared__ int s_sw;
    const int tid = threadIdx.x;
    // a vertex switched here is "dirty" for the next evaluation
    const int next_eval = ws.ctrl->iter + 1;
    const int lane = tid & 31;
    if (tid == 0) s_sw = 0;
    if (blockIdx.x == 0 && tid == 0) publish_result(ws, n_vertices);
    __syncthreads();
    const int4 *rec = reinterpret_cast<const int4 *>(ws.rec);
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int4 *__restrict__ grp_tab = ws.band_grp;
    const int total = BANDED ? grp_tab[groups].x : cg.task_off[kClasses];
    int switched = 0;
    int need_b = -1;    // (FRONTIER) the band band_need describes
    const int gw = (blockIdx.x * blockDim.x + tid) >> 5;
    bool band_need = true;
    int p = 0;          // the group holding the current task: grp_tab[p].x <= task
    int4 grp = BANDED ? grp_tab[0] : make_int4(0, 0, 0, 0);
    int next_start = (BANDED && groups > 1) ? grp_tab[1].x : total;
    for (int task = gw; task < total; task += warps) {
        int c, first_task, list0, cnt;
        if (BANDED) {
            while (task >= next_start) {   // (the same steps in every lane)
                ++p;
                grp = grp_tab[p];
                next_start = p + 1 < groups ? grp_tab[p + 1].x : total;
            }
            if (FRONTIER) {
                // a band none of whose blocks reaches a changed record: the
                // warp jumps to its first task in the next band that has one
                // (no vertex loaded, no cursor step per group in between)
                const int b = p / kClasses;
                if (b != need_b) {
                    need_b = b;
                    band_need = band_reaches_change(ws, b, cg.band_blocks, n_vertices);
                }
                if (!band_need) {
                    const int bands = groups / kClasses;
                    int b2 = b + 1;
                    while (b2 < bands && !band_reaches_change(ws, b2, cg.band_blocks, n_vertices))
                        ++b2;
                    if (b2 >= bands) break;   // (the same decision in every lane)
                    const int ts = grp_tab[b2 * kClasses].x;
                    p = b2 * kClasses;
                    grp = grp_tab[p];
                    next_start = p + 1 < groups ? grp_tab[p + 1].x : total;
                    need_b = b2;
                    band_need = true;
                    task = ts + (((gw - ts) % warps) + warps) % warps - warps;   // (+ warps below)
                    continue;
                }
            }
            c = grp.w;
            first_task = grp.x;
            list0 = grp.y;
            cnt = grp.z;
        } else {
            c = 0;
#pragma unroll
            for (int k = 1; k < kClasses; ++k)
                if (task >= cg.task_off[k]) c = k;
            first_task = cg.task_off[c];
            list0 = ws.ctrl->cls_off[c];
            cnt = ws.ctrl->cls_cnt[c];
        }
        const int g = 1 << c;
        const int sub = lane & (g - 1);
        const int idx = (task - first_task) * (32 >> c) + (lane >> c);
        bool valid = idx < cnt;
        const int v = valid ? ws.cls_list[list0 + idx] : 0;
        // batched: a graph whose last sweep switched nothing never switches
        // again (its records do not change), so its vertices are skipped
        if (valid && bs.G && bs.gconv[bs.gid[v]]) valid = false;
        if (FRONTIER) {
            // a vertex none of whose targets' records changed since the last
            // sweep chooses as it did then: skipped
            // (four edges of the lane at a time, their loads independent)
            bool any = false;
            if (valid) {
                // no changed block within reach of v's block's edges: skipped
                const int blk = v / kClassifyBlock;
                if (!((ws.need_blk[blk >> 5] >> (blk & 31)) & 1u)) valid = false;
            }
            if (valid) {
                const int e_end = __ldg(&row_ptr[v + 1]);
                for (int e = __ldg(&row_ptr[v]) + sub; e < e_end && !any; e += 4 * g) {
                    int t[4];
                    unsigned bw[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) t[u] = e + u * g < e_end ? __ldg(&col[e + u * g]) : -1;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        bw[u] = t[u] >= 0 ? ws.rec_dirty_blk[(t[u] / kDirtyBlock) >> 5] : 0u;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int blk = t[u] / kDirtyBlock;
                        if (t[u] >= 0 && ((bw[u] >> (blk & 31)) & 1u))
                            any |= ((ws.rec_dirty[t[u] >> 5] >> (t[u] & 31)) & 1u) != 0;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1)
                if (o < g) any |= __shfl_xor_sync(0xffffffffu, any, o) != 0;
            valid = valid && any;
        }
        if (!__any_sync(0xffffffffu, valid)) continue;   // (a whole task skipped)
        Cand best{INT_MIN, INT_MAX, LLONG_MIN};
        Cand own{INT_MIN, INT_MAX, LLONG_MIN};   // the current policy edge, in one lane
        if (valid) {
            const int a = __ldg(&row_ptr[v]), e_end = __ldg(&row_ptr[v + 1]);
            const int pv = ws.pi[v];
            int e = a + sub;
            for (; e + g < e_end; e += 2 * g) {   // two independent gathers in flight
                Cand x0 = edge_cand<RATIO>(col, w, rec, ws, sign, e);
                Cand x1 = edge_cand<RATIO>(col, w, rec, ws, sign, e + g);
                if (e == pv) own = x0;
                if (e + g == pv) own = x1;
                if (better(x0, best)) best = x0;
                if (better(x1, best)) best = x1;
            }
            if (e < e_end) {
                Cand x0 = edge_cand<RATIO>(col, w, rec, ws, sign, e);
                if (e == pv) own = x0;
                if (better(x0, best)) best = x0;
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            if (o < g) {
                Cand other;
                other.rank = __shfl_xor_sync(0xffffffffu, best.rank, o);
                other.e = __shfl_xor_sync(0xffffffffu, best.e, o);
                other.key = __shfl_xor_sync(0xffffffffu, best.key, o);
                if (better(other, best)) best = other;
            }
        }
        // own.e == INT_MAX except in the lane that met the policy edge
        if (valid && own.e != INT_MAX) {
            if (best.rank > own.rank || (best.rank == own.rank && best.key > own.key)) {
                ws.pi[v] = best.e;
                ws.succ[v] = __ldg(&col[best.e]);
                ws.wpi[v] = sign * __ldg(&w[best.e]);
                if (RATIO) ws.tpi[v] = __ldg(&ws.transit[best.e]);
                ws.sw_iter[v] = next_eval;
                if (bs.G) {
                    const int g = bs.gid[v];
                    if (bs.gsw[g] != next_eval) bs.gsw[g] = next_eval;
                }
                ++switched;
            }
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

// The initial pass for heavy vertices (after the classes are known): each
// chunk of the heavy edge sequence validates its edges as init_policy_kernel
// does and keeps the heaviest edge (ties: smallest index) of each heavy vertex
// it meets; one block per heavy vertex combines its chunks.  Grid-stride over
// the chunk and vertex counts in the control block (nothing to do without
// heavy vertices).
__global__ void __launch_bounds__(kHeavyThreads)
heavy_init_chunk_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col,
                        const int *__restrict__ w, int sign, int n, const int *__restrict__ gid,
                        Workspace ws) {
    __shared__ Cand s_b[2][kHeavyThreads / 32];
    __shared__ int s_max[2];
    const int H = ws.ctrl->cls_cnt[kClasses];
    const int *hv = ws.cls_list + ws.ctrl->cls_off[kClasses];
    const int total = ws.ctrl->heavy_edges;
    const int nchunks = (total + kHeavyChunk - 1) / kHeavyChunk;
    const int *__restrict__ tt = ws.transit;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Cand none{INT_MIN, INT_MAX, LLONG_MIN};
    if (threadIdx.x == 0) {
        s_max[0] = 0;
        s_max[1] = 0;
    }
    int maxabs = 0, maxt = 0;
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int g0 = c * kHeavyChunk, g1 = min(g0 + kHeavyChunk, total);
        int lo = 0, hi = H;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (ws.heavy_off[mid] <= g0) lo = mid; else hi = mid;
        }
        const int split = min(ws.heavy_off[lo + 1], g1);
        const int v0 = hv[lo], v1 = split < g1 ? hv[lo + 1] : v0;
        const int base0 = __ldg(&row_ptr[v0]) - ws.heavy_off[lo];
        const int base1 = split < g1 ? __ldg(&row_ptr[v1]) - ws.heavy_off[lo + 1] : 0;
        Cand b0 = none, b1 = none;
        for (int g = g0 + (int)threadIdx.x; g < g1; g += blockDim.x) {
            const bool first = g < split;
            const int e = (first ? base0 : base1) + g;
            const int t = __ldg(&col[e]);
            int x = __ldg(&w[e]);
            if ((unsigned)t >= (unsigned)n || (gid && gid[t] != gid[first ? v0 : v1])) {
                atomicOr(&ws.ctrl->err, kErrCol);
                atomicMin(&ws.ctrl->bad_index, e);
            }
            if (x == INT_MIN) {
                atomicOr(&ws.ctrl->err, kErrWeightMin);
                atomicMin(&ws.ctrl->bad_index, e);
                x = 0;
            }
            maxabs = max(maxabs, x < 0 ? -x : x);
            if (tt) {
                const int te = __ldg(&tt[e]);
                if (te < 1) {
                    atomicOr(&ws.ctrl->err, kErrTransit);
                    atomicMin(&ws.ctrl->bad_index, e);
                }
                maxt = max(maxt, te);
            }
            const Cand cand{0, e, (long long)sign * x};
            if (first) {
                if (better(cand, b0)) b0 = cand;
            } else if (better(cand, b1)) {
                b1 = cand;
            }
        }
        b0 = warp_best(b0);
        b1 = warp_best(b1);
        if (lane == 0) {
            s_b[0][warp] = b0;
            s_b[1][warp] = b1;
        }
        __syncthreads();
        if (warp == 0) {
            Cand x0 = lane < kHeavyThreads / 32 ? s_b[0][lane] : none;
            Cand x1 = lane < kHeavyThreads / 32 ? s_b[1][lane] : none;
            x0 = warp_best(x0);
            x1 = warp_best(x1);
            if (lane == 0) {
                ws.heavy_part[2 * c] = x0;
                ws.heavy_part[2 * c + 1] = x1;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        maxabs = max(maxabs, __shfl_xor_sync(0xffffffffu, maxabs, o));
        maxt = max(maxt, __shfl_xor_sync(0xffffffffu, maxt, o));
    }
    if (lane == 0) {
        if (maxabs) atomicMax(&s_max[0], maxabs);
        if (maxt) atomicMax(&s_max[1], maxt);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_max[0]) atomicMax(&ws.ctrl->maxabsw, s_max[0]);
        if (s_max[1]) atomicMax(&ws.ctrl->maxt, s_max[1]);
    }
}

__global__ void __launch_bounds__(kHeavyThreads)
heavy_init_final_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col,
                        const int *__restrict__ w, int sign, int n,
                        const int *__restrict__ init, Workspace ws) {
    __shared__ Cand s_w[kHeavyThreads / 32];
    const int H = ws.ctrl->cls_cnt[kClasses];
    const int *hv = ws.cls_list + ws.ctrl->cls_off[kClasses];
    for (int i = blockIdx.x; i < H; i += gridDim.x) {   // one block per heavy vertex
        const int v = hv[i];
        const Cand best = heavy_combine(ws, i, s_w);
        if (threadIdx.x == 0) {
            int e = best.e;
            if (init) {
                const int ei = __ldg(&init[v]);
                const int ra = __ldg(&row_ptr[v]), rb = __ldg(&row_ptr[v + 1]);
                if (ei >= ra && ei < rb) {
                    e = ei;
                } else {
                    atomicOr(&ws.ctrl->err, kErrInitPolicy);
                    atomicMin(&ws.ctrl->bad_index, v);
                }
            }
            const int t = __ldg(&col[e]);
            const int x = __ldg(&w[e]);
            ws.pi[v] = e;
            ws.succ[v] = ((unsigned)t < (unsigned)n) ? t : 0;
            ws.wpi[v] = sign * (x == INT_MIN ? 0 : x);
            if (ws.transit) ws.tpi[v] = __ldg(&ws.transit[e]);
            ws.sw_iter[v] = 0;
        }
    }
}

// Co-resident blocks of the initial pass on the current device.
static int init_grid() {
    static int cached_dev = -1, cached = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev != cached_dev) {
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, init_policy_kernel,
                                                          kSweepMaxThreads, 0) != cudaSuccess)
            return 0;
        cached_dev = dev;
        cached = sms * per_sm;
    }
    return cached;
}

void launch_init_policy(const int *row_ptr, const int *col, const int *w, int sign, int n, int m,
                        const int *init, Workspace ws, const BatchState *bs, cudaStream_t st,
                        int local_R, int count_win, int band_blocks) {
    // one wave of co-resident blocks (the tasks are taken grid-stride)
    int blocks = (n + kSweepMaxThreads - 1) / kSweepMaxThreads;
    const int resident = init_grid();
    if (resident > 0 && blocks > resident) blocks = resident;
    if (blocks > 1024) blocks = 1024;
    const int groups = sweep_groups(n, band_blocks);
    prof_begin(kProfInit, st);
    init_policy_kernel<<<blocks, kSweepMaxThreads, 0, st>>>(row_ptr, col, w, sign, n,
                                                            bs ? bs->gid : nullptr, init, local_R,
                                                            count_win, groups, ws);
    // heavy vertices (their count is on the device: fixed grids, grid-stride)
    int cb = (m / kHeavyChunk) + 1;
    if (cb > 1024) cb = 1024;
    int fb = (m / kHeavyEdges) + 1;
    if (fb > 1024) fb = 1024;
    heavy_init_chunk_kernel<<<cb, kHeavyThreads, 0, st>>>(row_ptr, col, w, sign, n,
                                                         bs ? bs->gid : nullptr, ws);
    heavy_init_final_kernel<<<fb, kHeavyThreads, 0, st>>>(row_ptr, col, w, sign, n, init, ws);
    prof_end(kProfInit, st);
}

// Co-resident blocks of the degree-class sweep per block size on the current
// device (host-side configuration, done before any launch is captured).
template <bool RATIO>
static int classes_grid(int threads) {
    static int cached_dev[3] = {-1, -1, -1}, cached_blocks[3] = {0, 0, 0};
    const int slot = threads == 128 ? 0 : threads == 256 ? 1 : 2;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cached_dev[slot] != dev) {
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, improve_kernel<RATIO, true, true>, threads,
                                                          0) != cudaSuccess ||
            sms <= 0 || per_sm <= 0)
            return 0;
        cached_blocks[slot] = sms * per_sm;
        cached_dev[slot] = dev;
    }
    return cached_blocks[slot];
}

int prepare_sweep_classes(int threads, bool ratio) {
    if (threads != 128 && threads != 256 && threads != 512) threads = kSweepThreads;
    return (ratio ? classes_grid<true>(threads) : classes_grid<false>(threads)) > 0 ? 0 : -1;
}

// ---------------------------------------------------------------------------
// Heavy vertices (more than kHeavyEdges out-edges).  Their edges, in the
// order of the heavy vertices and within each in CSR order, form one sequence
// of heavy_edges entries; chunk c holds entries [c * kHeavyChunk, ...).  One
// block per chunk finds the best candidate of each heavy vertex the chunk
// meets (at most two: the vertex holding its first entry, slot 0, and the
// next one, slot 1), and one block per heavy vertex combines its chunks and
// takes the switch decision exactly as the lane-group sweep does.

template <bool RATIO>
__global__ void __launch_bounds__(kHeavyThreads)
improve_heavy_chunk_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col,
                           const int *__restrict__ w, int sign, int nchunks, Workspace ws) {
    __shared__ Cand s_b[2][kHeavyThreads / 32];
    const int H = ws.ctrl->cls_cnt[kClasses];
    const int *hv = ws.cls_list + ws.ctrl->cls_off[kClasses];
    const int total = ws.ctrl->heavy_edges;
    const int4 *rec = reinterpret_cast<const int4 *>(ws.rec);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Cand none{INT_MIN, INT_MAX, LLONG_MIN};
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int g0 = c * kHeavyChunk, g1 = min(g0 + kHeavyChunk, total);
        // the heavy vertex holding entry g0: largest i with heavy_off[i] <= g0
        int lo = 0, hi = H;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (ws.heavy_off[mid] <= g0) lo = mid; else hi = mid;
        }
        const int split = min(ws.heavy_off[lo + 1], g1);   // entries below: vertex lo
        const int base0 = __ldg(&row_ptr[hv[lo]]) - ws.heavy_off[lo];
        const int base1 = split < g1 ? __ldg(&row_ptr[hv[lo + 1]]) - ws.heavy_off[lo + 1] : 0;
        Cand b0 = none, b1 = none;
        for (int g = g0 + (int)threadIdx.x; g < g1; g += blockDim.x) {
            const bool first = g < split;
            const Cand x = edge_cand<RATIO>(col, w, rec, ws, sign, (first ? base0 : base1) + g);
            if (first) {
                if (better(x, b0)) b0 = x;
            } else if (better(x, b1)) {
                b1 = x;
            }
        }
        b0 = warp_best(b0);
        b1 = warp_best(b1);
        if (lane == 0) {
            s_b[0][warp] = b0;
            s_b[1][warp] = b1;
        }
        __syncthreads();
        if (warp == 0) {
            Cand x0 = lane < kHeavyThreads / 32 ? s_b[0][lane] : none;
            Cand x1 = lane < kHeavyThreads / 32 ? s_b[1][lane] : none;
            x0 = warp_best(x0);
            x1 = warp_best(x1);
            if (lane == 0) {
                ws.heavy_part[2 * c] = x0;
                ws.heavy_part[2 * c + 1] = x1;
            }
        }
        __syncthreads();   // s_b is reused by the next chunk
    }
}

template <bool RATIO>
__global__ void __launch_bounds__(kHeavyThreads)
improve_heavy_final_kernel(const int *__restrict__ col, const int *__restrict__ w, int sign,
                           Workspace ws, BatchState bs) {
    __shared__ Cand s_w[kHeavyThreads / 32];
    const int H = ws.ctrl->cls_cnt[kClasses];
    const int *hv = ws.cls_list + ws.ctrl->cls_off[kClasses];
    const int next_eval = ws.ctrl->iter + 1;
    const int4 *rec = reinterpret_cast<const int4 *>(ws.rec);
    int switched = 0;
    for (int i = blockIdx.x; i < H; i += gridDim.x) {   // one block per heavy vertex
        const int v = hv[i];
        const Cand best = heavy_combine(ws, i, s_w);
        if (threadIdx.x == 0 && !(bs.G && bs.gconv[bs.gid[v]])) {
            const int t = ws.succ[v];
            const int4 r = __ldg(&rec[t]);
            const long long V = ((long long)(unsigned)r.x) | ((long long)r.y << 32);
            long long cur_key = (long long)r.w * (long long)ws.wpi[v] + V;
            if (RATIO) cur_key -= __ldg(&ws.recp[t]) * (long long)ws.tpi[v];
            if (best.rank > r.z || (best.rank == r.z && best.key > cur_key)) {
                ws.pi[v] = best.e;
                ws.succ[v] = __ldg(&col[best.e]);
                ws.wpi[v] = sign * __ldg(&w[best.e]);
                if (RATIO) ws.tpi[v] = __ldg(&ws.transit[best.e]);
                ws.sw_iter[v] = next_eval;
                if (bs.G) {
                    const int g = bs.gid[v];
                    if (bs.gsw[g] != next_eval) bs.gsw[g] = next_eval;
                }
                ++switched;
            }
        }
    }
    if (threadIdx.x == 0 && switched) {
        atomicAdd(&ws.ctrl->switched, switched);
        ws.ctrl->changed = 1;
    }
}

// The heavy vertices' chunk and combine kernels after a lane-group sweep;
// returns the number of launches (0 without heavy vertices).
int launch_sweep_heavy(const int *row_ptr, const int *col, const int *w, int sign, Workspace ws,
                       int H, int heavy_edges, BatchState bs, cudaStream_t st) {
    if (H <= 0 || heavy_edges <= 0) return 0;
    const bool ratio = ws.transit != nullptr;
    const int nchunks = (heavy_edges + kHeavyChunk - 1) / kHeavyChunk;
    const int cb = nchunks < 4096 ? nchunks : 4096;
    const int fb = H < 4096 ? H : 4096;
    if (ratio) {
        improve_heavy_chunk_kernel<true><<<cb, kHeavyThreads, 0, st>>>(row_ptr, col, w, sign,
                                                                      nchunks, ws);
        improve_heavy_final_kernel<true><<<fb, kHeavyThreads, 0, st>>>(col, w, sign, ws, bs);
    } else {
        improve_heavy_chunk_kernel<false><<<cb, kHeavyThreads, 0, st>>>(row_ptr, col, w, sign,
                                                                       nchunks, ws);
        improve_heavy_final_kernel<false><<<fb, kHeavyThreads, 0, st>>>(col, w, sign, ws, bs);
    }
    return 2;
}

int launch_sweep(const int *row_ptr, const int *col, const int *w, int sign, int n,
                 Workspace ws, const int *cls_cnt, int heavy_edges, BatchState bs, int threads,
                 int band_blocks, cudaStream_t st) {
    // the warp tasks: per class (one band), else an upper bound (each (band,
    // class) group rounds up to whole tasks; the kernel reads the exact count
    // from the group table)
    ClassGrid cg;
    long long tasks = 0;
    for (int c = 0; c < kClasses; ++c) {
        cg.task_off[c] = (int)tasks;
        tasks += (((long long)cls_cnt[c] << c) + 31) / 32;
    }
    cg.task_off[kClasses] = (int)tasks;
    cg.band_blocks = band_blocks;
    const int groups = sweep_groups(n, band_blocks);
    const bool banded = groups > kClasses;
    if (banded) tasks += groups;
    if (threads != 128 && threads != 256 && threads != 512) threads = kSweepThreads;
    const bool ratio = ws.transit != nullptr;
    const int grid_blocks = ratio ? classes_grid<true>(threads) : classes_grid<false>(threads);
    if (grid_blocks <= 0) return -1;
    const int wpb = threads / 32;
    long long blocks = (tasks + wpb - 1) / wpb;
    if (blocks > grid_blocks) blocks = grid_blocks;
    if (blocks < 1) blocks = 1;   // block 0 also publishes the evaluation's best cycle
    prof_begin(kProfSweep, st);
    const int nb = (int)blocks;
#define OCM_IMPROVE(R, B, F) \
    improve_kernel<R, B, F><<<nb, threads, 0, st>>>(row_ptr, col, w, sign, n, groups, cg, ws, bs)
    if (ratio && banded) {
        OCM_IMPROVE(true, true, false);
        OCM_IMPROVE(true, true, true);
    } else if (ratio) {
        OCM_IMPROVE(true, false, false);
        OCM_IMPROVE(true, false, true);
    } else if (banded) {
        OCM_IMPROVE(false, true, false);
        OCM_IMPROVE(false, true, true);
    } else {
        OCM_IMPROVE(false, false, false);
        OCM_IMPROVE(false, false, true);
    }
#undef OCM_IMPROVE
    int launches = 2;
    const int kh = launch_sweep_heavy(row_ptr, col, w, sign, ws, cls_cnt[kClasses], heavy_edges,
                                      bs, st);
    if (kh < 0) return -1;
    launches += kh;
    prof_end(kProfSweep, st);
    return launches;
}

}  // namespace ocm
