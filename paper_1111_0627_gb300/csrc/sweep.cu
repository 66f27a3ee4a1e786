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
// Layout: one CTA per tile of 256 consecutive vertices.  The tile's edges are
// streamed in chunks of 2048 with coalesced loads; each edge's target record
// (16 B: V, rank, q) is gathered and its key written to shared memory; then
// each thread reduces the segment of its own vertex.  A vertex with more
// edges than a chunk is reduced across chunks in registers.
#include "common.cuh"

namespace ocm {

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

// Phase 2 of a tile: thread-owned segmented reduction over the staged keys.
struct Best {
    int rank;
    long long key;
    int e;
};

template <bool kInit>
__global__ void __launch_bounds__(kThreads)
sweep_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col,
             const int *__restrict__ w, int sign, int n, Workspace ws) {
    __shared__ long long s_key[kSweepChunkE];
    __shared__ int s_rank[kSweepChunkE];
    __shared__ int s_maxw[kThreads / 32];

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int v0 = blockIdx.x * kSweepTileV;
    const int v = v0 + tid;
    const bool has_v = v < n;
    const int vend = min(v0 + kSweepTileV, n);
    const int e_begin = __ldg(&row_ptr[v0]);
    const int e_end = __ldg(&row_ptr[vend]);
    const int my_b = has_v ? __ldg(&row_ptr[v]) : 0;
    const int my_e = has_v ? __ldg(&row_ptr[v + 1]) : 0;
    const int my_pi = (!kInit && has_v) ? ws.pi[v] : -1;

    if (blockIdx.x == 0 && tid == 0) {
        // Publish the best cycle of the evaluation this sweep reads (it is
        // the answer if nothing switches), then reset the counters of the
        // next evaluation.  No other thread of this kernel touches them.
        Ctrl *c = ws.ctrl;
        if (!kInit) {
            unsigned long long b = c->best;
            int root = INT_MAX - (int)(unsigned)(b & 0xffffffffu);
            int i = ws.cid_of_root[root];
            c->res_root = root;
            c->res_len = ws.cyc_L[i];
            c->res_num = ws.cyc_p[i];
            c->res_den = ws.cyc_q[i];
            c->res_cycles = c->nrep;
        }
        c->cnt[0] = c->cnt[1] = c->cnt[2] = 0;
        c->nrep = 0;
        c->best = 0;
    }
    Best best{INT_MIN, LLONG_MIN, -1};
    int cur_rank = INT_MIN;
    long long cur_key = LLONG_MIN;
    int maxabs = 0;

    for (int cs = e_begin; cs < e_end; cs += kSweepChunkE) {
        const int ce = min(cs + kSweepChunkE, e_end);
        // phase 1: stream the chunk's edges, gather target records
        constexpr int U = kSweepChunkE / kThreads;
        int tgt[U], wt[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int e = cs + u * kThreads + tid;
            tgt[u] = 0;
            wt[u] = 0;
            if (e < ce) {
                tgt[u] = __ldg(&col[e]);
                wt[u] = __ldg(&w[e]);
            }
        }
        if (kInit) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int e = cs + u * kThreads + tid;
                if (e < ce) {
                    int t = tgt[u];
                    int x = wt[u];
                    if ((unsigned)t >= (unsigned)n) {
                        atomicOr(&ws.ctrl->err, kErrCol);
                        atomicMin(&ws.ctrl->bad_index, e);
                    }
                    if (x == INT_MIN) {
                        atomicOr(&ws.ctrl->err, kErrWeightMin);
                        atomicMin(&ws.ctrl->bad_index, e);
                        x = 0;
                    }
                    int ax = x < 0 ? -x : x;
                    maxabs = max(maxabs, ax);
                    s_key[e - cs] = (long long)(sign * x);
                    s_rank[e - cs] = 0;
                }
            }
        } else {
            Rec r[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int e = cs + u * kThreads + tid;
                if (e < ce) {
                    int4 raw = __ldg(reinterpret_cast<const int4 *>(ws.rec) + tgt[u]);
                    r[u].V = ((long long)(unsigned)raw.x) | ((long long)raw.y << 32);
                    r[u].rank = raw.z;
                    r[u].q = raw.w;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int e = cs + u * kThreads + tid;
                if (e < ce) {
                    s_key[e - cs] = (long long)r[u].q * (long long)(sign * wt[u]) + r[u].V;
                    s_rank[e - cs] = r[u].rank;
                }
            }
        }
        __syncthreads();
        // phase 2: each thread reduces its own vertex's edges in this chunk
        if (has_v) {
            int a = max(my_b, cs), b = min(my_e, ce);
            for (int e = a; e < b; ++e) {
                int rk = s_rank[e - cs];
                long long k = s_key[e - cs];
                if (rk > best.rank || (rk == best.rank && k > best.key)) {
                    best.rank = rk;
                    best.key = k;
                    best.e = e;
                }
                if (e == my_pi) {
                    cur_rank = rk;
                    cur_key = k;
                }
            }
        }
        __syncthreads();
    }

    if (kInit) {
        // block max of |w|
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) maxabs = max(maxabs, __shfl_xor_sync(0xffffffffu, maxabs, o));
        if (lane == 0) s_maxw[tid >> 5] = maxabs;
        __syncthreads();
        if (tid < 32) {
            int x = tid < kThreads / 32 ? s_maxw[tid] : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
            if (tid == 0) atomicMax(&ws.ctrl->maxabsw, x);
        }
        if (has_v && best.e >= 0) {
            int t = __ldg(&col[best.e]);
            ws.pi[v] = best.e;
            ws.succ[v] = ((unsigned)t < (unsigned)n) ? t : 0;
            int x = __ldg(&w[best.e]);
            ws.wpi[v] = sign * (x == INT_MIN ? 0 : x);
        }
        return;
    }

    bool sw = has_v && (best.rank > cur_rank || (best.rank == cur_rank && best.key > cur_key));
    if (sw) {
        ws.pi[v] = best.e;
        ws.succ[v] = __ldg(&col[best.e]);
        ws.wpi[v] = sign * __ldg(&w[best.e]);
    }
    unsigned mask = __ballot_sync(0xffffffffu, sw);
    if (mask && lane == 0) {
        atomicAdd(&ws.ctrl->switched, __popc(mask));
        ws.ctrl->changed = 1;
    }
}

void launch_init_policy(const int *row_ptr, const int *col, const int *w, int sign, int n, int m,
                        Workspace ws, cudaStream_t st) {
    (void)m;
    int tiles = (n + kSweepTileV - 1) / kSweepTileV;
    prof_begin(kProfInit, st);
    sweep_kernel<true><<<tiles, kThreads, 0, st>>>(row_ptr, col, w, sign, n, ws);
    prof_end(kProfInit, st);
}

void launch_sweep(const int *row_ptr, const int *col, const int *w, int sign, int n,
                  Workspace ws, cudaStream_t st) {
    int tiles = (n + kSweepTileV - 1) / kSweepTileV;
    prof_begin(kProfSweep, st);
    sweep_kernel<false><<<tiles, kThreads, 0, st>>>(row_ptr, col, w, sign, n, ws);
    prof_end(kProfSweep, st);
}

}  // namespace ocm
