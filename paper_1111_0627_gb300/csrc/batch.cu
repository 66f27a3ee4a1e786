// batch.cu -- the batched form: G independent graphs solved together as one
// disjoint-union CSR.
//
// Multichain policy iteration never lets one weakly connected component
// influence another: the improvement sweep of a vertex reads only its own
// out-edges' targets, and the ranks used to compare cycle means are a
// global order-preserving relabelling, so every graph follows exactly the
// trajectory it would follow alone (the paper's SCC extension, Sec. 3.3,
// solves its regions concurrently in the same spirit).  What the batch adds
// is per-graph bookkeeping: a graph id per vertex, the per-graph best cycle
// (Alg. 4's region-specific vote, made deterministic by a total order on
// (rank, root)), and the extraction of every graph's critical cycle at once.
#include <climits>

#include "common.cuh"

namespace ocm {

// Graph offsets: vptr[0] = 0, vptr[G] = N, every graph non-empty.
__global__ void __launch_bounds__(kThreads)
batch_check_kernel(const int *__restrict__ vptr, int G, int N, int *bs_gconv, int *bs_gsw,
                   Ctrl *ctrl) {
    const int stride = gridDim.x * blockDim.x;
    int local_max = 0;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += stride) {
        const int a = vptr[g], b = vptr[g + 1];
        bs_gconv[g] = 0;
        bs_gsw[g] = 0;
        if ((g == 0 && a != 0) || (g == G - 1 && b != N) || b <= a || a < 0 || b > N) {
            atomicOr(&ctrl->err, kErrRowPtr);
            atomicMin(&ctrl->bad_index, g);
        } else {
            local_max = max(local_max, b - a);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local_max = max(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    if ((threadIdx.x & 31) == 0 && local_max) atomicMax(&ctrl->max_ng, local_max);
}

// gid[v] = the g with vptr[g] <= v < vptr[g+1] (binary search, clamped so a
// malformed vptr cannot produce an out-of-range id before it is rejected).
__global__ void __launch_bounds__(kThreads)
batch_gid_kernel(const int *__restrict__ vptr, int G, int N, int *gid) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += stride) {
        int lo = 0, hi = G - 1;
        while (lo < hi) {
            const int mid = lo + (hi - lo + 1) / 2;
            if (__ldg(&vptr[mid]) <= v) lo = mid; else hi = mid - 1;
        }
        gid[v] = lo;
    }
}

int launch_batch_prepare(int N, int M, BatchState bs, Workspace ws, cudaStream_t st) {
    (void)M;
    int gb = (bs.G + kThreads - 1) / kThreads;
    if (gb > 1024) gb = 1024;
    int vb = (N + kThreads - 1) / kThreads;
    if (vb > 4096) vb = 4096;
    prof_begin(kProfInit, st);
    batch_check_kernel<<<gb, kThreads, 0, st>>>(bs.vptr, bs.G, N, bs.gconv, bs.gsw, ws.ctrl);
    batch_gid_kernel<<<vb, kThreads, 0, st>>>(bs.vptr, bs.G, N, bs.gid);
    prof_end(kProfInit, st);
    return 2;
}

// After each sweep: a graph none of whose vertices switched is final (the
// paper's per-region "work" flag, Sec. 3.3).  Its answer is taken from the
// evaluation that preceded this sweep -- the per-graph vote and the cycle
// tables are still those of that evaluation -- and it drops out of later
// evaluations and sweeps.
__global__ void __launch_bounds__(kThreads)
batch_converge_kernel(BatchState bs, Workspace ws) {
    const int stride = gridDim.x * blockDim.x;
    const int next_eval = ws.ctrl->iter + 1;   // the stamp of the sweep just run
    int active = 0;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < bs.G; g += stride) {
        if (bs.gconv[g]) continue;
        if (bs.gsw[g] == next_eval) {
            ++active;
            continue;
        }
        const unsigned long long packed = bs.gbest[g];
        const int root = INT_MAX - (int)(unsigned)(packed & 0xffffffffu);
        if (packed == 0 || root < bs.vptr[g] || root >= bs.vptr[g + 1]) {
            atomicOr(&ws.ctrl->err, kErrExtract);
            continue;
        }
        const int i = ws.cid_of_root[root];
        bs.groot[g] = root;
        bs.glen[g] = ws.cyc_L[i];
        bs.gp[g] = ws.cyc_p[i];
        bs.gq[g] = ws.cyc_q[i];
        bs.gconv[g] = 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) active += __shfl_xor_sync(0xffffffffu, active, o);
    if ((threadIdx.x & 31) == 0 && active) atomicAdd(&ws.ctrl->active_graphs, active);
}

__global__ void batch_active_reset_kernel(Ctrl *c) { c->active_graphs = 0; }

int launch_batch_converge(BatchState bs, Workspace ws, cudaStream_t st) {
    int gb = (bs.G + kThreads - 1) / kThreads;
    if (gb > 1024) gb = 1024;
    batch_active_reset_kernel<<<1, 1, 0, st>>>(ws.ctrl);
    batch_converge_kernel<<<gb, kThreads, 0, st>>>(bs, ws);
    return 2;
}

// Per-graph answers recorded when each graph converged.
__global__ void __launch_bounds__(kThreads)
batch_results_kernel(int sign, BatchState bs, Workspace ws, int64_t *num, int32_t *den,
                     int32_t *cycle_len) {
    const int stride = gridDim.x * blockDim.x;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < bs.G; g += stride) {
        if (!bs.gconv[g]) {
            atomicOr(&ws.ctrl->err, kErrExtract);
            continue;
        }
        num[g] = (int64_t)sign * bs.gp[g];
        den[g] = bs.gq[g];
        cycle_len[g] = bs.glen[g];
        bs.gfound[g] = 0;
    }
}

// Appends to a global list with one atomic per block.
static __device__ __forceinline__ void block_global_append(int *list, int *counter, bool pred,
                                                           int item) {
    __shared__ int s_base, s_cnt;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const unsigned mask = __ballot_sync(0xffffffffu, pred);
    int wbase = 0;
    if (lane == 0 && mask) wbase = atomicAdd(&s_cnt, __popc(mask));
    wbase = __shfl_sync(0xffffffffu, wbase, 0);
    __syncthreads();
    if (threadIdx.x == 0) s_base = s_cnt ? atomicAdd(counter, s_cnt) : 0;
    __syncthreads();
    if (pred) list[s_base + wbase + __popc(mask & ((1u << lane) - 1u))] = item;
}

// Candidates of every graph's critical cycle: root(v) = root of g(v) and
// len(v) < L_g (the set is closed under succ).
__global__ void __launch_bounds__(kThreads)
batch_candidates_kernel(int N, BatchState bs, Workspace ws) {
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < N; base += stride) {
        const int v = base + threadIdx.x;
        bool cand = false;
        if (v < N) {
            const int g = bs.gid[v];
            const JLS st = ws.jls[0][v];
            cand = (~st.J == bs.groot[g]) && st.len < bs.glen[g];
            if (cand) ws.aprev[v] = v;
        }
        block_global_append(ws.list[0], &ws.ctrl->ncand, cand, v);
    }
}

// Binary lifting round b: cur(v) <- J_b(cur(v)) if bit b of L_{g(v)} is set.
__global__ void __launch_bounds__(kThreads)
batch_lift_kernel(int b, BatchState bs, Workspace ws) {
    const int K = *reinterpret_cast<const volatile int *>(&ws.ctrl->ncand);
    const int *Jin = (b == 0) ? ws.succ : reinterpret_cast<const int *>(ws.jm[b & 1]);
    int *Jout = reinterpret_cast<int *>(ws.jm[(b + 1) & 1]);
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += stride) {
        const int v = ws.list[0][i];
        if ((bs.glen[bs.gid[v]] >> b) & 1) ws.aprev[v] = Jin[ws.aprev[v]];
        Jout[v] = Jin[Jin[v]];
    }
}

// v is on its graph's critical cycle iff succ^{L}(v) = v; it goes to
// position (L - len(v)) mod L of that graph's slice of cycle_out.
__global__ void __launch_bounds__(kThreads)
batch_scatter_kernel(BatchState bs, Workspace ws, int32_t *cycle_out) {
    const int K = *reinterpret_cast<const volatile int *>(&ws.ctrl->ncand);
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += stride) {
        const int v = ws.list[0][i];
        if (ws.aprev[v] == v) {
            const int g = bs.gid[v];
            const int L = bs.glen[g];
            const int len = ws.jls[0][v].len;
            const int pos = (len == 0) ? 0 : L - len;
            cycle_out[bs.vptr[g] + pos] = ws.pi[v];
            atomicAdd(&bs.gfound[g], 1);
        }
    }
}

__global__ void __launch_bounds__(kThreads)
batch_verify_kernel(BatchState bs, Ctrl *ctrl) {
    const int stride = gridDim.x * blockDim.x;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < bs.G; g += stride)
        if (bs.gfound[g] != bs.glen[g]) atomicOr(&ctrl->err, kErrExtract);
}

__global__ void batch_extract_reset_kernel(Ctrl *c) { c->ncand = 0; }

int launch_batch_finish(int N, int sign, int Lbits, BatchState bs, Workspace ws, int64_t *num,
                        int32_t *den, int32_t *cycle_len, int32_t *cycle_out, int grid,
                        cudaStream_t st) {
    int gb = (bs.G + kThreads - 1) / kThreads;
    if (gb > 1024) gb = 1024;
    prof_begin(kProfExtract, st);
    batch_results_kernel<<<gb, kThreads, 0, st>>>(sign, bs, ws, num, den, cycle_len);
    batch_extract_reset_kernel<<<1, 1, 0, st>>>(ws.ctrl);
    batch_candidates_kernel<<<grid, kThreads, 0, st>>>(N, bs, ws);
    int launches = 3;
    for (int b = 0; b < Lbits; ++b, ++launches) batch_lift_kernel<<<grid, kThreads, 0, st>>>(b, bs, ws);
    batch_scatter_kernel<<<grid, kThreads, 0, st>>>(bs, ws, cycle_out);
    batch_verify_kernel<<<gb, kThreads, 0, st>>>(bs, ws.ctrl);
    prof_end(kProfExtract, st);
    return launches + 2;
}

}  // namespace ocm
