// evaluate.cu -- evaluation of a policy (Alg. 1: MinMeanWeightCycle(G_pi) and
// the value propagation that follows it; Alg. 2: elimination*,
// cycleIdentification, reduce_min, setMinCycle, GpiPreprocess and
// valuePropagate*), re-designed as pointer-jumping kernels.
//
// G_pi is a functional graph: every vertex has one successor succ(v), every
// weakly connected component holds exactly one cycle (Sec. 2.4).  Per policy:
//   detect  (replaces elimination* + cycleIdentification): for each v, the
//           root of the cycle v reaches = the cycle's smallest vertex.
//           Doubling: J_{k+1}(v) = J_k(J_k(v)), M_{k+1}(v) = min(M_k(v),
//           M_k(J_k(v))), so A_k(v) = M_k(J_k(v)) is the smallest vertex in
//           positions [2^k, 2^(k+1)) of v's path.  If A_k(v) == A_{k-1}(v) = x,
//           x occurs twice on the path, hence on the cycle, and the stretch
//           between its occurrences covers the whole cycle, so x is the
//           cycle's smallest vertex.  Conversely once 2^(k-1) exceeds both the
//           depth of v and the cycle length the test holds, so the round count
//           adapts to the policy graph instead of log2(n).  A vertex whose
//           jump target is already resolved takes that root (the target lies
//           on its path).  Resolved vertices leave the worklist.
//   values  (replaces valuePropagate*, Alg. 3): cut each cycle at its root
//           (Alg. 1: the root is not re-entered, val(root) = 0) and jump with
//           accumulated (length, weight) pairs until every vertex reaches its
//           root: S(v) = s*w-weight and len(v) = length of v's path to it.
//   cycles  (replaces cycleIdentification + reduce_min): for root r,
//           W = s*w(pi(r)) + S(succ r), L = 1 + len(succ r); the mean is p/q =
//           W/L reduced.  Each mean gets an exact integer key floor(p n^2/q)
//           (distinct fractions with denominators <= n differ by >= 1/n^2) and
//           a rank = number of cycles with a smaller key.  The best cycle is
//           the largest mean, ties to the smallest root (Alg. 4's region vote,
//           made deterministic by a total order).
//   materialise: V(v) = q*S(v) - p*len(v), the record {V, rank, q} the next
//           improvement sweep gathers per edge target.
#include <climits>

#include "common.cuh"

namespace ocm {

static __device__ __forceinline__ int load_count(const int *p) {
    return *reinterpret_cast<const volatile int *>(p);
}

// ---------------------------------------------------------------- detect --
// State encoding: JM.J >= 0 -> unresolved jump state; JM.J < 0 -> resolved,
// root = ~J.  A list entry v >= 0 is a vertex to advance, ~v marks a resolved
// vertex whose state is copied into the other buffer once, so that both
// buffers hold it for later readers (no buffer is written while being read).
__global__ void __launch_bounds__(kThreads)
detect_round_kernel(int r, int n, Workspace ws) {
    Ctrl *c = ws.ctrl;
    const bool first = (r == 0);
    const int in_slot = r % 3, out_slot = (r + 1) % 3, zero_slot = (r + 2) % 3;
    const int count = first ? n : load_count(&c->cnt[in_slot]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->cnt[zero_slot] = 0;
        if (count > 0) c->rounds_detect += 1;
        c->items_detect += count;
    }
    if (count == 0) return;
    const JM *in = ws.jm[r & 1];
    JM *out = ws.jm[(r + 1) & 1];
    const int *lin = ws.list[in_slot];
    int *lout = ws.list[out_slot];
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < count; base += stride) {
        const int idx = base + threadIdx.x;
        bool keep = false, resolved = false, is_root = false;
        int v = 0;
        if (idx < count) {
            int item = first ? idx : lin[idx];
            if (item < 0) {
                v = ~item;
                out[v] = in[v];          // copy-forward of a resolved state
            } else {
                v = item;
                JM s = first ? JM{ws.succ[v], v} : in[v];
                int J = s.J;
                JM t = first ? JM{ws.succ[J], J} : in[J];
                int root = -1;
                if (t.J < 0) {
                    root = ~t.J;         // J already resolved: it lies on v's path
                } else if (!first && t.M == ws.aprev[v]) {
                    root = t.M;          // smallest vertex of the cycle
                } else {
                    out[v] = JM{t.J, min(s.M, t.M)};
                    ws.aprev[v] = t.M;
                    keep = true;
                }
                if (root >= 0) {
                    out[v] = JM{~root, 0};
                    ws.rep[v] = root;
                    resolved = true;
                    is_root = (root == v);
                }
            }
        }
        int pos = warp_append(&c->cnt[out_slot], keep || resolved, lane);
        if (keep) lout[pos] = v;
        if (resolved) lout[pos] = ~v;
        int rpos = warp_append(&c->nrep, is_root, lane);
        if (is_root) ws.cyc_root[rpos] = v;
    }
}

// ---------------------------------------------------------------- values --
// State encoding: JLS.J >= 0 -> unresolved; JLS.J < 0 -> final, root = ~J,
// (len, S) = length and weight of the whole path to the root.
__global__ void __launch_bounds__(kThreads)
value_init_kernel(int slot_base, int n, Workspace ws) {
    Ctrl *c = ws.ctrl;
    const int out_slot = (slot_base + 1) % 3, zero_slot = (slot_base + 2) % 3;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (load_count(&c->cnt[slot_base % 3]) != 0) atomicOr(&c->err, kErrDetect);
        c->cnt[zero_slot] = 0;
    }
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const int v = base + threadIdx.x;
        bool keep = false;
        if (v < n) {
            int rv = ws.rep[v];
            JLS st;
            bool fin;
            if (rv == v) {
                st = JLS{~v, 0, 0};
                fin = true;
            } else {
                int s = ws.succ[v];
                fin = (ws.rep[s] == s);
                st = JLS{fin ? ~s : s, 1, (long long)ws.wpi[v]};
            }
            ws.jls[0][v] = st;
            if (fin) ws.jls[1][v] = st;
            keep = !fin;
        }
        int pos = warp_append(&c->cnt[out_slot], keep, lane);
        if (keep) ws.list[out_slot][pos] = v;
    }
}

__global__ void __launch_bounds__(kThreads)
value_round_kernel(int slot, int j, Workspace ws) {
    Ctrl *c = ws.ctrl;
    const int in_slot = slot % 3, out_slot = (slot + 1) % 3, zero_slot = (slot + 2) % 3;
    const int count = load_count(&c->cnt[in_slot]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->cnt[zero_slot] = 0;
        if (count > 0) c->rounds_value += 1;
        c->items_value += count;
    }
    if (count == 0) return;
    const JLS *in = ws.jls[(j + 1) & 1];
    JLS *out = ws.jls[j & 1];
    const int *lin = ws.list[in_slot];
    int *lout = ws.list[out_slot];
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < count; base += stride) {
        const int idx = base + threadIdx.x;
        bool keep = false, fin = false;
        int v = 0;
        if (idx < count) {
            int item = lin[idx];
            if (item < 0) {
                v = ~item;
                out[v] = in[v];
            } else {
                v = item;
                JLS s = in[v];
                JLS t = in[s.J];
                JLS u{t.J, s.len + t.len, s.S + t.S};
                out[v] = u;
                fin = u.J < 0;
                keep = !fin;
            }
        }
        int pos = warp_append(&c->cnt[out_slot], keep || fin, lane);
        if (keep) lout[pos] = v;
        if (fin) lout[pos] = ~v;
    }
}

// ---------------------------------------------------------------- cycles --
__global__ void __launch_bounds__(kThreads)
cycle_stats_kernel(int final_slot, long long N2, Workspace ws) {
    Ctrl *c = ws.ctrl;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (load_count(&c->cnt[final_slot % 3]) != 0) atomicOr(&c->err, kErrValue);
    }
    const int K = load_count(&c->nrep);
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += stride) {
        int r = ws.cyc_root[i];
        int x = ws.succ[r];
        JLS st = ws.jls[0][x];
        long long W = (long long)ws.wpi[r] + st.S;
        long long L = 1 + (long long)st.len;
        long long g = gcd_ll(W, L);
        long long p = W / g, q = L / g;
        ws.cyc_p[i] = p;
        ws.cyc_q[i] = (int)q;
        ws.cyc_L[i] = (int)L;
        ws.cyc_key[i] = mean_key(p, q, N2);
        ws.cid_of_root[r] = i;
    }
}

constexpr int kRankTile = 2048;

__global__ void __launch_bounds__(kThreads)
cycle_rank_kernel(Workspace ws) {
    __shared__ long long s_key[kRankTile];
    Ctrl *c = ws.ctrl;
    const int K = load_count(&c->nrep);
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < K; base += stride) {
        const int i = base + threadIdx.x;
        const long long key = i < K ? ws.cyc_key[i] : 0;
        int rank = 0;
        for (int t0 = 0; t0 < K; t0 += kRankTile) {
            int tn = min(kRankTile, K - t0);
            __syncthreads();
            for (int j = threadIdx.x; j < tn; j += blockDim.x) s_key[j] = ws.cyc_key[t0 + j];
            __syncthreads();
            for (int j = 0; j < tn; ++j) rank += (s_key[j] < key);
        }
        if (i < K) {
            ws.cyc_rank[i] = rank;
            unsigned long long packed = ((unsigned long long)(unsigned)rank << 32) |
                                        (unsigned)(INT_MAX - ws.cyc_root[i]);
            atomicMax(&c->best, packed);
        }
    }
}

__global__ void __launch_bounds__(kThreads)
materialise_kernel(int n, Workspace ws) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ws.ctrl->changed = 0;
        ws.ctrl->switched = 0;
    }
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        JLS st = ws.jls[0][v];
        int i = ws.cid_of_root[~st.J];
        long long p = ws.cyc_p[i];
        int q = ws.cyc_q[i];
        Rec rec;
        rec.V = (long long)q * st.S - p * (long long)st.len;
        rec.rank = ws.cyc_rank[i];
        rec.q = q;
        ws.rec[v] = rec;
    }
}

static int ceil_log2(long long x) {
    int k = 0;
    while ((1LL << k) < x) ++k;
    return k;
}

// Launches one policy evaluation; returns the number of kernel launches.
int launch_evaluate(int n, long long N2, Workspace ws, int grid, cudaStream_t st) {
    int launches = 0;
    const int lg = ceil_log2(n);
    const int R2 = lg + 4;       // detect rounds incl. one copy-forward round
    for (int r = 0; r < R2; ++r, ++launches) {
        prof_begin(kProfDetect, st);
        detect_round_kernel<<<grid, kThreads, 0, st>>>(r, n, ws);
        prof_end(kProfDetect, st);
    }
    int slot = R2;               // value init appends to slot R2+1
    prof_begin(kProfValue, st);
    value_init_kernel<<<grid, kThreads, 0, st>>>(slot, n, ws);
    prof_end(kProfValue, st);
    ++launches;
    const int R5 = lg + 2;       // value rounds incl. one copy-forward round
    for (int j = 1; j <= R5; ++j, ++launches) {
        prof_begin(kProfValue, st);
        value_round_kernel<<<grid, kThreads, 0, st>>>(slot + j, j, ws);
        prof_end(kProfValue, st);
    }
    // Every final state is written in the buffer of its round and copied once
    // into the other, so after the last round both buffers hold all of them.
    prof_begin(kProfCycles, st);
    cycle_stats_kernel<<<grid, kThreads, 0, st>>>(slot + R5 + 1, N2, ws);
    prof_end(kProfCycles, st);
    prof_begin(kProfCycles, st);
    cycle_rank_kernel<<<grid, kThreads, 0, st>>>(ws);
    prof_end(kProfCycles, st);
    prof_begin(kProfMaterialise, st);
    materialise_kernel<<<grid, kThreads, 0, st>>>(n, ws);
    prof_end(kProfMaterialise, st);
    launches += 3;
    return launches;
}

// --------------------------------------------------------------- extract --
// Critical cycle of root r* (length L*): its vertices are exactly the v with
// root(v) = r*, len(v) < L* and succ^{L*}(v) = v; v sits at position
// (L* - len(v)) mod L* counted from r*.  succ^{L*} is evaluated for all
// candidates at once by binary lifting over the bits of L* (the candidate set
// is closed under succ, so the jump tables never leave it).
__global__ void __launch_bounds__(kThreads)
extract_candidates_kernel(int n, Workspace ws) {
    Ctrl *c = ws.ctrl;
    const int root = c->res_root, L = c->res_len;
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    int *cur = ws.aprev;
    for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const int v = base + threadIdx.x;
        bool cand = false;
        if (v < n) {
            JLS st = ws.jls[0][v];
            cand = (~st.J == root) && st.len < L;
            if (cand) cur[v] = v;
        }
        int pos = warp_append(&c->ncand, cand, lane);
        if (cand) ws.list[0][pos] = v;
    }
}

__global__ void __launch_bounds__(kThreads)
extract_round_kernel(int b, Workspace ws) {
    Ctrl *c = ws.ctrl;
    const int K = load_count(&c->ncand);
    const int L = c->res_len;
    const int *Jin = (b == 0) ? ws.succ : reinterpret_cast<const int *>(ws.jm[b & 1]);
    int *Jout = reinterpret_cast<int *>(ws.jm[(b + 1) & 1]);
    int *cur = ws.aprev;
    const bool take = (L >> b) & 1;
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += stride) {
        int v = ws.list[0][i];
        if (take) cur[v] = Jin[cur[v]];
        Jout[v] = Jin[Jin[v]];
    }
}

__global__ void __launch_bounds__(kThreads)
extract_scatter_kernel(Workspace ws, int *cycle_out) {
    Ctrl *c = ws.ctrl;
    const int K = load_count(&c->ncand);
    const int L = c->res_len;
    const int stride = gridDim.x * blockDim.x;
    int found = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += stride) {
        int v = ws.list[0][i];
        if (ws.aprev[v] == v) {
            int len = ws.jls[0][v].len;
            int pos = (len == 0) ? 0 : L - len;
            cycle_out[pos] = ws.pi[v];
            ++found;
        }
    }
    if (found) atomicAdd(&c->cnt[0], found);
}

__global__ void extract_reset_kernel(Workspace ws) {
    ws.ctrl->ncand = 0;
    ws.ctrl->cnt[0] = 0;
}

// Extracts the critical cycle (root and length already in ctrl->res_*);
// returns the number of kernel launches.
int launch_extract(int n, int Lstar, Workspace ws, int *cycle_out, int grid, cudaStream_t st) {
    prof_begin(kProfExtract, st);
    extract_reset_kernel<<<1, 1, 0, st>>>(ws);
    extract_candidates_kernel<<<grid, kThreads, 0, st>>>(n, ws);
    int launches = 2;
    int bits = 0;
    while ((1LL << bits) <= Lstar) ++bits;
    for (int b = 0; b < bits; ++b, ++launches) extract_round_kernel<<<grid, kThreads, 0, st>>>(b, ws);
    extract_scatter_kernel<<<grid, kThreads, 0, st>>>(ws, cycle_out);
    prof_end(kProfExtract, st);
    return launches + 1;
}

__global__ void __launch_bounds__(kThreads)
outputs_kernel(int n, Workspace ws, int64_t *eta_num, int32_t *eta_den, int64_t *potential,
               int32_t *policy) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        JLS st = ws.jls[0][v];
        int i = ws.cid_of_root[~st.J];
        if (eta_num) eta_num[v] = ws.cyc_p[i];
        if (eta_den) eta_den[v] = ws.cyc_q[i];
        if (potential) potential[v] = ws.rec[v].V;
        if (policy) policy[v] = ws.pi[v];
    }
}

void launch_outputs(int n, Workspace ws, int64_t *eta_num, int32_t *eta_den, int64_t *potential,
                    int32_t *policy, cudaStream_t st) {
    int blocks = (n + kThreads - 1) / kThreads;
    if (blocks > 8192) blocks = 8192;
    prof_begin(kProfExtract, st);
    outputs_kernel<<<blocks, kThreads, 0, st>>>(n, ws, eta_num, eta_den, potential, policy);
    prof_end(kProfExtract, st);
}

}  // namespace ocm
