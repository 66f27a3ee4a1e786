// evaluate.cu -- evaluation of a policy (Alg. 1: MinMeanWeightCycle(G_pi) and
// the value propagation that follows it; Alg. 2: elimination*,
// cycleIdentification, reduce_min, setMinCycle, GpiPreprocess and
// valuePropagate*), re-designed as pointer jumping in one persistent kernel.
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
//           on its path).
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
//
// Execution: one cooperative launch (all CTAs co-resident) runs every phase;
// rounds are separated by a grid barrier whose waits are bounded (on expiry
// the kernel records kErrTimeout and returns).  Rounds are dense over the
// vertices (coalesced own-state access, no worklist atomics); a bitmap marks
// vertices that are finished and whose final state sits in both jump buffers,
// so they cost nothing in later rounds.  A round writes only the buffer it
// does not read; a vertex resolved in round k copies its final state into the
// other buffer in round k+1.
#include <climits>

#include "common.cuh"

namespace ocm {

constexpr long long kBarrierSpinLimit = 1LL << 24;   // x 64 ns sleeps: about a second

static __device__ __forceinline__ int load_volatile(const int *p) {
    return *reinterpret_cast<const volatile int *>(p);
}

// Grid-wide barrier for a cooperative launch.  Returns false (for the whole
// block) once any block's wait has exceeded its limit.
static __device__ bool grid_barrier(Ctrl *c, unsigned nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &c->bar_gen;
        const unsigned g = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(&c->bar_count, 1u) == nblocks - 1) {
            c->bar_count = 0;
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else {
            long long spins = 0;
            while (*gen == g) {
                if (++spins > kBarrierSpinLimit || (load_volatile(&c->err) & kErrTimeout)) {
                    atomicOr(&c->err, kErrTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Adds the block's sum of x to *dst with one atomic.
static __device__ __forceinline__ void block_count(int x, int *dst) {
    __shared__ int s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s_sum, x);
    __syncthreads();
    if (threadIdx.x == 0 && s_sum) atomicAdd(dst, s_sum);
}

constexpr int kRankTile = 2048;
constexpr int kU = 4;   // vertices per thread per pass of a jump round

__global__ void __launch_bounds__(kEvalThreads, 1)
evaluate_kernel(int n, long long N2, int max_detect, int max_value, Workspace ws) {
    __shared__ long long s_key[kRankTile];
    Ctrl *c = ws.ctrl;
    const unsigned nblocks = gridDim.x;
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    const int first = blockIdx.x * blockDim.x;

    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->pending[0] = c->pending[1] = c->pending[2] = 0;
        c->pendv[0] = c->pendv[1] = c->pendv[2] = 0;
        c->nrep = 0;
        c->best = 0;
    }
    if (!grid_barrier(c, nblocks)) return;

    // ------------------------------------------------------------ detect
    // Each thread advances kU vertices per pass (v = base + u*stride + tid) so
    // that their dependent loads (done word -> own state -> target state)
    // overlap instead of running one chain at a time.
    int r = 0;
    for (;; ++r) {
        const JM *in = ws.jm[r & 1];
        JM *out = ws.jm[(r + 1) & 1];
        int pend = 0;
        for (int base = first; base < n; base += kU * stride) {
            unsigned word[kU];
            bool act[kU];
            JM s[kU], t[kU];
            int ap[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int v = base + u * stride + threadIdx.x;
                const bool warp_live = v - lane < n;
                word[u] = (r > 0 && warp_live) ? ws.done[v >> 5] : 0u;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int v = base + u * stride + threadIdx.x;
                act[u] = v < n && !((word[u] >> lane) & 1u);
                if (act[u]) s[u] = (r == 0) ? JM{ws.succ[v], v} : in[v];
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int v = base + u * stride + threadIdx.x;
                if (act[u] && s[u].J >= 0) {
                    const int J = s[u].J;
                    t[u] = (r == 0) ? JM{ws.succ[J], J} : in[J];
                    ap[u] = (r == 0) ? -1 : ws.aprev[v];
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int v = base + u * stride + threadIdx.x;
                bool done = !act[u], is_root = false;
                if (act[u]) {
                    if (s[u].J < 0) {
                        out[v] = s[u];       // resolved last round: copy forward
                        done = true;
                    } else {
                        int root = -1;
                        if (t[u].J < 0) {
                            root = ~t[u].J;  // target resolved: it lies on v's path
                        } else if (r > 0 && t[u].M == ap[u]) {
                            root = t[u].M;   // smallest vertex of the cycle
                        } else {
                            // (round 0: J_0 = succ, M_0(v) = v, no test yet)
                            out[v] = JM{t[u].J, min(s[u].M, t[u].M)};
                            ws.aprev[v] = t[u].M;
                        }
                        if (root >= 0) {
                            out[v] = JM{~root, 0};
                            ws.rep[v] = root;
                            is_root = (root == v);
                        }
                        ++pend;
                    }
                }
                const unsigned bits = __ballot_sync(0xffffffffu, done);
                if (lane == 0 && v < n) ws.done[v >> 5] = bits;
                const int pos = warp_append(&c->nrep, is_root, lane);
                if (is_root) ws.cyc_root[pos] = v;
            }
        }
        block_count(pend, &c->pending[r % 3]);
        if (blockIdx.x == 0 && threadIdx.x == 0) c->pending[(r + 1) % 3] = 0;
        if (!grid_barrier(c, nblocks)) return;
        const int left = load_volatile(&c->pending[r % 3]);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            c->rounds_detect += 1;
            c->items_detect += left;
        }
        if (left == 0) break;
        if (r + 1 >= max_detect) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&c->err, kErrDetect);
            return;
        }
    }

    // ------------------------------------------------------------ values
    // init: roots are final; a vertex whose successor is a root is final too
    {
        int pend = 0;
        for (int base = first; base < n; base += stride) {
            const int v = base + threadIdx.x;
            bool fin = true;
            if (v < n) {
                int rv = ws.rep[v];
                JLS st;
                if (rv == v) {
                    st = JLS{~v, 0, 0};
                } else {
                    int s = ws.succ[v];
                    fin = (ws.rep[s] == s);
                    st = JLS{fin ? ~s : s, 1, (long long)ws.wpi[v]};
                }
                ws.jls[0][v] = st;
                if (fin) ws.jls[1][v] = st;
                pend += !fin;
            }
            unsigned bits = __ballot_sync(0xffffffffu, fin);
            if (lane == 0 && base + (int)(threadIdx.x & ~31u) < n) ws.done[v >> 5] = bits;
        }
        block_count(pend, &c->pendv[0]);
    }
    if (!grid_barrier(c, nblocks)) return;
    if (load_volatile(&c->pendv[0]) != 0) {
        for (int j = 1;; ++j) {
            const JLS *in = ws.jls[(j + 1) & 1];
            JLS *out = ws.jls[j & 1];
            int pend = 0;
            for (int base = first; base < n; base += kU * stride) {
                unsigned word[kU];
                bool act[kU];
                JLS s[kU], t[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int v = base + u * stride + threadIdx.x;
                    word[u] = (v - lane < n) ? ws.done[v >> 5] : ~0u;
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int v = base + u * stride + threadIdx.x;
                    act[u] = v < n && !((word[u] >> lane) & 1u);
                    if (act[u]) s[u] = in[v];
                }
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    if (act[u] && s[u].J >= 0) t[u] = in[s[u].J];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int v = base + u * stride + threadIdx.x;
                    bool done = !act[u];
                    if (act[u]) {
                        if (s[u].J < 0) {
                            out[v] = s[u];
                            done = true;
                        } else {
                            out[v] = JLS{t[u].J, s[u].len + t[u].len, s[u].S + t[u].S};
                            ++pend;
                        }
                    }
                    const unsigned bits = __ballot_sync(0xffffffffu, done);
                    if (lane == 0 && v < n) ws.done[v >> 5] = bits;
                }
            }
            block_count(pend, &c->pendv[j % 3]);
            if (blockIdx.x == 0 && threadIdx.x == 0) c->pendv[(j + 1) % 3] = 0;
            if (!grid_barrier(c, nblocks)) return;
            const int left = load_volatile(&c->pendv[j % 3]);
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                c->rounds_value += 1;
                c->items_value += left;
            }
            if (left == 0) break;
            if (j + 1 > max_value) {
                if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&c->err, kErrValue);
                return;
            }
        }
    }

    // ------------------------------------------------------------ cycles
    const int K = load_volatile(&c->nrep);
    for (int i = first + threadIdx.x; i < K; i += stride) {
        int root = ws.cyc_root[i];
        int x = ws.succ[root];
        JLS st = ws.jls[0][x];
        long long W = (long long)ws.wpi[root] + st.S;
        long long L = 1 + (long long)st.len;
        long long g = gcd_ll(W, L);
        long long p = W / g, q = L / g;
        ws.cyc_p[i] = p;
        ws.cyc_q[i] = (int)q;
        ws.cyc_L[i] = (int)L;
        ws.cyc_key[i] = mean_key(p, q, N2);
        ws.cid_of_root[root] = i;
    }
    if (!grid_barrier(c, nblocks)) return;
    for (int base = first; base < K; base += stride) {
        const int i = base + threadIdx.x;
        const long long key = i < K ? ws.cyc_key[i] : 0;
        int rank = 0;
        for (int t0 = 0; t0 < K; t0 += kRankTile) {
            int tn = min(kRankTile, K - t0);
            __syncthreads();
            for (int q = threadIdx.x; q < tn; q += blockDim.x) s_key[q] = ws.cyc_key[t0 + q];
            __syncthreads();
            for (int q = 0; q < tn; ++q) rank += (s_key[q] < key);
        }
        if (i < K) {
            ws.cyc_rank[i] = rank;
            unsigned long long packed = ((unsigned long long)(unsigned)rank << 32) |
                                        (unsigned)(INT_MAX - ws.cyc_root[i]);
            atomicMax(&c->best, packed);
        }
    }
    if (!grid_barrier(c, nblocks)) return;

    // ------------------------------------------------------- materialise
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->changed = 0;
        c->switched = 0;
    }
    for (int v = first + threadIdx.x; v < n; v += stride) {
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

// Co-resident CTAs of the evaluation kernel on the current device.
static int evaluate_grid() {
    static int cached_dev = -1, cached = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev == cached_dev && cached > 0) return cached;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, evaluate_kernel, kEvalThreads, 0) !=
            cudaSuccess || per_sm < 1)
        return 0;
    cached_dev = dev;
    cached = sms * per_sm;
    return cached;
}

// One policy evaluation = one cooperative launch; returns 1, or -1 on a
// launch failure.
int launch_evaluate(int n, long long N2, Workspace ws, int grid, cudaStream_t st) {
    (void)grid;
    int blocks = evaluate_grid();
    if (blocks <= 0) return -1;
    int need = (n + kEvalThreads - 1) / kEvalThreads;
    if (need < blocks) blocks = need;
    const int lg = ceil_log2(n);
    int max_detect = lg + 4;
    int max_value = lg + 3;
    void *args[] = {&n, &N2, &max_detect, &max_value, &ws};
    prof_begin(kProfEvaluate, st);
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)evaluate_kernel, dim3(blocks),
                                                dim3(kEvalThreads), args, 0, st);
    prof_end(kProfEvaluate, st);
    return e == cudaSuccess ? 1 : -1;
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
    const int K = load_volatile(&c->ncand);
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
    const int K = load_volatile(&c->ncand);
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
