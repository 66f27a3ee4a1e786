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
#include "grid_sync.cuh"

namespace ocm {


constexpr int kRankTile = 2048;
constexpr int kU = 4;   // vertices per thread per pass of a jump round

// Appends item to a block-local list (warp-aggregated shared-memory atomic).
static __device__ __forceinline__ void block_append(int *list, int *s_cnt, bool pred, int item,
                                                    int lane) {
    const unsigned mask = __ballot_sync(0xffffffffu, pred);
    int base = 0;
    if (mask) {
        const int leader = __ffs(mask) - 1;
        if (lane == leader) base = atomicAdd(s_cnt, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
    }
    if (pred) list[base + __popc(mask & ((1u << lane) - 1u))] = item;
}


constexpr int kRankDirectMax = 65536;   // all-pairs rank count up to this many cycles
constexpr int kRankSplitMin = 4096;     // from this many cycles the count is spread over all blocks
constexpr int kRankPairTile = 1024;     // keys per piece of the spread count

// Inclusive sum of x over the block (all threads call it; 1024 threads).
static __device__ __forceinline__ int block_inclusive_scan(int x, int *s_warp) {
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
    return x + (warp > 0 ? s_warp[warp - 1] : 0);
}

// Dense ranks of the K cycle keys (rank = number of distinct keys below) for
// policies with many cycles, where counting over all pairs would cost K^2: a
// stable least-significant-digit radix sort of (key, cycle) pairs with 8-bit
// digits across the cooperative grid, then a scan of the run starts of the
// sorted keys.  Block b owns a contiguous chunk of positions in every pass;
// per pass: per-block digit histograms, one exclusive scan in (digit, block)
// order by block 0, and a stable scatter (warps of a block in turn, lanes
// with equal digits ranked by a match mask).  A pass whose digit is the same
// for all keys leaves the order unchanged and is skipped.  Scratch: the
// detection jump states and worklists, which are dead at this point.
// Returns false if a grid barrier gave up.
static __device__ bool radix_ranks(int K, const Workspace &ws, Ctrl *c, unsigned nblocks) {
    __shared__ int s_off[256];
    __shared__ int s_warp[32];
    __shared__ int s_skip;
    unsigned long long *keyA = reinterpret_cast<unsigned long long *>(ws.cyc_key);
    unsigned long long *keyB = reinterpret_cast<unsigned long long *>(ws.jm[0]);
    int *idA = ws.list[1], *idB = ws.list[0];
    const int G = (int)gridDim.x;
    const int chunk = (K + G - 1) / G;
    const int c0 = min(K, (int)blockIdx.x * chunk), c1 = min(K, c0 + chunk);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (int)(blockDim.x >> 5);
    // order-preserving unsigned image of the signed keys; identity ids
    for (int i = c0 + (int)threadIdx.x; i < c1; i += blockDim.x) {
        keyA[i] ^= 0x8000000000000000ULL;
        idA[i] = i;
    }
    for (int pass = 0; pass < 8; ++pass) {
        const int sh = 8 * pass;
        // two histogram buffers by pass parity: the skip test of one pass may
        // still read its buffer while the next pass fills the other
        int *hist = ws.list[2] + (pass & 1) * 256 * G;
        if (threadIdx.x < 256) s_off[threadIdx.x] = 0;
        __syncthreads();
        for (int i = c0 + (int)threadIdx.x; i < c1; i += blockDim.x)
            atomicAdd(&s_off[(int)((keyA[i] >> sh) & 255u)], 1);
        __syncthreads();
        if (threadIdx.x < 256) hist[threadIdx.x * G + blockIdx.x] = s_off[threadIdx.x];
        if (!grid_barrier(c, nblocks)) return false;
        if (blockIdx.x == 0) {
            // exclusive scan of hist[0 .. 256 G) in place, per = entries per thread
            const int total = 256 * G;
            const int per = (total + (int)blockDim.x - 1) / (int)blockDim.x;
            const int b0 = min(total, (int)threadIdx.x * per), b1 = min(total, b0 + per);
            int sum = 0;
            for (int i = b0; i < b1; ++i) sum += hist[i];
            const int incl = block_inclusive_scan(sum, s_warp);
            int run = incl - sum;
            for (int i = b0; i < b1; ++i) {
                const int x = hist[i];
                hist[i] = run;
                run += x;
            }
        }
        if (!grid_barrier(c, nblocks)) return false;
        if (threadIdx.x == 0) s_skip = 0;
        __syncthreads();
        if (threadIdx.x < 256) {
            const int lo = hist[threadIdx.x * G];
            const int hi = threadIdx.x < 255 ? hist[(threadIdx.x + 1) * G] : K;
            if (hi - lo == K) s_skip = 1;
            s_off[threadIdx.x] = hist[threadIdx.x * G + blockIdx.x];
        }
        __syncthreads();
        if (s_skip) continue;   // the same decision in every block
        for (int t0 = c0; t0 < c1; t0 += blockDim.x) {
            const int i = t0 + (int)threadIdx.x;
            const bool valid = i < c1;
            const unsigned long long k = valid ? keyA[i] : 0ULL;
            const int id = valid ? idA[i] : 0;
            // lanes past the chunk get distinct dummy digits so they match nobody
            const int dg = valid ? (int)((k >> sh) & 255u) : 256 + lane;
            const unsigned peers = __match_any_sync(0xffffffffu, dg);
            const int r = __popc(peers & ((1u << lane) - 1u));
            const bool leader = r == 0;
            for (int wv = 0; wv < nwarps; ++wv) {
                int base = 0;
                if (warp == wv && valid) base = s_off[dg];
                __syncwarp();
                if (warp == wv && valid) {
                    keyB[base + r] = k;
                    idB[base + r] = id;
                    if (leader) s_off[dg] = base + __popc(peers);
                }
                __syncthreads();
            }
        }
        unsigned long long *tk = keyA;
        keyA = keyB;
        keyB = tk;
        int *ti = idA;
        idA = idB;
        idB = ti;
        if (!grid_barrier(c, nblocks)) return false;
    }
    if (!grid_barrier(c, nblocks)) return false;
    // dense ranks: rank at sorted position i = (run starts in [0, i]) - 1
    int *bsum = ws.list[2];
    int cnt = 0;
    for (int i = c0 + (int)threadIdx.x; i < c1; i += blockDim.x)
        cnt += (i == 0 || keyA[i] != keyA[i - 1]) ? 1 : 0;
    const int tot = block_inclusive_scan(cnt, s_warp);
    if (threadIdx.x == blockDim.x - 1) bsum[blockIdx.x] = tot;
    if (!grid_barrier(c, nblocks)) return false;
    if (threadIdx.x == 0) {
        int b = 0;
        for (int k = 0; k < (int)blockIdx.x; ++k) b += bsum[k];
        s_off[0] = b;
    }
    __syncthreads();
    int carry = s_off[0];
    for (int t0 = c0; t0 < c1; t0 += blockDim.x) {
        const int i = t0 + (int)threadIdx.x;
        const int f = (i < c1 && (i == 0 || keyA[i] != keyA[i - 1])) ? 1 : 0;
        const int incl = block_inclusive_scan(f, s_warp);
        if (i < c1) ws.cyc_rank[idA[i]] = carry + incl - 1;
        carry += s_warp[nwarps - 1];
        __syncthreads();
    }
    return grid_barrier(c, nblocks);
}

// The phases after every vertex has its final (~root, len, S) in jls[F]
// (and, for the cycle ratio, its path time in jt[F]) and the roots are listed
// in cyc_root[0, nrep): per-cycle means, exact keys and ranks, the best cycle
// (per graph for a batch), and the records {V, rank, q} the next sweep
// gathers.  Called by every thread of a cooperative evaluation kernel.
//
// LOCAL (the two-level evaluation): a vertex whose local path ends at an exit
// holds its state to that exit, completed on the fly (final_value).
template <bool RATIO, bool LOCAL = false>
static __device__ void evaluate_tail(int n, long long N2, int F, const Workspace &ws,
                                     const BatchState &bs, long long *s_key) {
    Ctrl *c = ws.ctrl;
    const unsigned nblocks = gridDim.x;
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    const int first = blockIdx.x * blockDim.x;
    constexpr bool ratio = RATIO;
    // frontier sweep: mark the records this pass changes?  (decided from the
    // last sweep's switch count before block 0 clears it below)
    const int fm = c->frontier;
    const bool mark = fm != 0 && c->iter > 0 &&
                      (fm == 2 || (long long)c->switched < ((long long)n >> kFrontierSwitchShift));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->dirty_on = mark ? 1 : 0;
        c->dirty_cnt = 0;
    }
    if (mark && blockIdx.x == 0) {
        const int words = ((n + kDirtyBlock - 1) / kDirtyBlock + 31) / 32;
        for (int i = threadIdx.x; i < words; i += blockDim.x) ws.rec_dirty_blk[i] = 0u;
    }
    // ------------------------------------------------------------ cycles
    // mean W/L, or for the cycle ratio W/T with T the cycle's transit time
    const int K = load_volatile(&c->nrep);
    int qmax = 0;
    for (int i = first + threadIdx.x; i < K; i += stride) {
        int root = ws.cyc_root[i];
        int x = ws.succ[root];
        JLS st = LOCAL ? final_value(ws.jls[0], n, x) : ws.jls[F][x];
        long long W = (long long)ws.wpi[root] + st.S;
        long long L = 1 + (long long)st.len;
        const long long Tc = ratio ? (long long)ws.tpi[root] + ws.jt[F][x] : L;
        long long g = gcd_ll(W, Tc);
        long long p = W / g, q = Tc / g;
        ws.cyc_p[i] = p;
        ws.cyc_q[i] = (int)q;
        ws.cyc_L[i] = (int)L;
        if (!ratio) ws.cyc_key[i] = mean_key(p, q, N2);
        ws.cyc_rank[i] = 0;   // summed into by the spread all-pairs count
        qmax = max(qmax, (int)q);
        ws.cid_of_root[root] = i;
    }
    if (ratio) {
        // the order keys need N2 >= (largest denominator)^2 to separate
        // distinct ratios; the current cycles' largest one keeps them small
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) qmax = max(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
        if (lane == 0 && qmax) atomicMax(&c->qmax, qmax);
    }
    if (!grid_barrier(c, nblocks)) return;
    if (ratio) {
        const long long qm = load_volatile(&c->qmax);
        const long long N2r = qm * qm;
        // |key| <= max|w| * N2r (every ratio is at most max|w| in size, t >= 1)
        if ((__int128)N2r * (__int128)(c->maxabsw + 1) >= ((__int128)1 << 62)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&c->err, kErrRatioKey);
            return;
        }
        for (int i = first + threadIdx.x; i < K; i += stride)
            ws.cyc_key[i] = mean_key(ws.cyc_p[i], ws.cyc_q[i], N2r);
        if (!grid_barrier(c, nblocks)) return;
    }
    if (K > kRankDirectMax && n >= 2 * 256 * (int)gridDim.x) {
        if (!radix_ranks(K, ws, c, nblocks)) return;
    } else if (K >= kRankSplitMin) {
        // all pairs, spread: (kEvalThreads cycles x kRankPairTile keys)
        // pieces over every block, each adding its count of smaller keys to
        // the cycle's rank (integer sums: the order of the adds is immaterial)
        const int nI = (K + kEvalThreads - 1) / kEvalThreads;
        const int nT = (K + kRankPairTile - 1) / kRankPairTile;
        for (int wi = blockIdx.x; wi < nI * nT; wi += gridDim.x) {
            const int t0 = (wi % nT) * kRankPairTile;
            const int tn = min(kRankPairTile, K - t0);
            __syncthreads();
            for (int q = threadIdx.x; q < tn; q += blockDim.x) s_key[q] = ws.cyc_key[t0 + q];
            __syncthreads();
            const int i = (wi / nT) * kEvalThreads + threadIdx.x;
            if (i < K) {
                const long long key = ws.cyc_key[i];
                int cnt = 0;
                for (int q = 0; q < tn; ++q) cnt += (s_key[q] < key);
                if (cnt) atomicAdd(&ws.cyc_rank[i], cnt);
            }
        }
        if (!grid_barrier(c, nblocks)) return;
    } else {
        // all pairs: rank(i) = number of cycle keys below key(i)
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
            if (i < K) ws.cyc_rank[i] = rank;
        }
    }
    for (int i = first + threadIdx.x; i < K; i += stride) {
        const int rank = ws.cyc_rank[i];
        const int root = ws.cyc_root[i];
        unsigned long long packed = ((unsigned long long)(unsigned)rank << 32) |
                                    (unsigned)(INT_MAX - root);
        atomicMax(&c->best, packed);
        // batched: Alg. 4's region-specific vote, one region per graph,
        // deterministic because the packed key is a total order
        if (bs.G) atomicMax(&bs.gbest[bs.gid[root]], packed);
    }
    if (!grid_barrier(c, nblocks)) return;

    // ------------------------------------------------------- materialise
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->changed = 0;
        c->switched = 0;
    }
    // (warp-uniform trip counts: a warp covers 32 consecutive vertices, one
    // word of the change bitmap, in each of its kMU slots; the slots' loads
    // are issued together, stage by stage)
    constexpr int kMU = 4;
    int changed = 0;
    for (int base0 = first + (int)threadIdx.x - lane; base0 < n; base0 += kMU * stride) {
        JLS st[kMU];
        bool ok[kMU];
#pragma unroll
        for (int u = 0; u < kMU; ++u) {
            const int v = base0 + u * stride + lane;
            ok[u] = v < n && !(bs.G && bs.gconv[bs.gid[v]]);
            if (ok[u]) st[u] = LOCAL ? ws.jls[0][v] : ws.jls[F][v];
        }
        if (LOCAL) {   // final_value: a leaf's steps, then the exit's value
#pragma unroll
            for (int u = 0; u < kMU; ++u) {
                if (!ok[u]) continue;
                for (int k = 0; k < 2 && st[u].J >= 0; ++k) {
                    const JLS nx = ws.jls[0][st[u].J];
                    st[u] = JLS{nx.J, st[u].len + nx.len, st[u].S + nx.S};
                }
            }
            JLS xf[kMU];
#pragma unroll
            for (int u = 0; u < kMU; ++u)
                if (ok[u] && ~st[u].J >= n) xf[u] = ws.jls[0][~st[u].J - n];
#pragma unroll
            for (int u = 0; u < kMU; ++u)
                if (ok[u] && ~st[u].J >= n)
                    st[u] = JLS{xf[u].J, st[u].len + xf[u].len, st[u].S + xf[u].S};
        }
        int ci[kMU];
#pragma unroll
        for (int u = 0; u < kMU; ++u) ci[u] = ok[u] ? ws.cid_of_root[~st[u].J] : 0;
#pragma unroll
        for (int u = 0; u < kMU; ++u) {
            const int v = base0 + u * stride + lane;
            bool dirty = false;
            if (ok[u]) {
                const int i = ci[u];
                const long long p = ws.cyc_p[i];
                const int q = ws.cyc_q[i];
                Rec rec;
                const long long T = ratio ? ws.jt[F][v] : (long long)st[u].len;
                rec.V = (long long)q * st[u].S - p * T;
                rec.rank = ws.cyc_rank[i];
                rec.q = q;
                if (mark) {
                    const Rec old = ws.rec[v];
                    dirty = old.V != rec.V || old.rank != rec.rank || old.q != rec.q ||
                            (ratio && ws.recp[v] != p);
                }
                ws.rec[v] = rec;
                if (ratio) ws.recp[v] = p;
            }
            const int base = base0 + u * stride;
            if (mark && base < n) {
                const unsigned m = __ballot_sync(0xffffffffu, dirty);
                if (lane == 0) {
                    ws.rec_dirty[base >> 5] = m;
                    changed += __popc(m);
                    if (m) {   // (a plain read first: the 32 warps of a block share the bit)
                        const int blk = base / kDirtyBlock;
                        const unsigned bit = 1u << (blk & 31);
                        if (!(ws.rec_dirty_blk[blk >> 5] & bit))
                            atomicOr(&ws.rec_dirty_blk[blk >> 5], bit);
                    }
                }
            }
        }
    }
    if (mark) {
        __shared__ int s_changed;
        if (threadIdx.x == 0) s_changed = 0;
        __syncthreads();
        if (lane == 0 && changed) atomicAdd(&s_changed, changed);
        __syncthreads();
        if (threadIdx.x == 0 && s_changed)
            atomicAdd(reinterpret_cast<unsigned long long *>(&c->dirty_cnt),
                      (unsigned long long)s_changed);
        // the blocks of kClassifyBlock vertices whose edges reach a block with
        // a changed record (by the initial pass's range of target blocks)
        if (!grid_barrier(c, nblocks)) return;
        const int nb = (n + kClassifyBlock - 1) / kClassifyBlock;
        for (int base = first + (int)threadIdx.x - lane; base < nb; base += stride) {
            const int i = base + lane;
            bool need = false;
            if (i < nb) {
                const int2 rg = ws.blk_tgt[i];
                need = rg.x > rg.y || (rg.y >> 5) - (rg.x >> 5) >= kFrontierRangeWords;
                for (int wd = rg.x >> 5; !need && rg.x <= rg.y && wd <= (rg.y >> 5); ++wd) {
                    unsigned bits = ws.rec_dirty_blk[wd];
                    if (wd == (rg.x >> 5)) bits &= ~0u << (rg.x & 31);
                    if (wd == (rg.y >> 5)) bits &= ~0u >> (31 - (rg.y & 31));
                    need = bits != 0u;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, need);
            if (lane == 0) ws.need_blk[base >> 5] = m;
        }
    }
}

constexpr int kMinMask = 0x7fffffff;

// RATIO: optimal cycle ratio (transit times carried through values and
// cycles); a separate instance so that the mean keeps its register budget.
template <bool RATIO>
__global__ void __launch_bounds__(kEvalThreads, 1)
evaluate_kernel(int n, long long N2, int max_detect, int max_value, int stall_test, Workspace ws,
                BatchState bs) {
    __shared__ long long s_key[kRankTile];
    __shared__ int s_cnt;
    grid_sync_start();
    Ctrl *c = ws.ctrl;
    // vertices whose sw_iter equals this index switched in the last sweep
    const int eval_index = c->iter;
    const unsigned nblocks = gridDim.x;
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    const int first = blockIdx.x * blockDim.x;
    // every block owns a contiguous vertex range and keeps its worklist of
    // unfinished vertices inside the same range of the two list buffers
    const int R = (n + (int)gridDim.x - 1) / (int)gridDim.x;
    const int lo = min((int)blockIdx.x * R, n), hi = min(lo + R, n);
    int *LA = ws.list[0] + lo, *LB = ws.list[1] + lo;

    constexpr bool ratio = RATIO;   // optimal cycle ratio: times ride along
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->nrep = 0;
        c->best = 0;
        c->qmax = 0;
    }
    for (int g = first + threadIdx.x; g < bs.G; g += stride) bs.gbest[g] = 0;
    if (threadIdx.x == 0) s_cnt = 0;
    // No grid barrier is needed here: the counters reset above are first
    // used after the barrier that ends detection round 0 (round 0 resolves
    // nothing), and gbest only at the end.
    __syncthreads();
    // (test only: wait for one block more than exists, so the wait expires)
    if (stall_test && !grid_barrier(c, nblocks + 1u)) return;

    // ------------------------------------------------------------ detect
    // State: unresolved {J >= 0, M | dirty << 31}; resolved {~root, dirty}.
    // "dirty" ORs, over the same windows as M, whether a vertex switched in
    // the sweep before this evaluation; at resolution it covers v's whole
    // path and cycle, so a clean vertex keeps last evaluation's path sums.
    int cnt = hi - lo;
    int r = 0;
    for (;; ++r) {
        const JM *in = ws.jm[r & 1];
        JM *out = ws.jm[(r + 1) & 1];
        int *lin = (r & 1) ? LB : LA;
        int *lout = (r & 1) ? LA : LB;
        int pend = 0, kept = 0;
        for (int i0 = 0; i0 < cnt; i0 += kU * blockDim.x) {
            int item[kU];
            JM s[kU], t[kU];
            int ap[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int i = i0 + u * blockDim.x + threadIdx.x;
                item[u] = INT_MIN;
                if (i < cnt) {
                    item[u] = (r == 0) ? lo + i : lin[i];
                    // batched: vertices of converged graphs keep everything
                    if (r == 0 && bs.G && bs.gconv[bs.gid[lo + i]]) item[u] = INT_MIN;
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int it = item[u];
                if (it == INT_MIN) continue;
                const int v = it < 0 ? ~it : it;
                if (r == 0) {
                    s[u] = JM{ws.succ[v], v | ((ws.sw_iter[v] == eval_index) ? INT_MIN : 0)};
                    ap[u] = -1;
                } else {
                    s[u] = in[v];
                    ap[u] = it >= 0 ? ws.aprev[v] : 0;
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int it = item[u];
                if (it == INT_MIN || it < 0) continue;
                const int J = s[u].J;
                t[u] = (r == 0) ? JM{ws.succ[J], J | ((ws.sw_iter[J] == eval_index) ? INT_MIN : 0)}
                                : in[J];
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int it = item[u];
                bool keep = false, resolved = false, is_root = false;
                int v = 0;
                if (it != INT_MIN) {
                    v = it < 0 ? ~it : it;
                    if (it < 0) {
                        out[v] = s[u];        // resolved last round: copy forward
                    } else {
                        const int sdirty = (int)((unsigned)s[u].M >> 31);
                        int root = -1, dirty = 0;
                        if (t[u].J < 0) {
                            root = ~t[u].J;   // target resolved: it lies on v's path
                            dirty = sdirty | t[u].M;
                        } else if (r > 0 && (t[u].M & kMinMask) == ap[u]) {
                            root = ap[u];     // smallest vertex of the cycle
                            dirty = sdirty | (int)((unsigned)t[u].M >> 31);
                        } else {
                            // (round 0: J_0 = succ, M_0(v) = v, no test yet)
                            const int m = min(s[u].M & kMinMask, t[u].M & kMinMask);
                            out[v] = JM{t[u].J, m | ((s[u].M | t[u].M) & INT_MIN)};
                            ws.aprev[v] = t[u].M & kMinMask;
                            keep = true;
                        }
                        if (root >= 0) {
                            out[v] = JM{~root, dirty};
                            ws.rep[v] = root;
                            resolved = true;
                            is_root = (root == v);
                        }
                        ++pend;
                    }
                }
                block_append(lout, &s_cnt, keep || resolved, keep ? v : ~v, lane);
                kept += keep;
                const int pos = warp_append(&c->nrep, is_root, lane);
                if (is_root) ws.cyc_root[pos] = v;
            }
        }
        __syncthreads();
        cnt = s_cnt;
        __syncthreads();
        if (threadIdx.x == 0) s_cnt = 0;
        bool ok;
        int still;   // vertices still unresolved after this round
        const int left = grid_sum2_barrier(c, nblocks, pend, kept, &still, &ok);
        if (!ok) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            c->rounds_detect += 1;
            c->items_detect += left;
        }
        if (left == 0) break;
        if (still == 0) {
            // all resolved: instead of a round that only copies the states
            // resolved in this one into the other buffer, each block copies
            // its own (the list it just built) -- nothing reads another
            // block's jump state before the kernel ends
            for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                const int v = ~lout[i];
                ws.jm[r & 1][v] = out[v];
            }
            __syncthreads();
            break;
        }
        if (r + 1 >= max_detect) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&c->err, kErrDetect);
            return;
        }
    }

    // ------------------------------------------------------------ values
    // Only dirty vertices are recomputed: a clean vertex's path and cycle are
    // those of the last evaluation, whose final (root, len, S) is still in
    // both buffers.  Dirty roots are final at once, as is a dirty vertex whose
    // successor is a root; the rest jump until they meet a final state.
    cnt = 0;
    int left0 = 0;
    {
        int pend = 0;
        for (int i0 = 0; i0 < hi - lo; i0 += blockDim.x) {
            const int i = i0 + threadIdx.x;
            bool keep = false;
            int v = lo + i;
            if (i < hi - lo && !(bs.G && bs.gconv[bs.gid[v]])) {
                const JM d = ws.jm[0][v];
                if (d.M) {
                    const int root = ~d.J;
                    JLS st;
                    long long T = 0;
                    bool fin = true;
                    if (root == v) {
                        st = JLS{~v, 0, 0};
                    } else {
                        const int sv = ws.succ[v];
                        fin = (ws.rep[sv] == sv);
                        st = JLS{fin ? ~sv : sv, 1, (long long)ws.wpi[v]};
                        if (ratio) T = ws.tpi[v];
                    }
                    ws.jls[0][v] = st;
                    if (fin) ws.jls[1][v] = st;
                    if (ratio) {
                        ws.jt[0][v] = T;
                        if (fin) ws.jt[1][v] = T;
                    }
                    keep = !fin;
                }
            }
            block_append(LA, &s_cnt, keep, v, lane);
            pend += keep;
        }
        __syncthreads();
        cnt = s_cnt;
        __syncthreads();
        if (threadIdx.x == 0) s_cnt = 0;
        bool ok;
        left0 = grid_sum_barrier(c, nblocks, pend, &ok);
        if (!ok) return;
    }
    int F = 0;   // a value buffer holding every final state (both, once copied forward)
    if (left0 != 0) {
        for (int j = 1;; ++j) {
            const JLS *in = ws.jls[(j + 1) & 1];
            JLS *out = ws.jls[j & 1];
            // cycle ratio: the transit time of the path to J, jumped alongside
            const long long *tin = ws.jt[(j + 1) & 1];
            long long *tout = ws.jt[j & 1];
            int *lin = (j & 1) ? LA : LB;
            int *lout = (j & 1) ? LB : LA;
            int pend = 0, kept = 0;
            for (int i0 = 0; i0 < cnt; i0 += kU * blockDim.x) {
                int item[kU];
                JLS s[kU], t[kU];
                long long ts[kU], tt[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int i = i0 + u * blockDim.x + threadIdx.x;
                    item[u] = i < cnt ? lin[i] : INT_MIN;
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int it = item[u];
                    if (it != INT_MIN) {
                        s[u] = in[it < 0 ? ~it : it];
                        if (ratio) ts[u] = tin[it < 0 ? ~it : it];
                    }
                }
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    if (item[u] != INT_MIN && item[u] >= 0) {
                        t[u] = in[s[u].J];
                        if (ratio) tt[u] = tin[s[u].J];
                    }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int it = item[u];
                    bool keep = false, fin = false;
                    int v = 0;
                    if (it != INT_MIN) {
                        v = it < 0 ? ~it : it;
                        if (it < 0) {
                            out[v] = s[u];    // final last round: copy forward
                            if (ratio) tout[v] = ts[u];
                        } else {
                            const JLS nu{t[u].J, s[u].len + t[u].len, s[u].S + t[u].S};
                            out[v] = nu;
                            if (ratio) tout[v] = ts[u] + tt[u];
                            fin = nu.J < 0;
                            keep = !fin;
                            ++pend;
                        }
                    }
                    block_append(lout, &s_cnt, keep || fin, keep ? v : ~v, lane);
                    kept += keep;
                }
            }
            __syncthreads();
            cnt = s_cnt;
            __syncthreads();
            if (threadIdx.x == 0) s_cnt = 0;
            bool ok;
            int still;
            const int left = grid_sum2_barrier(c, nblocks, pend, kept, &still, &ok);
            if (!ok) return;
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                c->rounds_value += 1;
                c->items_value += left;
            }
            if (left == 0) break;
            if (still == 0) {
                // all final: the phases below read buffer F, which holds
                // every final state; each block copies the states its
                // vertices reached in this round into the other buffer
                // (read by no one before the kernel ends)
                F = j & 1;
                for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                    const int v = ~lout[i];
                    ws.jls[(j + 1) & 1][v] = out[v];
                    if (ratio) ws.jt[(j + 1) & 1][v] = tout[v];
                }
                break;
            }
            if (j + 1 > max_value) {
                if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&c->err, kErrValue);
                return;
            }
        }
    }

    evaluate_tail<RATIO>(n, N2, F, ws, bs, s_key);
}

static int ceil_log2(long long x) {
    int k = 0;
    while ((1LL << k) < x) ++k;
    return k;
}

// Co-resident CTAs of the evaluation kernel (mean or ratio instance) on the
// current device.
template <bool RATIO>
static int evaluate_grid() {
    static int cached_dev = -1, cached = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev == cached_dev && cached > 0) return cached;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, evaluate_kernel<RATIO>,
                                                      kEvalThreads, 0) != cudaSuccess ||
        per_sm < 1)
        return 0;
    cached_dev = dev;
    cached = sms * per_sm;
    return cached;
}

int prepare_evaluate(bool ratio) {
    return (ratio ? evaluate_grid<true>() : evaluate_grid<false>()) > 0 ? 0 : -1;
}

__global__ void __launch_bounds__(kEvalThreads, 1)
evaluate_local_kernel(int n, long long N2, int max_local, int max_node, int stall_test,
                      int nwords, Workspace ws, BatchState bs);
constexpr int kLocalBitmapWords = 40960;   // 160 KB: the bitmaps of ranges up to 436,906 vertices
// chunked local pass: vertices per chunk, and its two shared-memory buffers of
// 16-byte packed states
constexpr int kLocalChunkPerThread = 4;
constexpr int kLocalChunk = kLocalChunkPerThread * kEvalThreads;
constexpr int kPackedStateBytes = 16;
constexpr int kLocalChunkBytes = 2 * kLocalChunk * kPackedStateBytes;
static_assert(kLocalChunkBytes <= kLocalBitmapWords * 4, "chunk buffers within the opt-in size");
__global__ void __launch_bounds__(kEvalThreads, 1)
local_chunk_kernel(int n, int max_local, Workspace ws);
int evaluate_local_blocks(int n);

// One policy evaluation = one cooperative launch (the two-level form: the
// chunked local pass first, then the cooperative launch); returns the number
// of launches, or -1 on a launch failure.  local: the two-level evaluation
// (single graphs without transit times only).
int launch_evaluate(int n, long long N2, Workspace ws, int stall_test, BatchState bs,
                    cudaStream_t st, bool local, bool no_bitmap) {
    const bool ratio = ws.transit != nullptr;
    if (local && !ratio && bs.G == 0) {
        const int blocks = evaluate_local_blocks(n);
        if (blocks <= 0) return -1;
        const int R = (n + blocks - 1) / blocks;
        const int words = 3 * ((R + 31) / 32);   // two bitmaps and the prefix counts
        const int nwords = (words <= kLocalBitmapWords && !no_bitmap) ? words : 0;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(blocks);
        cfg.blockDim = dim3(kEvalThreads);
        cfg.dynamicSmemBytes = (size_t)nwords * 4;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        prof_begin(kProfEvaluate, st);
        // (a kernel of its own: the cooperative kernel's register budget would
        // spill the pass's state; it returns at once when the pass is off)
        local_chunk_kernel<<<blocks, kEvalThreads, kLocalChunkBytes, st>>>(n, ceil_log2(R) + 4, ws);
        const cudaError_t e0 = cudaGetLastError();
        const cudaError_t e = cudaLaunchKernelEx(&cfg, evaluate_local_kernel, n, N2,
                                                 ceil_log2(R) + 4, ceil_log2(n) + 4, stall_test,
                                                 nwords, ws, bs);
        prof_end(kProfEvaluate, st);
        return (e0 == cudaSuccess && e == cudaSuccess) ? 2 : -1;
    }
    int blocks = ratio ? evaluate_grid<true>() : evaluate_grid<false>();
    if (blocks <= 0) return -1;
    int need = (n + kEvalThreads - 1) / kEvalThreads;
    if (need < blocks) blocks = need;
    const int lg = ceil_log2(n);
    int max_detect = lg + 4;
    int max_value = lg + 3;
    // cooperative (all blocks co-resident, the grid barriers rely on it); the
    // launch attribute form is also what a CUDA graph kernel node records
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kEvalThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    prof_begin(kProfEvaluate, st);
    cudaError_t e =
        ratio ? cudaLaunchKernelEx(&cfg, evaluate_kernel<true>, n, N2, max_detect, max_value,
                                   stall_test, ws, bs)
              : cudaLaunchKernelEx(&cfg, evaluate_kernel<false>, n, N2, max_detect, max_value,
                                   stall_test, ws, bs);
    prof_end(kProfEvaluate, st);
    return e == cudaSuccess ? 1 : -1;
}

// --------------------------------------------------------------- extract --
// Appends item to a global list with one atomic per block (all threads of the
// block call it; the order within the list is immaterial).
static __device__ __forceinline__ void block_append_global(int *list, int *counter, bool pred,
                                                           int item, int lane) {
    __shared__ int s_cnt, s_base;
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

// Critical cycle of root r* (length L*): its vertices are exactly the v with
// root(v) = r*, len(v) < L* and succ^{L*}(v) = v; v sits at position
// (L* - len(v)) mod L* counted from r*.  succ^{L*} is evaluated for all
// candidates at once by binary lifting over the bits of L* (the candidate set
// is closed under succ, so the jump tables never leave it).
//
// Candidates are also restricted to the vertices at the end of a policy path
// of two edges (a vertex of a cycle is: its cycle predecessor has one too),
// marked in two passes over succ (A: has a predecessor, B: has a predecessor
// in A).  The set stays closed under succ (v in B makes succ(v)'s predecessor
// v in A) and loses the policy tree's leaves and their successors that no
// other vertex reaches, about half of a random policy graph.  Bitmaps: the
// frontier sweep's change bitmap and the spare done bitmap, both free once
// the loop has ended.
//
// After the two-level evaluation the cycle can be walked instead, segment by
// segment (extract_walk_kernel): from r*, a vertex's local state names the exit
// its path leaves its block range by (or r* itself, for the vertices of r*'s
// range that reach it first), so one thread follows the cycle from exit to
// exit, noting each segment's first vertex, length and position, and the
// block's threads then walk the segments at once.  It gives up (and the
// lifting runs) when the cycle has more than kWalkSegs segments or a segment
// more than kWalkSegLen vertices; the lifting kernels return at once when it
// succeeded.
constexpr int kWalkSegs = 1024;
constexpr int kWalkSegLen = 4096;

__global__ void __launch_bounds__(1024)
extract_walk_kernel(int n, int R, Workspace ws, int *cycle_out) {
    __shared__ int s_first[kWalkSegs], s_pos[kWalkSegs], s_len[kWalkSegs];
    __shared__ int s_k, s_ok;
    Ctrl *c = ws.ctrl;
    const int r = c->res_root, L = c->res_len;
    if (threadIdx.x == 0) {
        int ok = 1, k = 0, pos = 1;
        int y = ws.succ[r];
        while (y != r) {
            if (k >= kWalkSegs || y < 0 || y >= n) {
                ok = 0;
                break;
            }
            const int lo = (y / R) * R, hi = min(lo + R, n);
            const int sy = ws.succ[y];
            int cnt, next;
            if (sy < lo || sy >= hi) {   // y is an exit (its state is its value)
                cnt = 1;
                next = sy;
            } else {
                const JLS st = local_state(ws.jls[0], y);
                const int tag = ~st.J;
                if (tag == r) {            // y's path reaches r* inside the range
                    cnt = st.len;
                    next = r;
                } else if (tag >= n && tag - n < n) {   // ... or leaves it by an exit
                    cnt = st.len + 1;
                    next = ws.succ[tag - n];
                } else {
                    ok = 0;
                    break;
                }
            }
            if (cnt < 1 || cnt > kWalkSegLen || pos + cnt > L) {
                ok = 0;
                break;
            }
            s_first[k] = y;
            s_pos[k] = pos;
            s_len[k] = cnt;
            pos += cnt;
            ++k;
            y = next;
        }
        s_k = k;
        s_ok = ok && pos == L;
    }
    __syncthreads();
    if (!s_ok) return;
    if (threadIdx.x == 0) cycle_out[0] = ws.pi[r];
    for (int j = threadIdx.x; j < s_k; j += blockDim.x) {
        int v = s_first[j];
        const int p = s_pos[j];
        for (int q = 0; q < s_len[j]; ++q) {
            cycle_out[p + q] = ws.pi[v];
            v = ws.succ[v];
        }
    }
    if (threadIdx.x == 0) {
        c->cnt[0] = L;
        c->walk_ok = 1;
    }
}

__global__ void __launch_bounds__(kThreads) extract_clear_kernel(int words, Workspace ws) {
    if (load_volatile(&ws.ctrl->walk_ok)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x) {
        ws.rec_dirty[i] = 0u;
        ws.done[i] = 0u;
    }
}

// to[succ(v)] for every v (from == nullptr) or every v marked in from.
__global__ void __launch_bounds__(kThreads)
extract_pred_kernel(int n, const unsigned *from, unsigned *to, Workspace ws) {
    if (load_volatile(&ws.ctrl->walk_ok)) return;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (from && !((from[v >> 5] >> (v & 31)) & 1u)) continue;
        const int t = ws.succ[v];
        atomicOr(&to[t >> 5], 1u << (t & 31));
    }
}

__global__ void __launch_bounds__(kThreads)
extract_candidates_kernel(int n, Workspace ws) {
    Ctrl *c = ws.ctrl;
    if (load_volatile(&c->walk_ok)) return;   // (no candidates: the rounds have nothing to do)
    const int root = c->res_root, L = c->res_len;
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    int *cur = ws.aprev;
    for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const int v = base + threadIdx.x;
        bool cand = false;
        if (v < n) {
            const JLS st = final_value(ws.jls[0], n, v);
            cand = (~st.J == root) && st.len < L && ((ws.done[v >> 5] >> (v & 31)) & 1u);
            if (cand) cur[v] = v;
        }
        block_append_global(ws.list[0], &c->ncand, cand, v, lane);
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
extract_scatter_kernel(int n, Workspace ws, int *cycle_out) {
    Ctrl *c = ws.ctrl;
    const int K = load_volatile(&c->ncand);
    const int L = c->res_len;
    const int stride = gridDim.x * blockDim.x;
    int found = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += stride) {
        int v = ws.list[0][i];
        if (ws.aprev[v] == v) {
            int len = final_value(ws.jls[0], n, v).len;
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
    ws.ctrl->walk_ok = 0;
}

// Extracts the critical cycle (root and length already in ctrl->res_*);
// returns the number of kernel launches.  local_R: the block range size of
// the two-level evaluation the loop used (0: the one-level evaluation, no
// segment walk).
int launch_extract(int n, int Lstar, Workspace ws, int *cycle_out, int grid, int local_R,
                   cudaStream_t st) {
    prof_begin(kProfExtract, st);
    extract_reset_kernel<<<1, 1, 0, st>>>(ws);
    int walk = 0;
    if (local_R > 0) {
        extract_walk_kernel<<<1, 1024, 0, st>>>(n, local_R, ws, cycle_out);
        walk = 1;
    }
    extract_clear_kernel<<<grid, kThreads, 0, st>>>((n + 31) / 32, ws);
    extract_pred_kernel<<<grid, kThreads, 0, st>>>(n, nullptr, ws.rec_dirty, ws);
    extract_pred_kernel<<<grid, kThreads, 0, st>>>(n, ws.rec_dirty, ws.done, ws);
    extract_candidates_kernel<<<grid, kThreads, 0, st>>>(n, ws);
    int launches = 5 + walk;
    int bits = 0;
    while ((1LL << bits) <= Lstar) ++bits;
    for (int b = 0; b < bits; ++b, ++launches) extract_round_kernel<<<grid, kThreads, 0, st>>>(b, ws);
    extract_scatter_kernel<<<grid, kThreads, 0, st>>>(n, ws, cycle_out);
    prof_end(kProfExtract, st);
    return launches + 1;
}

__global__ void __launch_bounds__(kThreads)
outputs_kernel(int n, Workspace ws, int64_t *eta_num, int32_t *eta_den, int64_t *potential,
               int32_t *policy) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const JLS st = final_value(ws.jls[0], n, v);
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

namespace ocm {

// ---------------------------------------------------------------------------
// Two-level evaluation, for policy graphs whose edges mostly stay inside the
// contiguous vertex range a block of the cooperative grid owns (graphs with
// locality, like the synthetic locality graph, where a policy path runs for
// tens of steps inside a range before it leaves it).  Same results as
// evaluate_kernel (root = smallest vertex of the cycle, (len, S) to its first
// occurrence, the same records), computed in fewer jump rounds:
//   local:  every block runs detection and value propagation on its own range
//           with block barriers only, a vertex whose successor lies outside
//           the range (an "exit") being terminal: each vertex ends with the
//           root of a cycle inside the range, or with the exit its path
//           leaves by, the path's length and weight to it, and the smallest
//           vertex on the way.  By default a kernel of its own does it chunk
//           by chunk from the top of the range down (local_chunked: one
//           streaming pass when the paths climb, as on the locality graph);
//           a range with a cycle of its own, and every range once paths that
//           go back dominate, take the jump rounds of local_onepass or the
//           two-pass local_phase inside the cooperative kernel;
//   nodes:  the exits form a functional graph of their own (exit x -> the
//           exit that succ(x)'s local path ends at, with the segment's length,
//           weight and smallest vertex); detection by window minima on it
//           finds the roots of the cycles that cross ranges (the smallest
//           segment minimum on the node cycle is the cycle's smallest vertex);
//   fix:    the vertices of such a root's range whose local path ends at the
//           root's former exit repeat their value jumping, spread over the
//           whole grid, with the root as one more terminal, so that every path
//           reaching it stops at its first occurrence (with many such roots,
//           the blocks holding one repeat their whole local phase instead);
//   values: (len, S) of every exit to its root by jumping on the node graph;
//   expand: each vertex adds its local part to its exit's value where it is
//           read (final_value), a leaf of local_onepass first following its
//           one or two steps to a vertex with a state of its own
//           (local_state).
// The local rounds are O(log) of the path length inside a range instead of
// the whole depth and cycle length, and need no grid barrier.
// ---------------------------------------------------------------------------

// The node graph is kept in dense node order (node i is the exit list[2][i]):
// the exits' node indices, by vertex, and the detection buffers live in the
// cycle-ratio buffers, which the two-level evaluation (the mean only) does not
// use; the value buffers in the 16-byte scratch and the second value buffer
// (dead once the root fix is done).
constexpr int kNU = 2;   // nodes per thread per pass of a node round

static __device__ __forceinline__ int *node_index(const Workspace &ws) {
    return reinterpret_cast<int *>(ws.recp);
}

static __device__ __forceinline__ int block_sum_int(int x, int *s_red) {
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

// The local phase of block range [lo, hi).  Detection states: unresolved
// {J, window minimum}, resolved {~tag, aux} with tag = a root (< n) or n + x
// for exit x, aux = the smallest vertex on the path to the exit (exits: none,
// INT_MAX).  Value states {~tag, len, S} once final.  Both jump buffers hold
// every final state on return, rep[v] = tag.  rerun: vertices with rep[v] == v
// (roots) are terminals too and no root is listed again.  Returns false on an
// error (recorded in the control block).
static __device__ bool local_phase(int lo, int hi, int n, bool rerun, bool list_exits,
                                   int max_rounds, const Workspace &ws, int *LA, int *LB,
                                   int *s_cnt, int *s_red, int *work_total) {
    Ctrl *c = ws.ctrl;
    const int lane = threadIdx.x & 31;
    const int W = blockDim.x;
    const int pad = (W - ((hi - lo) % W)) % W;   // uniform trip counts for the warp votes
    for (int v = lo + (int)threadIdx.x; v < hi + pad; v += W) {
        bool is_exit = false;
        if (v < hi) {
            const int sv = ws.succ[v];
            is_exit = sv < lo || sv >= hi;
            if (rerun && ws.rep[v] == v) {
                const JM t{~v, 0};
                ws.jm[0][v] = t;
                ws.jm[1][v] = t;
                is_exit = false;
            } else if (is_exit) {
                const JM t{~(n + v), INT_MAX};
                ws.jm[0][v] = t;
                ws.jm[1][v] = t;
                ws.rep[v] = n + v;
            } else {
                ws.jm[0][v] = JM{sv, v};
            }
        }
        if (list_exits) {   // the node list: every exit once
            const int pos = warp_append(&c->node_cnt, is_exit, lane);
            if (is_exit) {
                ws.list[2][pos] = v;
                node_index(ws)[v] = pos;
            }
        }
    }
    __syncthreads();
    int work = 0;
    // ---- detection
    int cnt = hi - lo;
    for (int r = 0;; ++r) {
        const JM *in = ws.jm[r & 1];
        JM *out = ws.jm[(r + 1) & 1];
        const int *lin = (r & 1) ? LB : LA;
        int *lout = (r & 1) ? LA : LB;
        int done_work = 0, kept = 0;
        for (int i0 = 0; i0 < cnt; i0 += kU * W) {
            int item[kU], ap[kU];
            JM s[kU], t[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int i = i0 + u * W + (int)threadIdx.x;
                item[u] = i < cnt ? ((r == 0) ? lo + i : lin[i]) : INT_MIN;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int it = item[u];
                if (it == INT_MIN) continue;
                const int v = it < 0 ? ~it : it;
                s[u] = in[v];
                ap[u] = (r > 0 && it >= 0) ? ws.aprev[v] : 0;
                if (r == 0 && s[u].J < 0) item[u] = INT_MIN;   // a terminal
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (item[u] != INT_MIN && item[u] >= 0) t[u] = in[s[u].J];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int it = item[u];
                bool keep = false, resolved = false, is_root = false;
                int v = 0;
                if (it != INT_MIN) {
                    v = it < 0 ? ~it : it;
                    if (it < 0) {
                        out[v] = s[u];        // resolved last round: copy forward
                    } else {
                        int tag = -1, aux = 0;
                        if (t[u].J < 0) {
                            tag = ~t[u].J;    // the target is finished: v's path reaches it
                            aux = tag >= n ? min(s[u].M, t[u].M) : 0;
                        } else if (r > 0 && t[u].M == ap[u]) {
                            tag = ap[u];      // a cycle inside the range: its smallest vertex
                        } else {
                            out[v] = JM{t[u].J, min(s[u].M, t[u].M)};
                            ws.aprev[v] = t[u].M;
                            keep = true;
                        }
                        if (tag >= 0) {
                            out[v] = JM{~tag, aux};
                            ws.rep[v] = tag;
                            resolved = true;
                            is_root = !rerun && tag == v;
                        }
                        ++done_work;
                    }
                }
                block_append(lout, s_cnt, keep || resolved, keep ? v : ~v, lane);
                kept += keep;
                const int pos = warp_append(&c->nrep, is_root, lane);
                if (is_root) ws.cyc_root[pos] = v;
            }
        }
        __syncthreads();
        cnt = *s_cnt;
        const int left = block_sum_int(done_work, s_red);
        const int still = block_sum_int(kept, s_red);
        if (threadIdx.x == 0) *s_cnt = 0;
        __syncthreads();
        work += left;
        if (left == 0) break;
        if (still == 0) {
            for (int i = threadIdx.x; i < cnt; i += W) {
                const int v = ~lout[i];
                ws.jm[r & 1][v] = out[v];
            }
            __syncthreads();
            break;
        }
        if (r + 1 >= max_rounds) {
            if (threadIdx.x == 0) atomicOr(&c->err, kErrDetect);
            return false;
        }
    }
    // ---- values: terminals (roots, exits) are final at once, as is a vertex
    //      whose successor is one; the rest jump
    for (int v = lo + (int)threadIdx.x; v < hi + pad; v += W) {
        bool keep = false;
        if (v < hi) {
            const int tag = ws.rep[v];
            if (tag == v || tag == n + v) {
                const JLS f{~tag, 0, 0};
                ws.jls[0][v] = f;
                ws.jls[1][v] = f;
            } else {
                const int sv = ws.succ[v];
                const int ts = ws.rep[sv];
                const bool fin = ts == sv || ts == n + sv;
                const JLS st{fin ? ~ts : sv, 1, (long long)ws.wpi[v]};
                ws.jls[0][v] = st;
                if (fin) ws.jls[1][v] = st;
                keep = !fin;
            }
        }
        block_append(LA, s_cnt, keep, v, lane);
    }
    __syncthreads();
    cnt = *s_cnt;
    __syncthreads();
    if (threadIdx.x == 0) *s_cnt = 0;
    __syncthreads();
    for (int j = 1; cnt > 0; ++j) {
        const JLS *in = ws.jls[(j + 1) & 1];
        JLS *out = ws.jls[j & 1];
        const int *lin = (j & 1) ? LA : LB;
        int *lout = (j & 1) ? LB : LA;
        int done_work = 0, kept = 0;
        for (int i0 = 0; i0 < cnt; i0 += kU * W) {
            int item[kU];
            JLS s[kU], t[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int i = i0 + u * W + (int)threadIdx.x;
                item[u] = i < cnt ? lin[i] : INT_MIN;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (item[u] != INT_MIN) s[u] = in[item[u] < 0 ? ~item[u] : item[u]];
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (item[u] != INT_MIN && item[u] >= 0) t[u] = in[s[u].J];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int it = item[u];
                bool keep = false, fin = false;
                int v = 0;
                if (it != INT_MIN) {
                    v = it < 0 ? ~it : it;
                    if (it < 0) {
                        out[v] = s[u];        // final last round: copy forward
                    } else {
                        const JLS nu{t[u].J, s[u].len + t[u].len, s[u].S + t[u].S};
                        out[v] = nu;
                        fin = nu.J < 0;
                        keep = !fin;
                        ++done_work;
                    }
                }
                block_append(lout, s_cnt, keep || fin, keep ? v : ~v, lane);
                kept += keep;
            }
        }
        __syncthreads();
        cnt = *s_cnt;
        const int left = block_sum_int(done_work, s_red);
        const int still = block_sum_int(kept, s_red);
        if (threadIdx.x == 0) *s_cnt = 0;
        __syncthreads();
        work += left;
        if (left == 0) break;
        if (still == 0) {
            for (int i = threadIdx.x; i < cnt; i += W) {
                const int v = ~lout[i];
                ws.jls[(j + 1) & 1][v] = out[v];
            }
            __syncthreads();
            break;
        }
        if (j + 1 > max_rounds) {
            if (threadIdx.x == 0) atomicOr(&c->err, kErrValue);
            return false;
        }
    }
    *work_total += work;
    return true;
}

// One-pass local phase for ranges without a cycle of their own: a single
// jumping pass carries, for every vertex, its jump target, the length and
// weight of the path to it and the smallest vertex on the way, so the exit a
// path leaves by (its tag), the path's (len, S) and the path minimum the node
// graph needs all come out of the same rounds (the two-pass phase finds the
// tags in a detection pass first and jumps for the values afterwards).  The
// state is packed into 16 bytes: bits 0-20 the jump target, 21-41 the path
// length (saturating), 42-62 the path minimum (local indices; all ones: none),
// bit 63 finished, then the weight.  Ping-pong buffers: the 16-byte scratch
// and the second value buffer; a
// finished vertex writes its final {~tag, len, S} to jls[0] and its
// {~tag, path minimum} for the node graph once; rep holds n + x for an exit
// x and -1 for the others (the tags are in jls[0]).  A path still unfinished after
// as many steps as the range has vertices lies in the basin of a cycle inside
// the range: the block then reports it and runs the two-pass phase instead.
// Needs ranges of fewer than 2^21 - 1 vertices.  Returns 1 done, 0 a cycle
// inside the range, -1 an error.
struct __align__(16) PackedState {
    unsigned long long a;
    long long S;
};
constexpr unsigned long long kPkMask = (1ULL << 21) - 1;
constexpr unsigned long long kPkNone = kPkMask;            // "no vertex" / saturated length
constexpr int kMaxOnePassRange = (1 << 21) - 2;

static __device__ __forceinline__ PackedState pk_make(unsigned J, unsigned len, unsigned M,
                                                     bool fin, long long S) {
    return PackedState{(unsigned long long)J | ((unsigned long long)len << 21) |
                           ((unsigned long long)M << 42) | (fin ? (1ULL << 63) : 0ULL),
                       S};
}

// Leaves (vertices no vertex of the range points to, about a third of them in
// a random policy graph) are never a jump target, and neither are vertices
// whose predecessors are all leaves.  When three bitmaps of the range fit in
// shared memory (bits, nwords words: has a predecessor, has a predecessor that
// is no leaf, and per-word prefix counts of the latter), the kept vertices
// are renumbered densely in vertex order (rank = set bits before them) and
// the rounds run on that dense index space -- states and lists stay
// contiguous, so a warp's accesses fill whole sectors -- while the two levels
// of leaves keep the one step to their successor in jls[0] (J = succ >= 0),
// which every reader completes (local_state): no pass over the range for
// them at the end.  Without the bitmaps every vertex takes part.  In the packed state a pending vertex's
// jump target is a dense index, a finished one's the local index of its exit.
static __device__ int local_onepass(int lo, int hi, int n, int max_rounds, const Workspace &ws,
                                    int *LA, int *LB, int *s_cnt, int *s_red, int *s_flag,
                                    unsigned *bits, int nwords, int *work_total) {
    Ctrl *c = ws.ctrl;
    const int lane = threadIdx.x & 31;
    const int W = blockDim.x;
    const int nv = hi - lo;
    const int nw = (nv + 31) / 32;
    const bool trim = nwords > 0 && 3 * nw <= nwords;
    unsigned *keep_bits = bits + nw;   // vertices with a predecessor that is no leaf
    unsigned *pref = bits + 2 * nw;    // set keep bits in the words before each word
    PackedState *P[2] = {reinterpret_cast<PackedState *>(ws.scratch16) + lo,
                         reinterpret_cast<PackedState *>(ws.jls[1]) + lo};
    int *orig = ws.aprev + lo;    // dense index -> vertex
    if (threadIdx.x == 0) *s_flag = 0;
    __shared__ int s_warp[32];
    int nd = nv;                  // vertices in the dense space
    int my_exits = 0;             // exits among this thread's vertices
    if (trim) {
        for (int i = threadIdx.x; i < 2 * nw; i += W) bits[i] = 0u;
        __syncthreads();
        for (int v = lo + (int)threadIdx.x; v < hi; v += W) {
            const int sv = ws.succ[v];
            if (sv >= lo && sv < hi) atomicOr(&bits[(sv - lo) >> 5], 1u << ((sv - lo) & 31));
            else ++my_exits;
        }
        __syncthreads();
        // second level: a vertex whose predecessors are all leaves is no jump
        // target either (jumps start at kept vertices and follow successors)
        for (int v = lo + (int)threadIdx.x; v < hi; v += W) {
            const int l = v - lo;
            const int sv = ws.succ[v];
            if (((bits[l >> 5] >> (l & 31)) & 1u) && sv >= lo && sv < hi)
                atomicOr(&keep_bits[(sv - lo) >> 5], 1u << ((sv - lo) & 31));
        }
        __syncthreads();
        // exclusive prefix of the word popcounts: each thread a contiguous chunk
        const int per = (nw + W - 1) / W;
        const int w0 = min(nw, (int)threadIdx.x * per), w1 = min(nw, w0 + per);
        int sum = 0;
        for (int i = w0; i < w1; ++i) sum += __popc(keep_bits[i]);
        __shared__ int s_total;
        const int incl = block_inclusive_scan(sum, s_warp);
        int run = incl - sum;
        for (int i = w0; i < w1; ++i) {
            pref[i] = (unsigned)run;
            run += __popc(keep_bits[i]);
        }
        if (threadIdx.x == W - 1) s_total = incl;
        __syncthreads();
        nd = s_total;
    } else {
        for (int v = lo + (int)threadIdx.x; v < hi; v += W) {
            const int sv = ws.succ[v];
            my_exits += sv < lo || sv >= hi;
        }
    }
    // the node list: every exit once; each thread's exits take consecutive
    // slots (one global atomic per block)
    int xpos;
    {
        __shared__ int s_xbase;
        const int incl = block_inclusive_scan(my_exits, s_warp);
        if (threadIdx.x == W - 1) s_xbase = atomicAdd(&c->node_cnt, incl);
        __syncthreads();
        xpos = s_xbase + incl - my_exits;
    }
    auto dense = [&](int v) -> int {   // dense index of a kept vertex
        const int l = v - lo;
        return trim ? (int)pref[l >> 5] + __popc(keep_bits[l >> 5] & ((1u << (l & 31)) - 1u))
                    : l;
    };
    auto has_pred = [&](int v) -> bool {   // kept: a predecessor that is no leaf
        const int l = v - lo;
        return !trim || ((keep_bits[l >> 5] >> (l & 31)) & 1u);
    };
    for (int v = lo + (int)threadIdx.x; v < hi; v += W) {
        const int sv = ws.succ[v];
        const bool is_exit = sv < lo || sv >= hi;
        if (is_exit) {
            ws.jls[0][v] = JLS{~(n + v), 0, 0};
            ws.rep[v] = n + v;
            ws.jm[1][v] = JM{~(n + v), INT_MAX};
            node_index(ws)[v] = xpos;
            ws.list[2][xpos++] = v;
        } else {
            // one step to the successor: final for a leaf, completed on read;
            // a kept vertex overwrites it with its final state below
            ws.jls[0][v] = JLS{sv, 1, (long long)ws.wpi[v]};
            ws.rep[v] = -1;   // no root, no exit (the root fix sets the roots)
        }
        if (!has_pred(v)) continue;   // a leaf
        const int d = dense(v);
        orig[d] = v;
        if (is_exit) {
            const PackedState f = pk_make((unsigned)(v - lo), 0, (unsigned)kPkNone, true, 0);
            P[0][d] = f;
            P[1][d] = f;
        } else {
            P[0][d] = pk_make((unsigned)dense(sv), 1, (unsigned)(v - lo), false,
                              (long long)ws.wpi[v]);
        }
    }
    __syncthreads();
    int work = 0;
    int cnt = nd;   // round 0: every dense index (finished ones are skipped)
    for (int r = 0; cnt > 0; ++r) {
        const PackedState *in = P[r & 1];
        PackedState *out = P[(r + 1) & 1];
        const int *lin = (r & 1) ? LB : LA;
        int *lout = (r & 1) ? LA : LB;
        int done_work = 0, kept = 0;
        bool basin = false;
        for (int i0 = 0; i0 < cnt; i0 += kU * W) {
            int item[kU];
            PackedState s[kU], t[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int i = i0 + u * W + (int)threadIdx.x;
                item[u] = i < cnt ? ((r == 0) ? i : lin[i]) : INT_MIN;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                if (item[u] == INT_MIN) continue;
                s[u] = in[item[u] < 0 ? ~item[u] : item[u]];
                if (r == 0 && (s[u].a >> 63)) item[u] = INT_MIN;   // an exit
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (item[u] != INT_MIN && item[u] >= 0) t[u] = in[(int)(s[u].a & kPkMask)];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int it = item[u];
                bool keep = false, fin = false;
                int d = 0;
                if (it != INT_MIN) {
                    d = it < 0 ? ~it : it;
                    if (it < 0) {
                        out[d] = s[u];        // finished last round: copy forward
                    } else {
                        const unsigned J = (unsigned)(t[u].a & kPkMask);
                        const unsigned len = min((unsigned)((s[u].a >> 21) & kPkMask) +
                                                     (unsigned)((t[u].a >> 21) & kPkMask),
                                                 (unsigned)kPkNone);
                        const unsigned M = min((unsigned)((s[u].a >> 42) & kPkMask),
                                               (unsigned)((t[u].a >> 42) & kPkMask));
                        fin = (t[u].a >> 63) != 0;
                        const long long S = s[u].S + t[u].S;
                        out[d] = pk_make(J, len, M, fin, S);
                        if (fin) {
                            const int v = orig[d];
                            const int tag = n + lo + (int)J;   // the exit the path leaves by
                            ws.jls[0][v] = JLS{~tag, (int)len, S};
                            ws.jm[1][v] = JM{~tag, M == kPkNone ? INT_MAX : lo + (int)M};
                        } else if ((int)len >= nv) {
                            basin = true;     // no exit within the range: a cycle inside it
                        } else {
                            keep = true;
                        }
                        ++done_work;
                    }
                }
                block_append(lout, s_cnt, keep || fin, keep ? d : ~d, lane);
                kept += keep;
            }
        }
        if (basin) *s_flag = 1;
        __syncthreads();
        cnt = *s_cnt;
        const int left = block_sum_int(done_work, s_red);
        const int still = block_sum_int(kept, s_red);
        if (threadIdx.x == 0) *s_cnt = 0;
        __syncthreads();
        work += left;
        if (*s_flag) return 0;   // (the same decision in every thread)
        if (left == 0) break;
        if (still == 0) break;   // (the finished states are in jls[0] already)
        if (r + 1 > max_rounds) {
            if (threadIdx.x == 0) atomicOr(&c->err, kErrValue);
            return -1;
        }
    }
    *work_total += work;
    return 1;
}

// Path v -> J(s) followed by the path J(s) -> J(t): target, length
// (saturating), minimum and finished bit of t's end, weights added.
static __device__ __forceinline__ PackedState pk_compose(const PackedState &s,
                                                         const PackedState &t) {
    const unsigned len = min((unsigned)((s.a >> 21) & kPkMask) + (unsigned)((t.a >> 21) & kPkMask),
                             (unsigned)kPkNone);
    const unsigned M = min((unsigned)((s.a >> 42) & kPkMask), (unsigned)((t.a >> 42) & kPkMask));
    return pk_make((unsigned)(t.a & kPkMask), len, M, (t.a >> 63) != 0, s.S + t.S);
}

// Chunked local phase.  On graphs whose edges mostly point to higher vertices
// (the synthetic locality graph: every edge goes forward) a policy path
// inside a block range only climbs, so the range can be taken in chunks of
// kLocalChunk vertices from its top down, each chunk finishing its vertices
// from the states of the chunks above it:
//   states: a vertex whose successor lies outside the range is an exit; one
//           whose successor lies in a chunk done before starts from that
//           vertex's state (finished: its exit, or pending: a path that goes
//           back below); the others start with the one step;
//   jumping inside the chunk in shared memory (two buffers of packed states)
//           until no path ends inside the chunk (a path of as many steps as
//           the chunk has vertices that still does lies in the basin of a
//           cycle inside the range);
//   writes: finished vertices get their final state {~(n + exit), len, S}
//           (jls[0]) and path minimum (jm[1]); a vertex whose path goes back
//           to a lower chunk is pending (its packed state in the 16-byte
//           scratch, J >= 0 in jls[0]) and listed in LA; the exits are listed
//           in LB (the cooperative kernel makes them nodes).
// The pending vertices are finished at the end by jumping over the range
// (none on the locality graph).  Every vertex ends with a final state, so the
// readers have no leaves to complete.  Returns 1 done, 0 a cycle inside the
// range (every exit listed; the two-pass phase takes over), -1 an error;
// *pending_out is the number of vertices the chunks left pending,
// *exits_out the number of exits listed.
static_assert(sizeof(PackedState) == kPackedStateBytes, "packed state size");

// State of vertex u (lo <= u < hi) of a chunk done before: final in jls[0]
// (J < 0, with its path minimum in jm[1]) or pending in P.
static __device__ __forceinline__ PackedState chunk_done_state(const Workspace &ws,
                                                               const PackedState *P, int lo,
                                                               int n, int u) {
    const JLS f = ws.jls[0][u];
    const JM d = ws.jm[1][u];
    if (f.J >= 0) return P[u - lo];
    return pk_make((unsigned)(~f.J - n - lo), (unsigned)f.len,
                   d.M == INT_MAX ? (unsigned)kPkNone : (unsigned)(d.M - lo), true, f.S);
}

static __device__ __forceinline__ void chunk_write_final(const Workspace &ws, int lo, int n,
                                                         int v, const PackedState &s) {
    const int tag = n + lo + (int)(s.a & kPkMask);
    const unsigned M = (unsigned)((s.a >> 42) & kPkMask);
    ws.jls[0][v] = JLS{~tag, (int)((s.a >> 21) & kPkMask), s.S};
    ws.jm[1][v] = JM{~tag, M == kPkNone ? INT_MAX : lo + (int)M};
}

static __device__ int local_chunked(int lo, int hi, int n, int max_rounds, const Workspace &ws,
                                    int *LA, int *LB, int *s_cnt, int *s_red, int *s_flag,
                                    PackedState *sm, int *pending_out, int *exits_out,
                                    int *work_total) {
    Ctrl *c = ws.ctrl;
    const int lane = threadIdx.x & 31;
    const int W = blockDim.x;   // kEvalThreads
    const int nv = hi - lo;
    PackedState *Pg = reinterpret_cast<PackedState *>(ws.scratch16) + lo;
    __shared__ int s_xcnt;
    if (threadIdx.x == 0) {
        *s_flag = 0;
        s_xcnt = 0;
    }
    // successors and weights of the next chunk, loaded while the one before
    // it is resolved
    int nsv[kLocalChunkPerThread], nwv[kLocalChunkPerThread];
    {
        const int c_lo = max(lo, hi - kLocalChunk);
#pragma unroll
        for (int u = 0; u < kLocalChunkPerThread; ++u) {
            const int v = c_lo + (int)threadIdx.x + u * W;
            nsv[u] = v < hi ? ws.succ[v] : -1;
            nwv[u] = v < hi ? ws.wpi[v] : 0;
        }
    }
    __syncthreads();
    for (int c_hi = hi; c_hi > lo; c_hi -= kLocalChunk) {
        const int c_lo = max(lo, c_hi - kLocalChunk);
        const int cn = c_hi - c_lo;
        const int off = c_lo - lo;   // local index of the chunk's first vertex
        // ---- the chunk's states: the targets in chunks done before first
        //      (all gathers in flight at once), then the states
        bool ex[kLocalChunkPerThread];
        JLS tf[kLocalChunkPerThread];
        JM td[kLocalChunkPerThread];
#pragma unroll
        for (int u = 0; u < kLocalChunkPerThread; ++u) {
            const int k = (int)threadIdx.x + u * W;
            const int sv = nsv[u];
            ex[u] = k < cn && (sv < lo || sv >= hi);
            tf[u].J = INT_MIN;
            if (k < cn && sv >= c_hi && sv < hi) {
                tf[u] = ws.jls[0][sv];
                td[u] = ws.jm[1][sv];
            }
        }
#pragma unroll
        for (int u = 0; u < kLocalChunkPerThread; ++u) {
            const int k = (int)threadIdx.x + u * W;
            if (k >= cn) continue;
            const int v = c_lo + k;
            const int sv = nsv[u];
            PackedState s;
            if (ex[u]) {
                s = pk_make((unsigned)(v - lo), 0, (unsigned)kPkNone, true, 0);
            } else {
                s = pk_make((unsigned)(sv - lo), 1, (unsigned)(v - lo), false, (long long)nwv[u]);
                if (tf[u].J != INT_MIN) {   // the successor's chunk is done
                    const PackedState t =
                        tf[u].J >= 0
                            ? Pg[sv - lo]   // pending: its path goes back to a lower chunk
                            : pk_make((unsigned)(~tf[u].J - n - lo), (unsigned)tf[u].len,
                                      td[u].M == INT_MAX ? (unsigned)kPkNone
                                                         : (unsigned)(td[u].M - lo),
                                      true, tf[u].S);
                    s = pk_compose(s, t);
                }
            }
            sm[k] = s;
        }
        {   // prefetch the next chunk
            const int n_lo = max(lo, c_lo - kLocalChunk);
#pragma unroll
            for (int u = 0; u < kLocalChunkPerThread; ++u) {
                const int v = n_lo + (int)threadIdx.x + u * W;
                nsv[u] = v < c_lo ? ws.succ[v] : -1;
                nwv[u] = v < c_lo ? ws.wpi[v] : 0;
            }
        }
        __syncthreads();
        // ---- jumping inside the chunk
        int fb = 0;   // the buffer with the chunk's current states
        for (int r = 0;; ++r) {
            const PackedState *in = sm + fb * kLocalChunk;
            PackedState *out = sm + (fb ^ 1) * kLocalChunk;
            bool more = false;
#pragma unroll
            for (int u = 0; u < kLocalChunkPerThread; ++u) {
                const int k = (int)threadIdx.x + u * W;
                if (k >= cn) continue;
                PackedState s = in[k];
                const int j = (int)(s.a & kPkMask) - off;
                if (!(s.a >> 63) && j >= 0 && j < cn) {
                    s = pk_compose(s, in[j]);
                    const int j2 = (int)(s.a & kPkMask) - off;
                    if (!(s.a >> 63) && j2 >= 0 && j2 < cn) {
                        more = true;
                        if ((int)((s.a >> 21) & kPkMask) >= cn) *s_flag = 1;   // a cycle here
                    }
                }
                out[k] = s;
            }
            fb ^= 1;
            if (!__syncthreads_or(more) || *s_flag) break;
            if (r + 1 > max_rounds) {
                if (threadIdx.x == 0) atomicOr(&c->err, kErrValue);
                return -1;
            }
        }
        // ---- write the chunk out (the exits are listed in LB, in block order)
        const PackedState *fin = sm + fb * kLocalChunk;
#pragma unroll
        for (int u = 0; u < kLocalChunkPerThread; ++u) {
            const int k = (int)threadIdx.x + u * W;
            bool pend = false;
            if (k < cn) {
                const int v = c_lo + k;
                if (ex[u]) {
                    ws.jls[0][v] = JLS{~(n + v), 0, 0};
                    ws.jm[1][v] = JM{~(n + v), INT_MAX};
                    ws.rep[v] = n + v;
                } else {
                    const PackedState s = fin[k];
                    ws.rep[v] = -1;   // no root, no exit (the root fix sets the roots)
                    if (s.a >> 63) {
                        chunk_write_final(ws, lo, n, v, s);
                    } else {
                        Pg[v - lo] = s;
                        ws.jls[0][v] = JLS{lo + (int)(s.a & kPkMask), 0, 0};   // pending
                        pend = true;
                    }
                }
            }
            block_append(LA, s_cnt, pend, off + k, lane);
            block_append(LB, &s_xcnt, ex[u], c_lo + k, lane);
        }
        __syncthreads();
    }
    *exits_out = s_xcnt;
    const int np = *s_cnt;
    __syncthreads();
    if (threadIdx.x == 0) *s_cnt = 0;
    *pending_out = np;
    int work = nv;
    if (*s_flag) {
        *work_total += work;
        return 0;
    }
    if (np > 0) {
        // ---- the paths going back to a lower chunk: jumping over the range
        //      (their targets' states: final in jls[0], or pending in the
        //      round's input buffer)
        PackedState *P[2] = {Pg, reinterpret_cast<PackedState *>(ws.jls[1]) + lo};
        int f = 0;
        for (int r = 0;; ++r) {
            const PackedState *in = P[f];
            PackedState *out = P[f ^ 1];
            int still = 0;
            for (int i = threadIdx.x; i < np; i += W) {
                const int d = LA[i];
                PackedState s = in[d];
                if (!(s.a >> 63)) {
                    s = pk_compose(s, chunk_done_state(ws, in, lo, n, lo + (int)(s.a & kPkMask)));
                    if (!(s.a >> 63)) {
                        ++still;
                        if ((int)((s.a >> 21) & kPkMask) >= nv) *s_flag = 1;   // a cycle here
                    }
                }
                out[d] = s;
            }
            f ^= 1;
            work += np;
            const int left = block_sum_int(still, s_red);
            if (*s_flag) {
                *work_total += work;
                return 0;
            }
            if (left == 0) break;
            if (r + 1 > max_rounds) {
                if (threadIdx.x == 0) atomicOr(&c->err, kErrValue);
                return -1;
            }
        }
        for (int i = threadIdx.x; i < np; i += W) {
            const int d = LA[i];
            chunk_write_final(ws, lo, n, lo + d, P[f][d]);
        }
        __syncthreads();
    }
    *work_total += work;
    return 1;
}

// The chunked local pass of every block range of the two-level evaluation
// (same grid and ranges as evaluate_local_kernel, which follows it): per
// range, (status, exits) in chunk_info -- status 1 done, 0 a cycle inside the
// range (the two-pass phase takes over), -1 an error, 2 not run (ranges too
// large for the packed state) -- and the range's exits in list[1].  Returns
// at once when the pass is off.
__global__ void __launch_bounds__(kEvalThreads, 1)
local_chunk_kernel(int n, int max_local, Workspace ws) {
    extern __shared__ __align__(16) unsigned s_chunk[];
    __shared__ int s_cnt, s_flag;
    __shared__ int s_red[kEvalThreads / 32];
    Ctrl *c = ws.ctrl;
    const int chunks = load_volatile(&c->local_chunks);
    if (!chunks) return;
    const int R = (n + (int)gridDim.x - 1) / (int)gridDim.x;
    const int lo = min((int)blockIdx.x * R, n), hi = min(lo + R, n);
    if (hi - lo > kMaxOnePassRange) {
        if (threadIdx.x == 0) ws.chunk_info[blockIdx.x] = make_int2(2, 0);
        return;
    }
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    int np = 0, nx = 0, work = 0;
    const int st = local_chunked(lo, hi, n, max_local, ws, ws.list[0] + lo, ws.list[1] + lo,
                                 &s_cnt, s_red, &s_flag, reinterpret_cast<PackedState *>(s_chunk),
                                 &np, &nx, &work);
    if (threadIdx.x == 0) {
        ws.chunk_info[blockIdx.x] = make_int2(st, nx);
        if (chunks == 1 && np > (hi - lo) / 8) atomicOr(&c->chunk_bad, 1);
        if (work)
            atomicAdd(reinterpret_cast<unsigned long long *>(&c->items_detect),
                      (unsigned long long)work);
    }
}

constexpr int kRerunMaxRoots = 32;   // roots on the node graph fixed by the grid-wide rerun

__global__ void __launch_bounds__(kEvalThreads, 1)
evaluate_local_kernel(int n, long long N2, int max_local, int max_node, int stall_test,
                      int nwords, Workspace ws, BatchState bs) {
    extern __shared__ unsigned s_bits[];   // nwords: the local predecessor bitmaps
    __shared__ long long s_key[kRankTile];
    __shared__ int s_cnt;
    __shared__ int s_red[kEvalThreads / 32];
    __shared__ int s_rerun;
    __shared__ int s_roots[kRerunMaxRoots], s_tags[kRerunMaxRoots];
    grid_sync_start();
    Ctrl *c = ws.ctrl;
    const unsigned nblocks = gridDim.x;
    const int stride = gridDim.x * blockDim.x;
    const int first = blockIdx.x * blockDim.x;
    const int R = (n + (int)gridDim.x - 1) / (int)gridDim.x;
    const int lo = min((int)blockIdx.x * R, n), hi = min(lo + R, n);
    int *LA = ws.list[0] + lo, *LB = ws.list[1] + lo;
    const int stamp = c->iter + 1;   // marks the roots found on the node graph in this evaluation
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->nrep = 0;
        c->best = 0;
        c->qmax = 0;
        c->node_cnt = 0;
    }
    if (threadIdx.x == 0) s_cnt = 0;
    // (the counters reset above are first used after this barrier)
    if (!grid_barrier(c, nblocks)) return;
    if (stall_test && !grid_barrier(c, nblocks + 1u)) return;

    // ---- local phase of every block (block barriers only): one pass, or
    //      two where the range holds a cycle of its own
    int work = 0;
    {
        // the chunked pass (0: off, 1: on while no range leaves more than an
        // eighth of its vertices pending, 2: always); read by every block
        // before the barrier after which block 0 may turn it off
        const int chunks = load_volatile(&c->local_chunks);
        int one = 0;
        if (hi - lo <= kMaxOnePassRange) {
            if (chunks) {
                // done by local_chunk_kernel: list the range's exits (in
                // list[1]) as nodes, one global atomic
                const int2 info = ws.chunk_info[blockIdx.x];
                __shared__ int s_xbase;
                if (threadIdx.x == 0) s_xbase = info.y ? atomicAdd(&c->node_cnt, info.y) : 0;
                __syncthreads();
                for (int i = threadIdx.x; i < info.y; i += blockDim.x) {
                    const int v = LB[i];
                    ws.list[2][s_xbase + i] = v;
                    node_index(ws)[v] = s_xbase + i;
                }
                one = info.x;
            } else {
                one = local_onepass(lo, hi, n, max_local, ws, LA, LB, &s_cnt, s_red, &s_rerun,
                                    s_bits, nwords, &work);
            }
        }
        if (one < 0) return;
        if (one == 0 &&
            !local_phase(lo, hi, n, false, hi - lo > kMaxOnePassRange, max_local, ws, LA, LB,
                         &s_cnt, s_red, &work))
            return;
    }
    if (!grid_barrier(c, nblocks)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0 && c->local_chunks == 1 &&
        load_volatile(&c->chunk_bad))
        c->local_chunks = 0;   // the paths mostly go backwards: leaf-trimmed rounds from now on
    const int K_exit = load_volatile(&c->node_cnt);
    const int K_local = load_volatile(&c->nrep);
    const int *X = ws.list[2];

    // ---- node graph: detection by window minima over segment minima
    const int *node_of = node_index(ws);
    JM *ND[2] = {reinterpret_cast<JM *>(ws.jt[0]), reinterpret_cast<JM *>(ws.jt[1])};
    int *NAP = ws.tpi;   // previous window minimum of each node
    for (int i = first + threadIdx.x; i < K_exit; i += stride) {
        const int x = X[i];
        const int y = ws.succ[x];
        // y's local result: through a leaf's steps (local_onepass) to the
        // first vertex with a state of its own (the leaves passed count for
        // the path minimum)
        int z = y, mz = INT_MAX;
        JLS f = ws.jls[0][z];
        for (int k = 0; k < 2 && f.J >= 0; ++k) {
            mz = min(mz, z);
            z = f.J;
            f = ws.jls[0][z];
        }
        const int ty = ~f.J;
        JM node;
        if (ty < n) {
            node = JM{~ty, 0};   // succ(x)'s path ends on a cycle inside its range
        } else {
            const JM d = ws.jm[1][z];   // aux = smallest vertex before the exit
            node = JM{node_of[ty - n], min(x, min(mz, d.M))};
        }
        ND[0][i] = node;
        ws.jls[1][x] = JLS{~(n + x), 0, 0};   // the exits' local state in both buffers
    }
    if (!grid_barrier(c, nblocks)) return;
    int nr = 0;
    for (int r = 0;; ++r) {
        const JM *in = ND[r & 1];
        JM *out = ND[(r + 1) & 1];
        int pend = 0;
        // (warp-uniform trip counts: the roots met are marked with one atomic
        // per distinct root and warp -- a cycle is met by most nodes at once)
        const int lane = threadIdx.x & 31;
        for (int i0 = first + (int)threadIdx.x - lane; i0 < K_exit; i0 += kNU * stride) {
            JM sn[kNU], tn[kNU];
            int ap[kNU];
#pragma unroll
            for (int u = 0; u < kNU; ++u) {
                const int i = i0 + lane + u * stride;
                if (i < K_exit) {
                    sn[u] = in[i];
                    ap[u] = NAP[i];
                }
            }
#pragma unroll
            for (int u = 0; u < kNU; ++u)
                if (i0 + lane + u * stride < K_exit && sn[u].J >= 0) tn[u] = in[sn[u].J];
#pragma unroll
            for (int u = 0; u < kNU; ++u) {
                const int i = i0 + lane + u * stride;
                int root = -1;
                bool win = false;   // the root of a cycle of the node graph, found here
                if (i < K_exit) {
                    if (sn[u].J < 0) {
                        out[i] = sn[u];
                    } else {
                        if (tn[u].J < 0) {
                            root = ~tn[u].J;
                        } else if (r > 0 && tn[u].M == ap[u]) {
                            root = tn[u].M;   // the cycle's smallest vertex (it may lie inside a segment)
                            win = true;
                        }
                        if (root >= 0) {
                            out[i] = JM{~root, 0};
                        } else {
                            out[i] = JM{tn[u].J, min(sn[u].M, tn[u].M)};
                            NAP[i] = tn[u].M;
                            ++pend;
                        }
                    }
                }
                unsigned m = __ballot_sync(0xffffffffu, win);
                while (m) {
                    const int leader = __ffs(m) - 1;
                    const int r0 = __shfl_sync(0xffffffffu, root, leader);
                    m &= ~__ballot_sync(0xffffffffu, win && root == r0);
                    if (lane == leader && load_volatile(&ws.root_mark[r0]) != stamp &&
                        atomicExch(&ws.root_mark[r0], stamp) != stamp) {
                        const int pos = atomicAdd(&c->nrep, 1);
                        ws.cyc_root[pos] = r0;
                    }
                }
            }
        }
        bool ok;
        const int left = grid_sum_barrier(c, nblocks, pend, &ok);
        if (!ok) return;
        ++nr;
        if (left == 0) break;
        if (r + 1 >= max_node) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&c->err, kErrDetect);
            return;
        }
    }
    const int K_all = load_volatile(&c->nrep);
    // ---- the roots found on the node graph become terminals.  The vertices
    //      whose local result changes are those draining to a root's exit
    //      (the root's former tag); the whole grid repeats their local value
    //      jumping with the roots as extra terminals.  Too many roots: every
    //      block holding one repeats its whole local phase instead.
    const int k_new = K_all - K_local;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int k = min(k_new, kRerunMaxRoots);
        for (int i = 0; i < k; ++i) {
            const int rt = ws.cyc_root[K_local + i];
            c->fix_root[i] = rt;
            c->fix_tag[i] = ~local_state(ws.jls[0], rt).J;
        }
        c->fix_k = k;
        c->fix_cnt = 0;
    }
    if (!grid_barrier(c, nblocks)) return;   // the former tags are read
    for (int i = K_local + first + threadIdx.x; i < K_all; i += stride) ws.rep[ws.cyc_root[i]] =
        ws.cyc_root[i];
    if (!grid_barrier(c, nblocks)) return;
    if (k_new > kRerunMaxRoots) {
        if (threadIdx.x == 0) {
            int any = 0;
            for (int i = K_local; i < K_all && !any; ++i) {
                const int rt = ws.cyc_root[i];
                any = rt >= lo && rt < hi;
            }
            s_rerun = any;
        }
        __syncthreads();
        if (s_rerun &&
            !local_phase(lo, hi, n, true, false, max_local, ws, LA, LB, &s_cnt, s_red, &work))
            return;
    } else if (k_new > 0) {
        if (threadIdx.x < kRerunMaxRoots) {
            s_roots[threadIdx.x] = threadIdx.x < k_new ? c->fix_root[threadIdx.x] : -1;
            s_tags[threadIdx.x] = threadIdx.x < k_new ? c->fix_tag[threadIdx.x] : -1;
        }
        __syncthreads();
        // the members: vertices of the roots' ranges tagged with a root's exit
        int *FL = ws.list[0];
        const long long span = (long long)k_new * R;
        // (warp-uniform trip counts: the members are listed with one atomic
        // per warp)
        const int lane = threadIdx.x & 31;
        for (long long q0 = first + (int)threadIdx.x - lane; q0 < span; q0 += stride) {
            const long long q = q0 + lane;
            bool listed = false;
            int v = 0;
            if (q < span) {
                const int ri = (int)(q / R);
                const int rlo = (s_roots[ri] / R) * R;
                bool seen = false;   // a range holding several roots is scanned once
                for (int i = 0; i < ri; ++i) seen |= (s_roots[i] / R) * R == rlo;
                v = rlo + (int)(q % R);
                if (!seen && v < n) {
                    bool root = false, member = false;
                    const int tag = ~ws.jls[0][v].J;   // (a leaf of local_onepass: no tag)
                    for (int i = 0; i < k_new; ++i) {
                        root |= s_roots[i] == v;
                        member |= s_tags[i] == tag;
                    }
                    const int sv = ws.succ[v];
                    if (root) {
                        const JLS f{~v, 0, 0};
                        ws.jls[0][v] = f;
                        ws.jls[1][v] = f;
                    } else if (member && sv >= rlo && sv < min(rlo + R, n)) {   // exits stay final
                        const int ts = ws.rep[sv];
                        const bool fin = ts == sv || ts == n + sv;
                        const JLS st{fin ? ~ts : sv, 1, (long long)ws.wpi[v]};
                        ws.jls[0][v] = st;
                        ws.jls[1][v] = st;
                        if (fin) ws.rep[v] = ts;   // (its successor is a root or the exit)
                        listed = !fin;
                    }
                }
            }
            const int pos = warp_append(&c->fix_cnt, listed, lane);
            if (listed) FL[pos] = v;
        }
        if (!grid_barrier(c, nblocks)) return;
        const int K_fix = load_volatile(&c->fix_cnt);
        for (int j = 1; K_fix > 0; ++j) {
            const JLS *in = ws.jls[(j + 1) & 1];
            JLS *out = ws.jls[j & 1];
            int pend = 0;
            for (int i = first + threadIdx.x; i < K_fix; i += stride) {
                const int v = FL[i];
                const JLS sv = in[v];
                if (sv.J < 0) {
                    out[v] = sv;
                    continue;
                }
                const JLS t = in[sv.J];
                const JLS nu{t.J, sv.len + t.len, sv.S + t.S};
                out[v] = nu;
                pend += nu.J >= 0;
            }
            bool ok;
            const int left = grid_sum_barrier(c, nblocks, pend, &ok);
            if (!ok) return;
            if (left == 0) {
                for (int i = first + threadIdx.x; i < K_fix; i += stride) {
                    const int v = FL[i];
                    const JLS f = out[v];
                    ws.jls[(j + 1) & 1][v] = f;
                    ws.rep[v] = ~f.J;   // a root met on the way, or the exit as before
                }
                break;
            }
            if (j + 1 > max_local) {
                if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&c->err, kErrValue);
                return;
            }
        }
    }
    if (!grid_barrier(c, nblocks)) return;

    // ---- node graph: (len, S) of every exit to its root, in node order; the
    //      final states go back to the exits' entries of jls[0]
    JLS *NV[2] = {reinterpret_cast<JLS *>(ws.scratch16), ws.jls[1]};
    for (int i = first + threadIdx.x; i < K_exit; i += stride) {
        const int x = X[i];
        JLS node;
        if (ws.rep[x] == x) {
            node = JLS{~x, 0, 0};   // an exit that is itself a root
        } else {
            const JLS f = local_state(ws.jls[0], ws.succ[x]);
            const int ty = ~f.J;
            const int len = 1 + f.len;
            const long long S = (long long)ws.wpi[x] + f.S;
            if (ty < n) {
                node = JLS{~ty, len, S};
            } else {
                const int xn = ty - n;
                node = JLS{ws.rep[xn] == xn ? ~xn : node_of[xn], len, S};
            }
        }
        NV[0][i] = node;
    }
    if (!grid_barrier(c, nblocks)) return;
    int FN = 0;
    for (int j = 1;; ++j) {
        const JLS *in = NV[(j + 1) & 1];
        JLS *out = NV[j & 1];
        int pend = 0;
        for (int i0 = first + threadIdx.x; i0 < K_exit; i0 += kNU * stride) {
            JLS sn[kNU], tn[kNU];
#pragma unroll
            for (int u = 0; u < kNU; ++u)
                if (i0 + u * stride < K_exit) sn[u] = in[i0 + u * stride];
#pragma unroll
            for (int u = 0; u < kNU; ++u)
                if (i0 + u * stride < K_exit && sn[u].J >= 0) tn[u] = in[sn[u].J];
#pragma unroll
            for (int u = 0; u < kNU; ++u) {
                const int i = i0 + u * stride;
                if (i >= K_exit) continue;
                if (sn[u].J < 0) {
                    out[i] = sn[u];
                    continue;
                }
                const JLS nu{tn[u].J, sn[u].len + tn[u].len, sn[u].S + tn[u].S};
                out[i] = nu;
                pend += nu.J >= 0;
            }
        }
        bool ok;
        const int left = grid_sum_barrier(c, nblocks, pend, &ok);
        if (!ok) return;
        ++nr;
        FN = j & 1;
        if (left == 0) break;
        if (j + 1 > max_node) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&c->err, kErrValue);
            return;
        }
    }
    for (int i = first + threadIdx.x; i < K_exit; i += stride) ws.jls[0][X[i]] = NV[FN][i];
    if (!grid_barrier(c, nblocks)) return;

    // (the expansion of exit-bound vertices happens in the tail)
    if (threadIdx.x == 0 && work)
        atomicAdd(reinterpret_cast<unsigned long long *>(&c->items_detect),
                  (unsigned long long)work);
    if (blockIdx.x == 0 && threadIdx.x == 0) c->rounds_detect += nr;
    evaluate_tail<false, true>(n, N2, 0, ws, bs, s_key);
}

}  // namespace ocm

namespace ocm {

// Co-resident CTAs of the two-level evaluation kernel on the current device.
static int evaluate_local_grid() {
    static int cached_dev = -1, cached = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev == cached_dev && cached > 0) return cached;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    // co-resident with the largest bitmap any launch uses
    if (cudaFuncSetAttribute(evaluate_local_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kLocalBitmapWords * 4) != cudaSuccess ||
        cudaFuncSetAttribute(local_chunk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kLocalChunkBytes) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, evaluate_local_kernel,
                                                      kEvalThreads, kLocalBitmapWords * 4) !=
            cudaSuccess ||
        per_sm < 1)
        return 0;
    cached_dev = dev;
    cached = sms * per_sm;
    return cached;
}

int prepare_evaluate_local() { return evaluate_local_grid() > 0 ? 0 : -1; }

// Blocks of the two-level evaluation for n vertices (its ranges are n / blocks).
int evaluate_local_blocks(int n) {
    int blocks = evaluate_local_grid();
    const int need = (n + kEvalThreads - 1) / kEvalThreads;
    if (blocks > need) blocks = need;
    return blocks;
}

}  // namespace ocm
