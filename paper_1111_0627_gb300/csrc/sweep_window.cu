// sweep_window.cu -- the improvement sweep (Alg. 1's pass over all vertices,
// Alg. 2 SPFPassIter) for graphs whose edges mostly point near their source
// in vertex order.
//
// The sweep gathers the 16-byte record (V, rank, q) of every edge's target.
// Through L1 each such gather costs a cache-line lookup of its own, and that
// lookup rate, not HBM, bounds the degree-class sweep of sweep.cu.  Here one
// block per SM owns a contiguous chunk of vertices and walks it in tiles of
// kWinTile vertices; the records of a window of vertices around the tile sit
// in shared memory, in a ring of kWinRegions regions of kWinTile records that
// the Tensor Memory Accelerator fills: while a tile is swept, one bulk copy
// (cp.async.bulk, completing on an mbarrier) brings the region the next tile
// adds to the window, and a bulk L2 prefetch brings the next tile's edges.
// Targets inside the window are read from shared memory, the others from
// global memory as before.  The window of tile [a, a + T) is
// [a - hb, a - hb + (kWinRegions - 1) T): hb (0 .. 4T) is chosen per solve
// from the initial pass's count of edges whose target falls in
// [v - hb, v - hb + 4T) (the halo every vertex of the tile is sure to see).
//
// Inside a tile the vertices are grouped by degree class in shared memory and
// served exactly as improve_kernel serves them (a lane group per vertex, the
// same candidate order, strict switching, ties to the smaller edge index), so
// the sweep switches the same vertices to the same edges.  Vertices with more
// than kHeavyEdges out-edges are left to the heavy kernels of sweep.cu.
#include <climits>

#include "common.cuh"
#include "grid_sync.cuh"

namespace ocm {

constexpr int kWinRegions = 6;                      // the window's 5 regions and the one filling
constexpr int kWinRing = kWinRegions * kWinTile;    // records in shared memory (192 KB)
constexpr int kWinSpan = (kWinRegions - 1) * kWinTile;
constexpr int kWinThreads = 1024;
constexpr int kWinWarps = kWinThreads / 32;
static_assert(kWinTile == 2 * kWinThreads, "two class passes per tile");
static_assert(kWinSpan == kWinTile + kWinHalo, "the window: the tile and its halo");

static __device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

static __device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Announces `bytes` of copies on the barrier's current phase and arrives.
static __device__ __forceinline__ void mbar_expect(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Waits for the phase with the given parity to complete, at most limit_ns of
// GPU time; false when the limit ran out.
static __device__ bool mbar_wait(unsigned long long *bar, unsigned parity, long long limit_ns) {
    const unsigned a = smem_addr(bar);
    const long long t0 = global_ns();
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// Bulk copy of records [x0, x0 + kWinTile) clipped to [0, n) into their ring
// slots ((x - L0) mod kWinRing); returns the bytes issued (the caller has
// announced them on the barrier).
static __device__ __forceinline__ unsigned region_bytes(long long x0, int n) {
    const long long lo = x0 < 0 ? 0 : x0;
    const long long hi = x0 + kWinTile < n ? x0 + kWinTile : n;
    return hi > lo ? (unsigned)((hi - lo) * (long long)sizeof(int4)) : 0u;
}

static __device__ __forceinline__ void region_copy(int4 *ring, const int4 *rec, long long x0,
                                                   int slot0, int n, unsigned long long *bar) {
    const long long lo = x0 < 0 ? 0 : x0;
    const long long hi = x0 + kWinTile < n ? x0 + kWinTile : n;
    if (hi <= lo) return;
    const unsigned bytes = (unsigned)((hi - lo) * (long long)sizeof(int4));
    const int4 *src = rec + lo;
    int4 *dst = ring + slot0 + (int)(lo - x0);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Prefetch into L2 of the whole 16-byte blocks inside [p, p + count) ints.
static __device__ __forceinline__ void prefetch_l2(const int *p, long long count) {
    const unsigned long long a = (unsigned long long)p;
    const unsigned long long b = a + (unsigned long long)count * 4ULL;
    const unsigned long long a16 = (a + 15ULL) & ~15ULL, b16 = b & ~15ULL;
    for (unsigned long long s = a16; s + 16 <= b16;) {
        const unsigned long long len = (b16 - s) < (1ULL << 20) ? (b16 - s) : (1ULL << 20);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s), "r"((unsigned)len)
                     : "memory");
        s += len;
    }
}

__global__ void __launch_bounds__(kWinThreads, 1)
improve_window_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col,
                      const int *__restrict__ w, int sign, int n, int epl, int hb, Workspace ws,
                      BatchState bs) {
    extern __shared__ int4 s_ring[];                  // kWinRing records
    // the tile's vertices by class: {first edge, (index in the tile << 11) | degree}
    __shared__ int2 s_list[kWinTile];
    __shared__ int s_cnt[kClasses], s_off[kClasses], s_cur[kClasses], s_task[kClasses + 1];
    __shared__ int s_sw;
    __shared__ __align__(8) unsigned long long s_bar[3];   // [0], [1]: per tile; [2]: prologue
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Ctrl *c = ws.ctrl;
    const long long limit = c->wait_ns;
    const int next_eval = c->iter + 1;
    const int4 *rec = reinterpret_cast<const int4 *>(ws.rec);
    const int chunk = (n + (int)gridDim.x - 1) / (int)gridDim.x;
    const int c0 = min((int)blockIdx.x * chunk, n), c1 = min(c0 + chunk, n);
    const int ntiles = (c1 - c0 + kWinTile - 1) / kWinTile;
    const long long L0 = (long long)c0 - hb;          // window start of tile 0
    if (blockIdx.x == 0 && tid == 0) publish_result(ws, n);
    if (tid == 0) {
        s_sw = 0;
        for (int i = 0; i < 3; ++i) mbar_init(&s_bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (ntiles == 0) return;
    if (tid == 0) {
        // the first window: regions 0 .. kWinRegions - 2
        unsigned bytes = 0;
        for (int r = 0; r < kWinRegions - 1; ++r) bytes += region_bytes(L0 + (long long)r * kWinTile, n);
        mbar_expect(&s_bar[2], bytes);
        for (int r = 0; r < kWinRegions - 1; ++r)
            region_copy(s_ring, rec, L0 + (long long)r * kWinTile, r * kWinTile, n, &s_bar[2]);
        prefetch_l2(col + row_ptr[c0], (long long)row_ptr[min(c0 + kWinTile, c1)] - row_ptr[c0]);
        prefetch_l2(w + row_ptr[c0], (long long)row_ptr[min(c0 + kWinTile, c1)] - row_ptr[c0]);
    }
    // a wait that runs out ends the sweep with kErrTimeout (the same decision
    // in every thread); the copy it waited for is then waited for once more
    int fail_bar = -1;
    unsigned fail_par = 0;
    if (__syncthreads_or(!mbar_wait(&s_bar[2], 0, limit))) fail_bar = 2;
    int switched = 0;
    for (int k = 0; k < ntiles && fail_bar < 0; ++k) {
        const int a = c0 + k * kWinTile, tn = min(kWinTile, c1 - a);
        const long long wlo = L0 + (long long)k * kWinTile;   // window [wlo, wlo + kWinSpan)
        const int base = (k % kWinRegions) * kWinTile;         // ring slot of wlo
        if (k > 0) {
            const int bi = (k - 1) & 1;
            const unsigned par = ((k - 1) >> 1) & 1;
            if (__syncthreads_or(!mbar_wait(&s_bar[bi], par, limit))) {
                fail_bar = bi;
                fail_par = par;
                break;
            }
        }
        if (tid == 0) {
            // the region tile k + 1 adds (its slots held tile k - 1's first
            // region, which nobody reads any more), and tile k + 1's edges
            if (k + 1 < ntiles) {
                const long long x0 = wlo + kWinSpan;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect(&s_bar[k & 1], region_bytes(x0, n));
                region_copy(s_ring, rec, x0, ((k + kWinRegions - 1) % kWinRegions) * kWinTile, n,
                            &s_bar[k & 1]);
                const int b0 = a + kWinTile, b1 = min(b0 + kWinTile, c1);
                prefetch_l2(col + row_ptr[b0], (long long)row_ptr[b1] - row_ptr[b0]);
                prefetch_l2(w + row_ptr[b0], (long long)row_ptr[b1] - row_ptr[b0]);
                prefetch_l2(row_ptr + b0, (long long)(b1 - b0) + 1);
                prefetch_l2(ws.pi + b0, (long long)(b1 - b0));
            }
            for (int q = 0; q < kClasses; ++q) {
                s_cnt[q] = 0;
                s_cur[q] = 0;
            }
        }
        __syncthreads();
        // ---- the tile's vertices by degree class (two vertices a thread)
        int cls[2];
        int2 item[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = tid + h * kWinThreads;
            int q = -1;
            if (i < tn) {
                const int v = a + i;
                const int e0 = __ldg(&row_ptr[v]), d = __ldg(&row_ptr[v + 1]) - e0;
                q = degree_class(d, epl);
                item[h] = make_int2(e0, (i << 11) | (d & 2047));
                // batched: a graph whose last sweep switched nothing is done
                if (q >= kClasses || (bs.G && bs.gconv[bs.gid[v]])) q = -1;
            }
            cls[h] = q;
#pragma unroll
            for (int q2 = 0; q2 < kClasses; ++q2) {
                const unsigned m = __ballot_sync(0xffffffffu, q == q2);
                if (lane == 0 && m) atomicAdd(&s_cnt[q2], __popc(m));
            }
        }
        __syncthreads();
        if (tid == 0) {
            int off = 0, tasks = 0;
            for (int q = 0; q < kClasses; ++q) {
                s_off[q] = off;
                s_task[q] = tasks;
                off += s_cnt[q];
                tasks += ((s_cnt[q] << q) + 31) >> 5;
            }
            s_task[kClasses] = tasks;
        }
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = cls[h];
#pragma unroll
            for (int q2 = 0; q2 < kClasses; ++q2) {
                const unsigned m = __ballot_sync(0xffffffffu, q == q2);
                int b = 0;
                if (lane == 0 && m) b = atomicAdd(&s_cur[q2], __popc(m));
                b = __shfl_sync(0xffffffffu, b, 0);
                if (q == q2) s_list[s_off[q2] + b + __popc(m & ((1u << lane) - 1u))] = item[h];
            }
        }
        __syncthreads();
        // ---- warp tasks: a lane group of 2^q lanes per vertex of class q
        const int total = s_task[kClasses];
        for (int task = warp; task < total; task += kWinWarps) {
            int q = 0;
#pragma unroll
            for (int k2 = 1; k2 < kClasses; ++k2)
                if (task >= s_task[k2]) q = k2;
            const int g = 1 << q;
            const int sub = lane & (g - 1);
            const int idx = (task - s_task[q]) * (32 >> q) + (lane >> q);
            const bool valid = idx < s_cnt[q];
            const int2 it = valid ? s_list[s_off[q] + idx] : make_int2(0, 0);
            const int v = a + (it.y >> 11);
            Cand best{INT_MIN, INT_MAX, LLONG_MIN};
            Cand own{INT_MIN, INT_MAX, LLONG_MIN};   // the current policy edge, in one lane
            if (valid) {
                const int e_end = it.x + (it.y & 2047);
                const int pv = ws.pi[v];
                auto cand = [&](int e) -> Cand {
                    const int t = __ldg(&col[e]);
                    const int x = __ldg(&w[e]);
                    const long long off = (long long)t - wlo;
                    int4 r;
                    if (off >= 0 && off < kWinSpan) {
                        int s = base + (int)off;
                        if (s >= kWinRing) s -= kWinRing;
                        r = s_ring[s];
                    } else {
                        r = __ldg(&rec[t]);
                    }
                    const long long V = ((long long)(unsigned)r.x) | ((long long)r.y << 32);
                    return Cand{r.z, e, (long long)r.w * (long long)(sign * x) + V};
                };
                int e = it.x + sub;
                for (; e + g < e_end; e += 2 * g) {
                    const Cand x0 = cand(e);
                    const Cand x1 = cand(e + g);
                    if (e == pv) own = x0;
                    if (e + g == pv) own = x1;
                    if (better(x0, best)) best = x0;
                    if (better(x1, best)) best = x1;
                }
                if (e < e_end) {
                    const Cand x0 = cand(e);
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
            if (valid && own.e != INT_MAX &&
                (best.rank > own.rank || (best.rank == own.rank && best.key > own.key))) {
                ws.pi[v] = best.e;
                ws.succ[v] = __ldg(&col[best.e]);
                ws.wpi[v] = sign * __ldg(&w[best.e]);
                ws.sw_iter[v] = next_eval;
                if (bs.G) {
                    const int gg = bs.gid[v];
                    if (bs.gsw[gg] != next_eval) bs.gsw[gg] = next_eval;
                }
                ++switched;
            }
        }
        __syncthreads();   // the tile's ring region and class list are free again
    }
    if (fail_bar >= 0) {
        if (tid == 0) atomicOr(&c->err, kErrTimeout);
        mbar_wait(&s_bar[fail_bar], fail_par, limit);
        return;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) switched += __shfl_xor_sync(0xffffffffu, switched, o);
    if (lane == 0 && switched) atomicAdd(&s_sw, switched);
    __syncthreads();
    if (tid == 0 && s_sw) {
        atomicAdd(&c->switched, s_sw);
        c->changed = 1;
    }
}

// Co-resident blocks of the window sweep on the current device (one per SM).
static int window_grid() {
    static int cached_dev = -1, cached = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev == cached_dev && cached > 0) return cached;
    int sms = 0, per_sm = 0;
    if (cudaFuncSetAttribute(improve_window_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kWinRing * (int)sizeof(int4)) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, improve_window_kernel, kWinThreads,
                                                      kWinRing * (int)sizeof(int4)) !=
            cudaSuccess ||
        sms <= 0 || per_sm <= 0)
        return 0;
    cached = sms * per_sm;
    cached_dev = dev;
    return cached;
}

int prepare_sweep_window() { return window_grid() > 0 ? 0 : -1; }

int launch_sweep_window(const int *row_ptr, const int *col, const int *w, int sign, int n,
                        int epl, int hb, Workspace ws, const int *cls_cnt, int heavy_edges,
                        BatchState bs, cudaStream_t st) {
    const int blocks = window_grid();
    if (blocks <= 0) return -1;
    prof_begin(kProfSweep, st);
    improve_window_kernel<<<blocks, kWinThreads, kWinRing * sizeof(int4), st>>>(
        row_ptr, col, w, sign, n, epl, hb, ws, bs);
    const int kh = launch_sweep_heavy(row_ptr, col, w, sign, ws, cls_cnt[kClasses], heavy_edges,
                                      bs, st);
    prof_end(kProfSweep, st);
    if (kh < 0) return -1;
    return 1 + kh;
}

}  // namespace ocm
