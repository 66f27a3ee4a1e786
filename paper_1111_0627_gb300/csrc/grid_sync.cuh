// grid_sync.cuh -- the bounded grid-wide barrier of the library's cooperative
// kernels (policy evaluation, single-lambda rebuild, SCC decomposition and its
// sort).  Every block of a cooperative launch is co-resident, so a counter in
// device memory can act as a barrier; waits are bounded by a wall-clock limit
// (the GPU's global nanosecond timer), after which the kernel records
// kErrTimeout and returns instead of hanging.
#pragma once

#include "common.cuh"

namespace ocm {

// Limit argument of the barriers below: 0 = the control block's wait_ns (set
// per call from ocm_options.wait_limit_ms, two seconds by default).
constexpr long long kWaitFromCtrl = 0;

static __device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

static __device__ __forceinline__ int load_volatile(const int *p) {
    return *reinterpret_cast<const volatile int *>(p);
}

// Per block, the number of grid barriers passed in this launch (used by
// thread 0 only).  Every cooperative kernel calls grid_sync_start() first.
static __device__ __forceinline__ unsigned *bar_round() {
    __shared__ unsigned r;
    return &r;
}

static __device__ __forceinline__ void grid_sync_start() {
    if (threadIdx.x == 0) *bar_round() = 0;
}

// Grid-wide barrier of a cooperative launch that also sums one count per
// thread over the whole grid.  Thread 0 of each block adds its block's total
// to the slot of barrier g (g = barriers this block passed before, the same
// for every block), then counts its arrival with a release add; the barrier
// is complete once the arrivals reach nblocks * (g + 1), which every block
// polls with acquire loads -- no block has to publish a release, saving the
// second round trip a last-arriver scheme needs.  Block 0 clears the slot of
// barrier g + 2 before it arrives at g: that slot was last read before
// barrier g - 1 completed and is next written after barrier g + 1 completes.
// Waits are bounded by `limit` nanoseconds (kWaitFromCtrl: the control
// block's wait_ns); on expiry every block records kErrTimeout and *ok becomes
// false.  `which` selects the kernel's GridBar.
template <bool TWO>
static __device__ __forceinline__ int grid_sum_barrier_impl(Ctrl *c, unsigned nblocks, int x,
                                                            int y, int *ysum, bool *ok,
                                                            long long limit, int which) {
    __shared__ int s_sum, s_sum2;
    __shared__ int s_total, s_total2;
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        s_sum = 0;
        if (TWO) s_sum2 = 0;
    }
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        if (TWO) y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (x) atomicAdd(&s_sum, x);
        if (TWO && y) atomicAdd(&s_sum2, y);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        GridBar *b = &c->bar[which];
        const long long lim = limit > 0 ? limit : c->wait_ns;
        unsigned *rp = bar_round();
        const unsigned g = *rp;
        const int slot = (int)(g & 3u);
        if (s_sum) atomicAdd(&b->sum[slot], s_sum);
        if (TWO && s_sum2) atomicAdd(&b->sum2[slot], s_sum2);
        if (blockIdx.x == 0) {
            b->sum[(g + 2) & 3u] = 0;
            b->sum2[(g + 2) & 3u] = 0;
        }
        __threadfence();
        asm volatile("red.release.gpu.global.add.u64 [%0], %1;"
                     :: "l"(&b->arrive), "l"(1ULL) : "memory");
        const unsigned long long target = (unsigned long long)nblocks * (g + 1);
        int okv = 1;
        const long long t0 = global_ns();
        for (unsigned it = 1;; ++it) {
            unsigned long long a;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];"
                         : "=l"(a) : "l"(&b->arrive) : "memory");
            if (a >= target) break;
            if ((it & 63u) == 0 &&
                (global_ns() - t0 > lim || (load_volatile(&c->err) & kErrTimeout))) {
                atomicOr(&c->err, kErrTimeout);
                okv = 0;
                break;
            }
        }
        int t;
        asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];"
                     : "=r"(t) : "l"(&b->sum[slot]) : "memory");
        s_total = t;
        if (TWO) {
            asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];"
                         : "=r"(t) : "l"(&b->sum2[slot]) : "memory");
            s_total2 = t;
        }
        s_ok = okv;
        *rp = g + 1;
    }
    __syncthreads();
    *ok = s_ok != 0;
    if (TWO) *ysum = s_total2;
    return s_total;
}

static __device__ __forceinline__ int grid_sum_barrier(Ctrl *c, unsigned nblocks, int x, bool *ok,
                                                       long long limit = kWaitFromCtrl,
                                                       int which = 0) {
    return grid_sum_barrier_impl<false>(c, nblocks, x, 0, nullptr, ok, limit, which);
}

// The same barrier summing two counts: returns the sum of x, *ysum gets the
// sum of y.
static __device__ __forceinline__ int grid_sum2_barrier(Ctrl *c, unsigned nblocks, int x, int y,
                                                        int *ysum, bool *ok) {
    return grid_sum_barrier_impl<true>(c, nblocks, x, y, ysum, ok, kWaitFromCtrl, 0);
}

static __device__ __forceinline__ bool grid_barrier(Ctrl *c, unsigned nblocks,
                                                    long long limit = kWaitFromCtrl,
                                                    int which = 0) {
    bool ok;
    grid_sum_barrier(c, nblocks, 0, &ok, limit, which);
    return ok;
}

}  // namespace ocm
