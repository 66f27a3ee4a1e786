// grid_sync.cuh -- the bounded grid-wide barrier of the library's cooperative
// kernels (policy evaluation, SCC decomposition).  Every block of a
// cooperative launch is co-resident, so a counter in device memory can act as
// a barrier; waits are bounded by an SM-clock limit, after which the kernel
// records kErrTimeout and returns instead of hanging.
#pragma once

#include "common.cuh"

namespace ocm {

constexpr long long kBarrierClockLimit = 4000000000LL;   // SM cycles: about two seconds
constexpr long long kStallTestClockLimit = 20000000LL;   // about 10 ms (OCM_FLAG_TEST_STALL)

static __device__ __forceinline__ int load_volatile(const int *p) {
    return *reinterpret_cast<const volatile int *>(p);
}

// Grid-wide barrier of a cooperative launch that also sums one count per
// thread over the whole grid: the block total rides on the arrival atomic
// (arrivals in the high 32 bits, counts in the low 32), and the last block
// to arrive publishes the grand total before releasing the others.  Waits
// are bounded by an SM-clock limit; on expiry every block records
// kErrTimeout and *ok becomes false.
static __device__ int grid_sum_barrier(Ctrl *c, unsigned nblocks, int x, bool *ok,
                                       long long limit = kBarrierClockLimit) {
    __shared__ int s_sum;
    __shared__ int s_total;
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s_sum, x);
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &c->bar_gen;
        const unsigned g = *gen;
        __threadfence();
        const unsigned long long old =
            atomicAdd(&c->bar_word, (1ULL << 32) | (unsigned long long)(unsigned)s_sum);
        int okv = 1;
        if ((unsigned)(old >> 32) == nblocks - 1) {
            c->bar_total = (int)(unsigned)(old & 0xffffffffULL) + s_sum;
            c->bar_word = 0;
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (clock64() - t0 > limit ||
                    (load_volatile(&c->err) & kErrTimeout)) {
                    atomicOr(&c->err, kErrTimeout);
                    okv = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_total = load_volatile(&c->bar_total);
        s_ok = okv;
    }
    __syncthreads();
    *ok = s_ok != 0;
    return s_total;
}

static __device__ __forceinline__ bool grid_barrier(Ctrl *c, unsigned nblocks,
                                                    long long limit = kBarrierClockLimit) {
    bool ok;
    grid_sum_barrier(c, nblocks, 0, &ok, limit);
    return ok;
}

}  // namespace ocm
