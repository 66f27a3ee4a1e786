// static_ws.cu -- ocm_solve_static: the solver for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they want a solve: code running inside a memory-capped or pre-partitioned
// process whose pool is already handed out, plugins and real-time loops that
// must not allocate after start-up, or hosts without a device allocator of
// their own to lend.  For them this file keeps the solver's scratch space in a
// fixed array that lives in the library image itself: it is created when the
// library's GPU code is loaded on a device and stays there until the process
// exits (on every device that loads the library).
//
// The entry point only adds the workspace; the solve itself is ocm_solve,
// unchanged.
#include <cstring>

#include "common.cuh"

// Scratch for ocm_solve_static, shared by every call on a device.
static __device__ __align__(256) unsigned char g_static_workspace[OCM_STATIC_WORKSPACE_BYTES];

namespace {

// Device address of g_static_workspace in the current context.  In host code
// the array's name only stands for the host-side shadow symbol, so the real
// address must come from the runtime, with the device current.  It is looked
// up on every call rather than cached: a context that was torn down and
// created again (cudaDeviceReset, a reset of the primary context) reloads the
// module, and the array may then sit elsewhere.  Once the module is loaded the
// lookup allocates nothing.
int static_workspace_address(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_workspace);
    if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return OCM_ERR_CUDA;
    }
    *out = p;
    return OCM_OK;
}

}  // namespace

extern "C" int ocm_solve_static(const int32_t *row_ptr, const int32_t *col_idx, const int32_t *w,
                                int32_t n, int32_t m, int mode, int64_t *num, int32_t *den,
                                int32_t *cycle_out, int32_t *cycle_len, void *stream,
                                const ocm_options *opt, ocm_stats *stats) {
    if (n < 1 || m < 1) return OCM_ERR_INVALID_ARG;
    const size_t need = (opt && (opt->flags & OCM_FLAG_SINGLE_LAMBDA))
                            ? ocm_workspace_size_single(n, m)
                            : ocm_workspace_size(n, m);
    if (need == 0 || need > (size_t)OCM_STATIC_WORKSPACE_BYTES) return OCM_ERR_WORKSPACE;
    void *ws = nullptr;
    int rc = static_workspace_address(&ws);
    if (rc != OCM_OK) return rc;
    // ocm_solve initialises everything it reads (its control block is reset
    // by its first kernel, every other array is written before it is read),
    // so the previous call's contents need no clearing here.  Benchmark
    // instrumentation would create CUDA events, and instantiating the loop
    // graph would have the driver allocate, so the instrumentation is paused
    // and the loop is driven from the host.
    ocm_options o;
    if (opt) o = *opt; else memset(&o, 0, sizeof o);
    o.flags |= OCM_FLAG_HOST_LOOP;
    ocm::ProfilePause pause;   // this thread only; other threads keep their events
    return ocm_solve(row_ptr, col_idx, w, n, m, mode, num, den, cycle_out, cycle_len, ws,
                     (size_t)OCM_STATIC_WORKSPACE_BYTES, stream, &o, stats);
}
