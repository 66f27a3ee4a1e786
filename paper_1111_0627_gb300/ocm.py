"""Python binding of the optimal-cycle-mean solver (argument marshalling only).

Every step of the computation runs in the CUDA kernels of ``libocm.so``;
this module checks tensor types, allocates the caller-owned workspace and
output tensors with PyTorch, and calls the C ABI of ``include/ocm.h`` with
raw device pointers and the current CUDA stream.  There is no CPU fallback.

    >>> num, den, cycle = solve(row_ptr, col_idx, w, mode="max")[:3]

``OCMFunction`` exposes lambda* to autograd: the forward is ``ocm_solve`` on
the int32 weights, the backward is ``ocm_backward`` (d lambda*/d w(e) =
1/|C*| on the critical cycle C*, 0 elsewhere).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from fractions import Fraction

import torch

from . import _native

OCM_MAX, OCM_MIN = 0, 1
OCM_FLAG_TEST_STALL = 1
OCM_FLAG_HOST_LOOP = 2
OCM_FLAG_SINGLE_LAMBDA = 4
OCM_FLAG_EVAL_LOCAL = 8     # force the two-level evaluation (include/ocm.h)
OCM_FLAG_EVAL_GLOBAL = 16   # forbid it
OCM_FLAG_TEST_NO_BITMAP = 32  # test only: the two-level evaluation without its bitmaps
OCM_FLAG_TEST_SMALL_BANDS = 64  # test only: the class sweep's task order in 1,024-vertex bands
OCM_FLAG_TEST_FRONTIER = 128  # test only: the frontier sweep after every evaluation but the first
OCM_FLAG_TEST_LOCAL_CHUNKS = 256     # test only: the chunked local phase in every evaluation
OCM_FLAG_TEST_NO_LOCAL_CHUNKS = 512  # test only: never the chunked local phase
OCM_SWEEP_DEFAULT, OCM_SWEEP_CLASSES, OCM_SWEEP_TILES, OCM_SWEEP_WINDOW = 0, 1, 2, 3


class OCMError(RuntimeError):
    """A negative status returned by the C ABI."""

    def __init__(self, status: int, where: str):
        lib = _native.load()
        msg = lib.ocm_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


def _mode(mode) -> int:
    if mode in (OCM_MAX, "max"):
        return OCM_MAX
    if mode in (OCM_MIN, "min"):
        return OCM_MIN
    raise ValueError(f"mode must be 'max' or 'min', got {mode!r}")


def _dev_i32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.int32:
        raise TypeError(f"{name} must be int32, got {t.dtype}")
    return t.contiguous()


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _init_policy(init_policy, n: int):
    if init_policy is None:
        return None
    t = _dev_i32(init_policy, "init_policy")
    if t.numel() != n:
        raise ValueError("init_policy needs one entry per vertex")
    return t


def _transit(transit, m: int):
    if transit is None:
        return None
    t = _dev_i32(transit, "transit")
    if t.numel() != m:
        raise ValueError("transit needs one entry per edge")
    return t


def workspace_bytes(n: int, m: int, single_lambda: bool = False) -> int:
    lib = _native.load()
    if single_lambda:
        return int(lib.ocm_workspace_size_single(n, m))
    return int(lib.ocm_workspace_size(n, m))


def make_workspace(n: int, m: int, device=None, single_lambda: bool = False) -> torch.Tensor:
    nbytes = workspace_bytes(n, m, single_lambda)
    if nbytes == 0:
        raise ValueError("graph size out of range")
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


@dataclass
class Solution:
    num: int
    den: int
    cycle: torch.Tensor               # int32 device tensor of CSR edge indices
    stats: dict = field(default_factory=dict)
    eta_num: torch.Tensor | None = None
    eta_den: torch.Tensor | None = None
    potential: torch.Tensor | None = None
    policy: torch.Tensor | None = None

    @property
    def value(self) -> Fraction:
        return Fraction(self.num, self.den)

    def __iter__(self):
        return iter((self.num, self.den, self.cycle))


def solve(row_ptr: torch.Tensor, col_idx: torch.Tensor, w: torch.Tensor, mode="max", *,
          workspace: torch.Tensor | None = None, stream=None, max_iters: int = 0,
          certificate: bool = False, cycle_out: torch.Tensor | None = None,
          flags: int = 0, edges_per_lane: int = 0, sweep_threads: int = 0,
          sweep_kind: int = 0, tune: bool = False,
          init_policy: torch.Tensor | None = None,
          transit: torch.Tensor | None = None,
          single_lambda: bool = False, wait_limit_ms: int = 0) -> Solution:
    """Optimal cycle mean of a CSR graph on the GPU (``ocm_solve``).

    Returns the exact reduced mean num/den (max or min sense) and a critical
    cycle as CSR edge indices.  With ``certificate=True`` also returns the
    per-vertex cycle means (eta_num/eta_den) and potentials of the final
    policy, in the maximising sense of s*w (s = -1 in min mode).  ``tune=True``
    uses the sweep layout and launch parameters the autotuner recorded for
    graphs of this shape (results never depend on them).  ``single_lambda``
    runs the paper's own form of the iteration (one lambda, the policy graph
    rebuilt around the chosen cycle each time); every vertex must reach that
    cycle, as in a strongly connected graph.  ``wait_limit_ms`` bounds every
    device-side wait of the call (0: two seconds)."""
    lib = _native.load()
    rp = _dev_i32(row_ptr, "row_ptr")
    col = _dev_i32(col_idx, "col_idx")
    ww = _dev_i32(w, "w")
    n, m = rp.numel() - 1, col.numel()
    if ww.numel() != m:
        raise ValueError("w and col_idx must have the same length")
    dev = rp.device
    if single_lambda:
        flags = int(flags) | OCM_FLAG_SINGLE_LAMBDA
    if workspace is None:
        workspace = make_workspace(n, m, dev, bool(int(flags) & OCM_FLAG_SINGLE_LAMBDA))
    if cycle_out is None:
        cycle_out = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    opt = _native.OcmOptions()
    opt.max_iters = int(max_iters)
    opt.flags = int(flags)
    opt.wait_limit_ms = int(wait_limit_ms)
    if tune and not (edges_per_lane or sweep_threads or sweep_kind):
        from .autotune import lookup
        found = lookup(rp)
        if found:
            sweep_kind, edges_per_lane, sweep_threads = found
    opt.edges_per_lane = int(edges_per_lane)
    opt.sweep_threads = int(sweep_threads)
    opt.sweep_kind = int(sweep_kind)
    init = _init_policy(init_policy, n)
    if init is not None:
        opt.init_policy = init.data_ptr()
    tt = _transit(transit, m)
    if tt is not None:
        opt.transit = tt.data_ptr()
    extra = {}
    if certificate:
        extra = dict(eta_num=torch.empty(n, dtype=torch.int64, device=dev),
                     eta_den=torch.empty(n, dtype=torch.int32, device=dev),
                     potential=torch.empty(n, dtype=torch.int64, device=dev),
                     policy=torch.empty(n, dtype=torch.int32, device=dev))
        for k, t in extra.items():
            setattr(opt, k, t.data_ptr())
    num = ctypes.c_int64(0)
    den = ctypes.c_int32(0)
    clen = ctypes.c_int32(0)
    st = _native.OcmStats()
    rc = lib.ocm_solve(rp.data_ptr(), col.data_ptr(), ww.data_ptr(), n, m, _mode(mode),
                       ctypes.byref(num), ctypes.byref(den), cycle_out.data_ptr(),
                       ctypes.byref(clen), workspace.data_ptr(), workspace.numel(),
                       _stream_ptr(stream), ctypes.byref(opt), ctypes.byref(st))
    if rc != 0:
        raise OCMError(rc, "ocm_solve")
    return Solution(int(num.value), int(den.value), cycle_out[:int(clen.value)], st.as_dict(),
                    **extra)


@dataclass
class BatchSolution:
    num: torch.Tensor          # int64 [G]
    den: torch.Tensor          # int32 [G]
    cycle_len: torch.Tensor    # int32 [G]
    cycle_out: torch.Tensor    # int32 [N]; graph g's cycle at graph_vptr[g]
    graph_vptr: torch.Tensor   # int32 [G+1]
    stats: dict = field(default_factory=dict)

    def cycle(self, g: int) -> torch.Tensor:
        start = int(self.graph_vptr[g])
        return self.cycle_out[start:start + int(self.cycle_len[g])]


def workspace_bytes_batch(G: int, N: int, M: int) -> int:
    return int(_native.load().ocm_workspace_size_batch(G, N, M))


def solve_batch(graph_vptr: torch.Tensor, row_ptr: torch.Tensor, col_idx: torch.Tensor,
                w: torch.Tensor, mode="max", *, workspace: torch.Tensor | None = None,
                stream=None, max_iters: int = 0, flags: int = 0,
                init_policy: torch.Tensor | None = None,
                transit: torch.Tensor | None = None, wait_limit_ms: int = 0,
                small_vertices: int = 0, sweep_kind: int = 0, edges_per_lane: int = 0,
                sweep_threads: int = 0, tune: bool = False) -> BatchSolution:
    """Optimal cycle means of G graphs given as one disjoint-union CSR
    (``ocm_solve_batch``); each result equals solving that graph alone.
    ``init_policy`` (int32 [N], global edge ids) warm-starts every graph;
    ``transit`` (int32 [M]) gives optimal cycle ratios.  Graphs with at most
    ``small_vertices`` vertices (0: the library default, < 0: none) are solved
    one per thread block by the persistent per-graph kernel.  ``tune=True``
    uses the split and sweep launch parameters that
    :func:`paper_1111_0627_gb300.autotune.tune_batch` recorded for batches of
    this shape (results never depend on them)."""
    lib = _native.load()
    vp = _dev_i32(graph_vptr, "graph_vptr")
    rp = _dev_i32(row_ptr, "row_ptr")
    col = _dev_i32(col_idx, "col_idx")
    ww = _dev_i32(w, "w")
    G, N, M = vp.numel() - 1, rp.numel() - 1, col.numel()
    dev = rp.device
    if workspace is None:
        nbytes = workspace_bytes_batch(G, N, M)
        if nbytes == 0:
            raise ValueError("batch size out of range")
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    num = torch.empty(G, dtype=torch.int64, device=dev)
    den = torch.empty(G, dtype=torch.int32, device=dev)
    clen = torch.empty(G, dtype=torch.int32, device=dev)
    cyc = torch.empty(N, dtype=torch.int32, device=dev)
    opt = _native.OcmOptions()
    opt.max_iters = int(max_iters)
    opt.flags = int(flags)
    opt.wait_limit_ms = int(wait_limit_ms)
    if tune and not (small_vertices or sweep_kind or edges_per_lane or sweep_threads):
        from .autotune import lookup_batch
        found = lookup_batch(vp, rp)
        if found:
            small_vertices, sweep_kind, edges_per_lane, sweep_threads = found
    opt.batch_small_vertices = int(small_vertices)
    opt.sweep_kind = int(sweep_kind)
    opt.edges_per_lane = int(edges_per_lane)
    opt.sweep_threads = int(sweep_threads)
    init = _init_policy(init_policy, N)
    if init is not None:
        opt.init_policy = init.data_ptr()
    tt = _transit(transit, M)
    if tt is not None:
        opt.transit = tt.data_ptr()
    st = _native.OcmStats()
    rc = lib.ocm_solve_batch(vp.data_ptr(), rp.data_ptr(), col.data_ptr(), ww.data_ptr(), G, N, M,
                             _mode(mode), num.data_ptr(), den.data_ptr(), clen.data_ptr(),
                             cyc.data_ptr(), workspace.data_ptr(), workspace.numel(),
                             _stream_ptr(stream), ctypes.byref(opt), ctypes.byref(st))
    if rc != 0:
        raise OCMError(rc, "ocm_solve_batch")
    return BatchSolution(num, den, clen, cyc, vp, st.as_dict())


def scc(row_ptr: torch.Tensor, col_idx: torch.Tensor, *, workspace: torch.Tensor | None = None,
        stream=None) -> tuple[torch.Tensor, int]:
    """Strongly connected components (``ocm_scc``): int32 labels, label = the
    smallest vertex of the component, and the number of components."""
    lib = _native.load()
    rp = _dev_i32(row_ptr, "row_ptr")
    col = _dev_i32(col_idx, "col_idx")
    n, m = rp.numel() - 1, col.numel()
    if workspace is None:
        nbytes = int(lib.ocm_workspace_size_scc(n, m))
        if nbytes == 0:
            raise ValueError("graph size out of range")
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=rp.device)
    labels = torch.empty(n, dtype=torch.int32, device=rp.device)
    count = ctypes.c_int32(0)
    rc = lib.ocm_scc(rp.data_ptr(), col.data_ptr(), n, m, labels.data_ptr(), ctypes.byref(count),
                     workspace.data_ptr(), workspace.numel(), _stream_ptr(stream))
    if rc != 0:
        raise OCMError(rc, "ocm_scc")
    return labels, int(count.value)


@dataclass
class SccSolution:
    labels: torch.Tensor       # int32 [n]: smallest vertex of each vertex's component
    root: torch.Tensor         # int32 [G]: smallest vertex of each component with a cycle
    num: torch.Tensor          # int64 [G]
    den: torch.Tensor          # int32 [G]
    cycle_len: torch.Tensor    # int32 [G]
    offsets: torch.Tensor      # int32 [G+1]
    cycle_out: torch.Tensor    # int32: component c's cycle at offsets[c]
    stats: dict = field(default_factory=dict)

    def cycle(self, c: int) -> torch.Tensor:
        start = int(self.offsets[c])
        return self.cycle_out[start:start + int(self.cycle_len[c])]


def solve_scc(row_ptr: torch.Tensor, col_idx: torch.Tensor, w: torch.Tensor, mode="max", *,
              workspace: torch.Tensor | None = None, stream=None, max_iters: int = 0,
              flags: int = 0) -> SccSolution:
    """Optimal cycle mean of every strongly connected component that holds a
    cycle (``ocm_solve_scc``); vertices without out-edges are allowed."""
    lib = _native.load()
    rp = _dev_i32(row_ptr, "row_ptr")
    col = _dev_i32(col_idx, "col_idx")
    ww = _dev_i32(w, "w")
    n, m = rp.numel() - 1, col.numel()
    if ww.numel() != m:
        raise ValueError("w and col_idx must have the same length")
    dev = rp.device
    if workspace is None:
        nbytes = int(lib.ocm_workspace_size_solve_scc(n, m))
        if nbytes == 0:
            raise ValueError("graph size out of range")
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    root = torch.empty(n, dtype=torch.int32, device=dev)
    off = torch.empty(n + 1, dtype=torch.int32, device=dev)
    num = torch.empty(n, dtype=torch.int64, device=dev)
    den = torch.empty(n, dtype=torch.int32, device=dev)
    clen = torch.empty(n, dtype=torch.int32, device=dev)
    cyc = torch.empty(n, dtype=torch.int32, device=dev)
    G = ctypes.c_int32(0)
    opt = _native.OcmOptions()
    opt.max_iters = int(max_iters)
    opt.flags = int(flags)
    st = _native.OcmStats()
    rc = lib.ocm_solve_scc(rp.data_ptr(), col.data_ptr(), ww.data_ptr(), n, m, _mode(mode),
                           labels.data_ptr(), ctypes.byref(G), root.data_ptr(), off.data_ptr(),
                           num.data_ptr(), den.data_ptr(), clen.data_ptr(), cyc.data_ptr(),
                           workspace.data_ptr(), workspace.numel(), _stream_ptr(stream),
                           ctypes.byref(opt), ctypes.byref(st))
    if rc != 0:
        raise OCMError(rc, "ocm_solve_scc")
    g = int(G.value)
    return SccSolution(labels, root[:g], num[:g], den[:g], clen[:g], off[:g + 1], cyc,
                       st.as_dict())


def backward(cycle: torch.Tensor, grad_lambda: torch.Tensor, m: int, *, stream=None,
             out: torch.Tensor | None = None, transit: torch.Tensor | None = None) -> torch.Tensor:
    """d lambda*/d w scaled by grad_lambda (``ocm_backward``, or
    ``ocm_backward_ratio`` for an optimal cycle ratio solved with ``transit``);
    float32 [m]."""
    lib = _native.load()
    cyc = _dev_i32(cycle, "cycle")
    gl = grad_lambda.reshape(1).to(dtype=torch.float32).contiguous()
    if out is None:
        out = torch.empty(m, dtype=torch.float32, device=cyc.device)
    tt = _transit(transit, m)
    if tt is not None:
        rc = lib.ocm_backward_ratio(cyc.data_ptr(), cyc.numel(), tt.data_ptr(), gl.data_ptr(), m,
                                    out.data_ptr(), _stream_ptr(stream))
    else:
        rc = lib.ocm_backward(cyc.data_ptr(), cyc.numel(), gl.data_ptr(), m, out.data_ptr(),
                              _stream_ptr(stream))
    if rc != 0:
        raise OCMError(rc, "ocm_backward")
    return out


def backward_batch(sol: "BatchSolution", grad_lambda: torch.Tensor, M: int, *, stream=None,
                   out: torch.Tensor | None = None) -> torch.Tensor:
    """Per-graph d lambda*_g/d w scaled by grad_lambda[g] (``ocm_backward_batch``)."""
    lib = _native.load()
    gl = grad_lambda.reshape(-1).to(dtype=torch.float32).contiguous()
    G = sol.graph_vptr.numel() - 1
    if gl.numel() != G:
        raise ValueError("grad_lambda needs one entry per graph")
    if out is None:
        out = torch.empty(M, dtype=torch.float32, device=sol.cycle_out.device)
    rc = lib.ocm_backward_batch(sol.graph_vptr.data_ptr(), sol.cycle_out.data_ptr(),
                                sol.cycle_len.data_ptr(), gl.data_ptr(), G, M, out.data_ptr(),
                                _stream_ptr(stream))
    if rc != 0:
        raise OCMError(rc, "ocm_backward_batch")
    return out


class OCMFunction(torch.autograd.Function):
    """lambda*(w) as a differentiable function of the edge weights.

    forward(w_float, row_ptr, col_idx, w_int, mode, transit) -> lambda* (float32 scalar)
    ``w_float`` is the float view of the weights that receives the gradient;
    the solve itself uses the exact int32 weights ``w_int``.  The gradient is
    1/|C*| on the edges of the critical cycle C* (1/t(C*) for an optimal cycle
    ratio with transit times ``transit``) and 0 elsewhere, which is the
    derivative wherever C* is the unique optimal cycle."""

    @staticmethod
    def forward(ctx, w_float, row_ptr, col_idx, w_int, mode="max", transit=None):
        sol = solve(row_ptr, col_idx, w_int, mode, transit=transit)
        ctx.save_for_backward(sol.cycle)
        ctx.m = col_idx.numel()
        ctx.transit = transit
        return torch.tensor(sol.num / sol.den, dtype=torch.float32, device=w_float.device)

    @staticmethod
    def backward(ctx, grad_out):
        (cycle,) = ctx.saved_tensors
        g = backward(cycle, grad_out, ctx.m, transit=ctx.transit)
        return g, None, None, None, None, None
