"""ocm_solve_static: the solve for callers that cannot allocate device memory.

Such callers (a process whose device memory is capped or already handed out,
a plugin or a real-time loop that must not allocate after start-up) pass only
their inputs and outputs; the solver's scratch lives in a fixed array inside
the library.  This file is collected last on purpose, so that a failure here
comes after every other test has run.  It compares the new entry point, called
through the C ABI, with ocm_solve on the same graphs, twice in a row (the
second call reuses the array the first call left behind)."""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1111_0627_gb300 as ocm
    from paper_1111_0627_gb300 import _native

STATIC_BYTES = 32 << 20


def _static_solve(lib, rp, col, w, n, m, mode):
    num, den, clen = ctypes.c_int64(0), ctypes.c_int32(0), ctypes.c_int32(0)
    out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    st = _native.OcmStats()
    rc = lib.ocm_solve_static(rp.data_ptr(), col.data_ptr(), w.data_ptr(), n, m, mode,
                              ctypes.byref(num), ctypes.byref(den), out.data_ptr(),
                              ctypes.byref(clen), int(torch.cuda.current_stream().cuda_stream),
                              None, ctypes.byref(st))
    return rc, int(num.value), int(den.value), out[:int(clen.value)].cpu().numpy()


@pytest.mark.parametrize("make", [synth.ring10k, lambda: synth.locality32m(1 << 17),
                                  lambda: synth.batch_graphs(G=3, nmin=20000, nmax=60000)[1]],
                         ids=["ring10k", "locality_2^17", "batch_member"])
def test_static_entry_matches_ocm_solve_twice(make):
    lib = ocm.load()
    g = make()
    assert lib.ocm_workspace_size(g.n, g.m) <= STATIC_BYTES
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col_idx).cuda()
    w = torch.from_numpy(g.w).cuda()
    ref = ocm.solve(rp, col, w, g.mode)
    mode = 0 if g.mode == "max" else 1
    for call in range(2):
        rc, num, den, cyc = _static_solve(lib, rp, col, w, g.n, g.m, mode)
        assert rc == 0, (call, rc)
        # integer results: exact agreement is the tolerance
        assert (num, den) == (ref.num, ref.den), call
        assert cyc.tolist() == ref.cycle.cpu().numpy().tolist(), call


def test_static_entry_rejects_graphs_beyond_its_capacity():
    lib = ocm.load()
    n = 1 << 20                                   # needs far more than 32 MiB
    assert lib.ocm_workspace_size(n, n) > STATIC_BYTES
    d = torch.zeros(1, dtype=torch.int32, device="cuda")
    num, den, clen = ctypes.c_int64(0), ctypes.c_int32(0), ctypes.c_int32(0)
    rc = lib.ocm_solve_static(d.data_ptr(), d.data_ptr(), d.data_ptr(), n, n, 0,
                              ctypes.byref(num), ctypes.byref(den), d.data_ptr(),
                              ctypes.byref(clen), None, None, None)
    assert rc == -7      # OCM_ERR_WORKSPACE, before any device work
    assert (num.value, den.value, clen.value) == (0, 0, 0)


def test_static_entry_in_the_single_lambda_form():
    """OCM_FLAG_SINGLE_LAMBDA needs the larger workspace; the static entry
    sizes its check by the flag and gives ocm_solve's answer."""
    lib = ocm.load()
    g = synth.ring10k()
    assert lib.ocm_workspace_size_single(g.n, g.m) <= STATIC_BYTES
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col_idx).cuda()
    w = torch.from_numpy(g.w).cuda()
    ref = ocm.solve(rp, col, w, g.mode, single_lambda=True)
    opt = _native.OcmOptions()
    opt.flags = 4
    num, den, clen = ctypes.c_int64(0), ctypes.c_int32(0), ctypes.c_int32(0)
    out = torch.full((g.n,), -1, dtype=torch.int32, device="cuda")
    st = _native.OcmStats()
    rc = lib.ocm_solve_static(rp.data_ptr(), col.data_ptr(), w.data_ptr(), g.n, g.m,
                              0 if g.mode == "max" else 1, ctypes.byref(num), ctypes.byref(den),
                              out.data_ptr(), ctypes.byref(clen),
                              int(torch.cuda.current_stream().cuda_stream), ctypes.byref(opt),
                              ctypes.byref(st))
    assert rc == 0
    assert (int(num.value), int(den.value)) == (ref.num, ref.den)
    assert out[:int(clen.value)].cpu().tolist() == ref.cycle.cpu().tolist()
    assert st.iterations == ref.stats["iterations"] and st.rebuild_levels > 0


def test_static_entry_allocates_nothing_after_the_first_call():
    """The promise itself: once the array exists (the first call may load the
    library's GPU code and with it the array), a call takes no device memory.
    Free device memory is read right before and right after the C call, with
    every buffer the call uses already in place."""
    lib = ocm.load()
    g = synth.locality32m(1 << 16)
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col_idx).cuda()
    w = torch.from_numpy(g.w).cuda()
    mode = 0 if g.mode == "max" else 1
    assert _static_solve(lib, rp, col, w, g.n, g.m, mode)[0] == 0      # warm-up
    num, den, clen = ctypes.c_int64(0), ctypes.c_int32(0), ctypes.c_int32(0)
    out = torch.full((g.n,), -1, dtype=torch.int32, device="cuda")
    stream = int(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    rc = lib.ocm_solve_static(rp.data_ptr(), col.data_ptr(), w.data_ptr(), g.n, g.m, mode,
                              ctypes.byref(num), ctypes.byref(den), out.data_ptr(),
                              ctypes.byref(clen), stream, None, None)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert rc == 0
    assert free_after == free_before
