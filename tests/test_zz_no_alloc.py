"""efft_execute_noalloc: the transform for callers that cannot call cudaMalloc
(a framework whose pooled allocator owns all device memory, or a pipeline that
cannot afford cudaMalloc's implicit device synchronisation).

It runs the plan path's kernels with the twiddle tables and state word in a
file-scope device array of the library.  Its output must equal that of the
plan entry point (efft_plan_create + efft_execute) within the parity
tolerance of the other tests, on consecutive calls, including calls that
change N (the tables are rebuilt) and calls that reuse the previous tables.

This file is named so that pytest collects it last; it also passes alone in
a fresh process (the first call performs the per-device set-up).
"""
import ctypes

import numpy as np
import pytest

import oracle

TOL = {"c128": 1e-14, "c64": 2e-6}


def _noalloc(t, sign=-1, flags=0):
    import torch

    import paper_1409_5757_gb300 as efft
    code = efft.EFFT_C128 if t.dtype == torch.complex128 else efft.EFFT_C64
    return efft._lib().efft_execute_noalloc(ctypes.c_void_p(t.data_ptr()), t.numel(), code, sign, flags,
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_argument_checks_need_no_gpu():
    from paper_1409_5757_gb300 import build
    build.build()
    import paper_1409_5757_gb300 as efft
    L = efft._lib()
    assert L.efft_execute_noalloc(None, 1 << 25, 1, -1, 0, None) == 1   # above 2^24
    assert L.efft_execute_noalloc(None, 3, 1, -1, 0, None) == 1         # not a power of two
    assert L.efft_execute_noalloc(None, 0, 1, -1, 0, None) == 1
    assert L.efft_execute_noalloc(None, 1 << 10, 5, -1, 0, None) == 2
    assert L.efft_execute_noalloc(None, 1 << 10, 1, 2, 0, None) == 3
    assert L.efft_execute_noalloc(None, 1 << 10, 1, -1, 0x100, None) == 12


@pytest.mark.gpu
def test_noalloc_matches_plan_execute_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1409_5757_gb300 as efft
    from paper_1409_5757_gb300 import inputs

    # consecutive calls: same N twice (tables reused), then N changes (tables
    # rebuilt), both dtypes, both signs, flags, the direct-sum size, the largest
    # size and the trivial size
    calls = [("c128", 20, -1, 0), ("c128", 20, -1, 0), ("c128", 20, 1, efft.EFFT_FLAG_NORMALIZE),
             ("c64", 13, -1, 0), ("c128", 13, 1, 0), ("c128", 3, -1, 0), ("c64", 24, -1, 0),
             ("c128", 24, -1, efft.EFFT_FLAG_DIGIT_REVERSED_OUT), ("c128", 0, -1, 0), ("c128", 17, -1, 0)]
    for i, (name, e, sign, flags) in enumerate(calls):
        N = 1 << e
        dt = torch.complex128 if name == "c128" else torch.complex64
        x = torch.empty(N, dtype=dt, device="cuda")
        inputs.fill_uniform(x, seed=500 + i)
        y = x.clone()
        plan = efft.Plan(N, efft.EFFT_C128 if name == "c128" else efft.EFFT_C64, sign, flags)
        plan.execute(x.data_ptr(), torch.cuda.current_stream().cuda_stream)
        rc = _noalloc(y, sign, flags)
        assert rc == 0, (i, rc)
        torch.cuda.synchronize()
        a = x.cpu().numpy().astype(np.complex128)
        b = y.cpu().numpy().astype(np.complex128)
        err = oracle.rel_l2(b, a)
        assert err <= TOL[name] * max(e, 1), (i, name, e, err)
        plan.destroy()


@pytest.mark.gpu
def test_noalloc_rejects_bad_buffers_and_sizes():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1409_5757_gb300 as efft
    L = efft._lib()
    big = 1 << 25
    t = torch.zeros(16, dtype=torch.complex128, device="cuda")
    assert L.efft_execute_noalloc(ctypes.c_void_p(t.data_ptr()), big, 1, -1, 0, None) == 1
    h = torch.zeros(1024, dtype=torch.complex128)
    assert L.efft_execute_noalloc(ctypes.c_void_p(h.data_ptr()), 1024, 1, -1, 0, None) == 4
    assert L.efft_execute_noalloc(ctypes.c_void_p(t.data_ptr() + 8), 8, 1, -1, 0, None) == 5


def _plan_result(x, sign, flags):
    """The plan entry point's output for x (on a copy)."""
    import torch

    import paper_1409_5757_gb300 as efft
    code = efft.EFFT_C128 if x.dtype == torch.complex128 else efft.EFFT_C64
    y = x.clone()
    plan = efft.Plan(x.numel(), code, sign, flags)
    plan.execute(y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    plan.destroy()
    return y.cpu().numpy().astype(np.complex128)


@pytest.mark.gpu
def test_noalloc_leaves_free_device_memory_unchanged():
    """The entry point's promise: after one warm-up call per variant (the
    first launch of a kernel may load its code), a run of calls at several N
    changes the device's free memory by nothing."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_5757_gb300 import inputs
    variants = [("c128", 20, -1), ("c64", 16, 1), ("c128", 11, 1), ("c64", 24, -1), ("c128", 2, -1)]
    bufs = []
    for i, (name, e, sign) in enumerate(variants):
        dt = torch.complex128 if name == "c128" else torch.complex64
        x = torch.empty(1 << e, dtype=dt, device="cuda")
        inputs.fill_uniform(x, seed=900 + i)
        bufs.append((x, sign))
    for x, sign in bufs:  # warm-up: every kernel variant launched once
        assert _noalloc(x, sign) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for x, sign in bufs:
            assert _noalloc(x, sign) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


@pytest.mark.gpu
def test_noalloc_captured_call_regenerates_its_tables():
    """A call captured into a CUDA graph with an N the array does not hold:
    an eager call with that N made before the graph is launched must not
    trust tables the capture never wrote, and the graph, launched after calls
    with other N, regenerates its own.  Both are compared with the plan entry
    point."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_5757_gb300 import inputs
    # the array holds 2^14 tables before the capture
    w = torch.empty(1 << 14, dtype=torch.complex128, device="cuda")
    inputs.fill_uniform(w, seed=951)
    assert _noalloc(w, -1) == 0
    torch.cuda.synchronize()
    N, e = 1 << 18, 18
    xg = torch.empty(N, dtype=torch.complex128, device="cuda")
    inputs.fill_uniform(xg, seed=952)
    want_g = _plan_result(xg, -1, 0)
    xe = torch.empty(N, dtype=torch.complex128, device="cuda")
    inputs.fill_uniform(xe, seed=953)
    want_e = _plan_result(xe, -1, 0)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
            rc_capture = _noalloc(xg, -1)
    assert rc_capture == 0
    torch.cuda.synchronize()
    # eager call with the captured N before the graph ever ran
    assert _noalloc(xe, -1) == 0
    torch.cuda.synchronize()
    assert oracle.rel_l2(xe.cpu().numpy(), want_e) <= TOL["c128"] * e
    # another N in between, then the graph
    assert _noalloc(w, +1) == 0
    g.replay()
    torch.cuda.synchronize()
    assert oracle.rel_l2(xg.cpu().numpy(), want_g) <= TOL["c128"] * e
    del g
