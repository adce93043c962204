"""Host-side checks of the C ABI (no GPU needed).

The libraries are compiled here (nvcc cross-compiles sm_103a without a GPU);
these tests check that every entry point declared in include/*.h is exported
and that argument validation happens before any CUDA call.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def libs():
    from paper_1409_5757_gb300 import build
    return build.build()


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(efft_[a-z_0-9]+)\s*\(", txt, flags=re.M)))


@pytest.mark.parametrize("header,lib", [("efft.h", "libefft.so"), ("efft_inputs.h", "libefft_inputs.so")])
def test_every_declared_symbol_is_exported(libs, header, lib):
    names = _declared(header)
    assert len(names) >= 4
    so = ctypes.CDLL(libs[lib])
    for n in names:
        assert hasattr(so, n), f"{lib} does not export {n}"


def test_binding_covers_header(libs):
    import paper_1409_5757_gb300 as efft
    assert set(_declared("efft.h")) == set(efft._SIGNATURES)


def test_argument_errors_before_cuda(libs):
    import paper_1409_5757_gb300 as efft
    L = efft._lib()
    h = ctypes.c_void_p()
    assert L.efft_plan_create(None, 8, 1, -1, 0) == 4                    # NULL out
    assert L.efft_plan_create(ctypes.byref(h), 0, 1, -1, 0) == 1         # N = 0
    assert L.efft_plan_create(ctypes.byref(h), 34, 1, -1, 0) == 1        # odd factor 17 > 15
    assert L.efft_plan_create(ctypes.byref(h), 3 * 1024, 1, -1, 2) == 9  # 1/N not exact for N = 3 * 2^10
    assert L.efft_plan_create(ctypes.byref(h), 1 << 34, 1, -1, 0) == 1   # too large
    assert L.efft_plan_create(ctypes.byref(h), 1 << 10, 2, -1, 0) == 2   # dtype
    assert L.efft_plan_create(ctypes.byref(h), 1 << 10, 1, 0, 0) == 3    # sign
    assert L.efft_plan_create(ctypes.byref(h), 1 << 10, 1, 1, 0x80) == 12  # flags
    assert h.value is None


def test_plan_handle_checks(libs):
    import paper_1409_5757_gb300 as efft
    L = efft._lib()
    assert L.efft_plan_destroy(None) == 0
    bogus = ctypes.create_string_buffer(256)
    assert L.efft_plan_destroy(ctypes.cast(bogus, ctypes.c_void_p)) == 10
    assert L.efft_execute(None, None, None) == 10
    assert L.efft_execute(ctypes.cast(bogus, ctypes.c_void_p), None, None) == 10
    assert L.efft_execute_host(None, None, None, None) == 10
    assert L.efft_plan_radices(None, None, 0, None) == 10
    assert L.efft_plan_info(None, None, None) == 10


def test_strerror_and_version(libs):
    import paper_1409_5757_gb300 as efft
    L = efft._lib()
    for code in list(efft.STATUS) + [99, -1]:
        s = L.efft_strerror(code)
        assert isinstance(s, bytes) and len(s) > 3
    assert L.efft_version() == 1


def test_no_cuda_device_reports_cuda_error(libs):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1409_5757_gb300 as efft
    h = ctypes.c_void_p()
    assert efft._lib().efft_plan_create(ctypes.byref(h), 1 << 10, 1, -1, 0) == 11
    with pytest.raises(efft.EfftError):
        efft.Plan(1 << 10)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_1409_5757_gb300 as efft
    monkeypatch.setattr(efft, "_LIB", None)
    monkeypatch.setattr(efft, "lib_path", lambda: str(tmp_path / "libefft.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        efft._lib()


def _planner_choice():
    """The planner's default schedule, with its three-pass table read from
    the source."""
    src = open(os.path.join(ROOT, "paper_1409_5757_gb300", "csrc", "efft.cu")).read()
    body = src[src.index("static const int kA[34] = {") + len("static const int kA[34] = {"):]
    body = body[:body.index("};")]
    kA = [int(v) for v in re.sub(r"/\*.*?\*/", "", body).replace("\n", " ").split(",")]
    assert len(kA) == 34

    def choose(e):
        if e <= 3:
            return []
        if e <= 11:
            return [e]
        if e <= 22 and e % 2 == 0:
            return [e // 2, e // 2]
        return [kA[e], e - 2 * kA[e], kA[e]]
    return choose


def test_radix_schedule_is_symmetric():
    """The planner's three-pass table gives symmetric radices, so the digit
    reversal is an involution; all radices 16..2048, and at most 2^10 rows in
    the first pass below 2^32."""
    choose = _planner_choice()
    for e in range(4, 34):
        r = choose(e)
        assert sum(r) == e and r == r[::-1] and all(4 <= x <= 11 for x in r), (e, r)
        if 28 <= e <= 31:
            assert r[0] <= 10, (e, r)


def test_arith_constants_match_mpmath():
    """The float-pair constants cos(pi/8), sin(pi/8), cos(pi/4) in the kernels
    are hi = RN32(v), lo = RN32(v - hi)."""
    import mpmath
    import numpy as np
    src = open(os.path.join(ROOT, "paper_1409_5757_gb300", "csrc", "efft_arith.cuh")).read()
    mpmath.mp.dps = 50
    want = {"K_C1": mpmath.cos(mpmath.pi / 8), "K_S1": mpmath.sin(mpmath.pi / 8), "K_R": mpmath.cos(mpmath.pi / 4)}
    for name, v in want.items():
        m = re.search(name + r"\(\) \{ return \{([-0-9.e+]+)f, ([-0-9.e+]+)f\}", src)
        assert m, name
        hi, lo = np.float32(float(m.group(1))), np.float32(float(m.group(2)))
        assert hi == np.float32(float(v))
        assert lo == np.float32(float(v - mpmath.mpf(float(hi))))


def test_schedule_and_batch_argument_errors_before_cuda(libs):
    import paper_1409_5757_gb300 as efft
    L = efft._lib()
    h = ctypes.c_void_p()

    def radices(*r):
        return (ctypes.c_int * max(len(r), 1))(*r), len(r)

    def create(n, r, flags=0):
        arr, np_ = radices(*r)
        return L.efft_plan_create_with_radices(ctypes.byref(h), n, 1, -1, flags, arr, np_)
    assert create(1 << 12, [6, 5]) == 9             # sum != log2 N
    assert create(1 << 11, [6, 5]) == 9             # not symmetric
    assert create(1 << 12, [12]) == 9               # radix above 2^11
    assert create(1 << 12, [3, 6, 3]) == 9          # radix below 2^4
    assert create(1 << 16, [4, 4, 4, 4]) == 9       # four passes
    assert create(1 << 4, []) == 9                  # N > 8 needs a pass
    assert create(1 << 3, [3]) == 9                 # N <= 8: direct sums only
    assert create(1 << 12, [6, 6], flags=0x4) == 12  # autotune with an explicit schedule
    assert create(34, [6, 6]) == 1
    # N = M * 2^e: one pass of log2 R_0 = e within 2048 points, or (a, b, a)
    assert create(12, [3]) == 9                     # log2 R_0 != e
    assert create(3 << 12, [12]) == 9               # one pass above 2048 points
    assert create(3 << 12, [4, 5, 3]) == 9          # not symmetric
    assert create(3 << 12, [0, 12, 0]) == 9         # outer radix 1
    assert create(3 << 12, [4, 5, 4]) == 9          # 2a + b != e
    assert create(3 << 26, [5, 16, 5]) == 9         # middle radix 3 * 2^16 above 2048
    assert create(3 << 12, [3, 6, 3], flags=0x4) == 12
    assert L.efft_plan_create_with_radices(None, 1 << 12, 1, -1, 0, radices(6, 6)[0], 2) == 4
    assert h.value is None

    sizes = (ctypes.c_uint64 * 3)(1 << 10, 1 << 12, 1 << 10)
    assert L.efft_batch_create(None, sizes, 3, 0, -1, 0) == 4
    assert L.efft_batch_create(ctypes.byref(h), None, 3, 0, -1, 0) == 4
    assert L.efft_batch_create(ctypes.byref(h), sizes, 0, 0, -1, 0) == 1
    assert L.efft_batch_create(ctypes.byref(h), sizes, 3, 2, -1, 0) == 2
    assert L.efft_batch_create(ctypes.byref(h), sizes, 3, 0, 0, 0) == 3
    assert L.efft_batch_create(ctypes.byref(h), sizes, 3, 0, -1, 0x80) == 12
    bad = (ctypes.c_uint64 * 2)(1 << 10, 17 << 10)
    assert L.efft_batch_create(ctypes.byref(h), bad, 2, 0, -1, 0) == 1
    big = (ctypes.c_uint64 * 1)(1 << 34)
    assert L.efft_batch_create(ctypes.byref(h), big, 1, 0, -1, 0) == 1
    assert h.value is None


def test_batch_and_autotune_handle_checks(libs):
    import paper_1409_5757_gb300 as efft
    L = efft._lib()
    bogus = ctypes.create_string_buffer(256)
    bp = ctypes.cast(bogus, ctypes.c_void_p)
    assert L.efft_batch_destroy(None) == 0
    assert L.efft_batch_destroy(bp) == 10
    assert L.efft_batch_execute(None, None, None) == 10
    assert L.efft_batch_execute(bp, None, None) == 10
    assert L.efft_batch_info(None, None, None) == 10
    assert L.efft_batch_execute_host_stream(None, 1, None, None, None, None) == 1   # no batch list
    arr = (ctypes.c_void_p * 1)(bp.value)
    assert L.efft_batch_execute_host_stream(arr, 0, None, None, None, None) == 1    # nbatches < 1
    assert L.efft_batch_execute_host_stream(arr, 1, None, None, None, None) == 10   # foreign handle
    assert L.efft_plan_autotune(None, None, None, None, None, 0, None) == 10
    assert L.efft_plan_autotune(bp, None, None, None, None, 0, None) == 10


def test_schedule_candidates_are_valid():
    """The accepted schedules of every size: the planner's own choice is one
    of them, and every one sums to log2 N, is symmetric and uses radices
    2^4..2^11."""
    import sys
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity_util import schedule_candidates
    for e in range(0, 34):
        cands = schedule_candidates(e)
        if e <= 3:
            assert cands == [[]]
            continue
        assert cands, e
        for r in cands:
            assert sum(r) == e and r == r[::-1] and all(4 <= v <= 11 for v in r), (e, r)
        assert len(cands) <= 10
        assert _planner_choice()(e) in cands, e


def test_plan_schedule_power_of_two_matches_the_planner_table(libs):
    """efft_plan_schedule (the compiled planner, no device) against the
    Python reading of its table, for every N = 2^0..2^33 and both dtypes."""
    import paper_1409_5757_gb300 as efft
    choose = _planner_choice()
    for code in (efft.EFFT_C128, efft.EFFT_C64):
        for e in range(0, 34):
            got = efft.plan_schedule(1 << e, code)
            assert got == [1 << r for r in choose(e)], (code, e, got)


def test_plan_schedule_mixed_sizes(libs):
    """N = M * 2^e: the radices multiply to N, are palindromic, only the
    middle (or only) radix carries M, the outer ones are powers of two at
    most 2^11 (complex128) / 2^10 (complex64), and the outer radix is the
    largest one that leaves the middle pass 2^b >= 16 whenever one does."""
    import paper_1409_5757_gb300 as efft
    L = efft._lib()
    for code, amax in ((efft.EFFT_C128, 11), (efft.EFFT_C64, 10)):
        for M in (3, 5, 7, 9, 11, 13, 15):
            for e in range(0, 31):
                N = M << e
                if N > (1 << 33):
                    continue
                r = efft.plan_schedule(N, code)
                prod = 1
                for v in r:
                    prod *= v
                assert prod == N, (code, N, r)
                assert r == r[::-1]
                if N <= 2048:
                    assert r == [N]
                    continue
                assert len(r) == 3 and r[0] & (r[0] - 1) == 0 and r[1] % M == 0
                a = r[0].bit_length() - 1
                feasible = [c for c in range(1, amax + 1) if 2 * c <= e and N // (1 << (2 * c)) <= 2048
                            and ((N >> (2 * c)) & -(N >> (2 * c))).bit_length() - 1 >= 4]
                if feasible:
                    assert a == max(feasible), (code, N, r, feasible)
    assert efft.plan_schedule(3 << 28, efft.EFFT_C128) == [2048, 192, 2048]
    assert efft.plan_schedule(3 << 28, efft.EFFT_C64) == [1024, 768, 1024]
    assert efft.plan_schedule(3 << 10, efft.EFFT_C128) == [8, 48, 8]
    assert efft.plan_schedule(15 << 7, efft.EFFT_C64) == [1920]
    n = ctypes.c_int()
    arr = (ctypes.c_uint64 * 4)()
    assert L.efft_plan_schedule(17, 1, arr, 4, ctypes.byref(n)) == 1     # odd factor 17
    assert L.efft_plan_schedule(0, 1, arr, 4, ctypes.byref(n)) == 1      # N = 0
    assert L.efft_plan_schedule(1 << 34, 1, arr, 4, ctypes.byref(n)) == 1
    assert L.efft_plan_schedule(1 << 10, 7, arr, 4, ctypes.byref(n)) == 2  # dtype
    assert L.efft_plan_schedule(1 << 10, 1, arr, 4, None) == 4           # npasses NULL


def test_real_plan_argument_errors_before_cuda(libs):
    import paper_1409_5757_gb300 as efft
    L = efft._lib()
    h = ctypes.c_void_p()
    assert L.efft_plan_create_real(None, 16, 1, -1, 0) == 4
    assert L.efft_plan_create_real(ctypes.byref(h), 1, 1, -1, 0) == 1        # N < 2
    assert L.efft_plan_create_real(ctypes.byref(h), 34, 1, -1, 0) == 1       # N/2 = 17: odd factor > 15
    assert L.efft_plan_create_real(ctypes.byref(h), 45, 1, -1, 0) == 1       # odd N
    assert L.efft_plan_create_real(ctypes.byref(h), 1 << 35, 1, -1, 0) == 1  # above 2^34 reals
    assert L.efft_plan_create_real(ctypes.byref(h), 16, 2, -1, 0) == 2       # precision
    assert L.efft_plan_create_real(ctypes.byref(h), 16, 1, 0, 0) == 3        # direction
    assert L.efft_plan_create_real(ctypes.byref(h), 16, 1, -1, 0x1) == 12    # digit-reversed output
    assert h.value is None
