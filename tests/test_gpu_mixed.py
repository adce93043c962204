"""N = M * 2^e (M odd <= 15, the paper's size set of Sec. 2.1) against the
oracle (direct sum of Eq. 1 up to 4096 points, the M-way decimation above).

Tolerances as for powers of two, with log2 N rounded up."""
import numpy as np
import pytest

import oracle
from parity_util import TOL, host_input

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ODDS = (3, 5, 7, 9, 11, 13, 15)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _code(name):
    import paper_1409_5757_gb300 as efft
    return efft.EFFT_C128 if name == "c128" else efft.EFFT_C64


def _gpu(x, name, sign=-1, flags=0):
    import paper_1409_5757_gb300 as efft
    t = torch.from_numpy(x.astype(np.complex128 if name == "c128" else np.complex64)).cuda()
    p = efft.Plan(x.size, _code(name), sign, flags)
    p.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128), p


def _check(got, ref, name, N, what=""):
    err = oracle.rel_l2(got, ref)
    lim = TOL[name] * max(np.ceil(np.log2(N)), 1)
    assert err <= lim, f"{what} {name} N={N}: rel-L2 {err:.3e} > {lim:.3e}"
    return err


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("M", ODDS)
@pytest.mark.parametrize("e", [0, 1, 2, 3, 5, 8, 9, 11, 12, 14, 17, 20])
def test_mixed_sizes(orc, name, M, e):
    N = M << e
    if N > (1 << 22):
        pytest.skip("size covered by the large test")
    x = host_input(orc, name, N, seed=7000 + 31 * M + e)
    got, _ = _gpu(x, name, -1)
    _check(got, orc.dft(x, -1), name, N)


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("N", [3 * 4096, 5 << 15, 15 << 16])
def test_mixed_inverse_sign(orc, name, N):
    x = host_input(orc, name, N, seed=N)
    got, _ = _gpu(x, name, +1)
    _check(got, orc.dft(x, +1), name, N, "sign +1")


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("N", [3 << 14, 7 << 16, 9 << 13])
def test_mixed_digit_reversed(orc, name, N):
    """Three passes (A, B, A): position q0*B*A + q1*A + q2 holds
    X[q0 + A q1 + A B q2] (A = 2^radices[0], B = N / A^2)."""
    import paper_1409_5757_gb300 as efft
    x = host_input(orc, name, N, seed=3)
    got, p = _gpu(x, name, -1, efft.EFFT_FLAG_DIGIT_REVERSED_OUT)
    r = p.radices()
    assert len(r) == 3 and r[0] == r[2]
    A = 1 << r[0]
    B = N // (A * A)
    assert A * B * A == N and B % (1 << r[1]) == 0
    P = np.arange(N)
    q0, q1, q2 = P // (B * A), (P // A) % B, P % A
    X = orc.dft(x, -1)
    _check(got, X[q0 + A * q1 + A * B * q2], name, N, "digit-reversed")


@pytest.mark.parametrize("name,N", [("c128", 3 << 24), ("c64", 5 << 24), ("c128", 15 << 20)])
def test_mixed_large(orc, name, N):
    x = host_input(orc, name, N, seed=11)
    got, _ = _gpu(x, name, -1)
    _check(got, orc.dft(x, -1), name, N, "large")


@pytest.mark.parametrize("name,N,a", [("c128", 5 << 20, 8), ("c64", 11 << 20, 8), ("c128", 9 << 22, 9),
                                      ("c64", 13 << 22, 9), ("c64", 3 << 26, 10)])
def test_mixed_outer_passes_on_specialised_kernels(orc, name, N, a):
    """(2^a, M 2^b, 2^a) with a in 8..11: the outer passes run on the
    power-of-two pass kernels (first pass at stride M * 2^(e-a)), the middle
    one on the mixed-radix kernel; both signs against the full oracle."""
    import paper_1409_5757_gb300 as efft
    assert efft.Plan(N, _code(name), -1).radices()[::2] == [a, a]
    x = host_input(orc, name, N, seed=N % 1000)
    for sign in (-1, 1):
        got, _ = _gpu(x, name, sign)
        _check(got, orc.dft(x, sign), name, N, f"sign {sign}")


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("e,a", [(10, 3), (12, 4), (13, 4), (14, 4), (17, 6), (20, 7), (24, 9)])
def test_mixed_two_stage_middle_pass(orc, name, e, a):
    """N = 3 * 2^e on the explicit schedule (2^a, 3 * 2^b, 2^a), b = e - 2a in
    4..6: the middle radices 48, 96 and 192 at strides 2^a >= 16 run the
    two-stage register kernel (radix 3 * 2^(b-4), then 16); a = 3 keeps the
    Stockham kernel.  Both signs, every element against the oracle."""
    import paper_1409_5757_gb300 as efft
    N = 3 << e
    b = e - 2 * a
    x = host_input(orc, name, N, seed=900 + e)
    for sign in (-1, 1):
        t = torch.from_numpy(x.astype(np.complex128 if name == "c128" else np.complex64)).cuda()
        p = efft.Plan(N, _code(name), sign, 0, radices=[a, b, a])
        assert p.radices() == [a, b, a]
        p.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        _check(t.cpu().numpy().astype(np.complex128), orc.dft(x, sign), name, N, f"(a={a}, b={b}) sign {sign}")


def test_mixed_extreme_magnitudes_and_nan(orc):
    N = 3 << 12
    x = orc.gen_uniform(4, N)
    for scale in (1e-300, 1e300):
        got, _ = _gpu(x * scale, "c128", -1)
        _check(got, orc.dft(x, -1) * scale, "c128", N, f"scale {scale}")
    y = x.copy()
    y[17] = np.nan
    got, _ = _gpu(y, "c128", -1)
    assert np.all(np.isnan(got.real))


def test_mixed_round_trip(orc):
    import paper_1409_5757_gb300 as efft
    for name in ("c128", "c64"):
        N = 5 << 16
        x = host_input(orc, name, N, seed=5)
        t = torch.from_numpy(x.astype(np.complex128 if name == "c128" else np.complex64)).cuda()
        efft.fft_(t, -1)
        efft.fft_(t, +1)
        got = t.cpu().numpy().astype(np.complex128) / N
        assert oracle.rel_l2(got, x) <= 2 * TOL[name] * 19


def test_mixed_batch_matches_single_plans(orc):
    import paper_1409_5757_gb300 as efft
    sizes = [3 << 10, 1 << 12, 15 << 7, 5 << 16, 3 << 10, 7, 12, 3 << 14, 3 << 17]
    xs = [host_input(orc, "c64", n, seed=40 + i) for i, n in enumerate(sizes)]
    ts = [torch.from_numpy(x.astype(np.complex64)).cuda() for x in xs]
    refs = [t.clone() for t in ts]
    efft.fft_batch_(ts)
    for r in refs:
        efft.fft_(r)
    torch.cuda.synchronize()
    for n, x, t, r in zip(sizes, xs, ts, refs):
        assert torch.equal(t, r), n
        _check(t.cpu().numpy().astype(np.complex128), orc.dft(x, -1), "c64", n, "batch")


def test_mixed_plan_rules():
    import paper_1409_5757_gb300 as efft
    with pytest.raises(efft.EfftError) as ei:
        efft.Plan(3 << 10, efft.EFFT_C128, -1, efft.EFFT_FLAG_NORMALIZE)
    assert ei.value.status == 9
    p = efft.Plan(3 << 10, efft.EFFT_C128, -1)
    scratch = torch.empty(3 << 10, dtype=torch.complex128, device="cuda")
    # the tuner scans the outer radix; of the variant knobs only the first
    # pass's tile width applies to N = M * 2^e
    res = p.autotune_candidates(scratch.data_ptr(), 0)
    assert len(res) >= 2 and all(c["radices"][0] * c["radices"][1] * c["radices"][2] == 3 << 10 for c in res)
    for knobs in ((-1, 1, -1), (-1, -1, 0), (-1, -1, -1, 1)):
        with pytest.raises(efft.EfftError) as ei:
            p.set_variant(*knobs)
        assert ei.value.status == 9
    p.set_variant(1, -1, -1)
    p.set_variant(-1, -1, -1)
    # 3 * 2^10 > 2048 points: three passes + the swap + half a sweep of range scan
    assert p.info()["hbm_passes"] == 4.5
    assert efft.Plan(3 << 8, efft.EFFT_C128, -1).info()["hbm_passes"] == 1.5  # one pass
