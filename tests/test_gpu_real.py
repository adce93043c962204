"""Real-data transforms (the perm layout of Eq. 3, Sec. 2.1; the in-place
mirrored pairs of Sec. 3.4) against the oracle's rdft_perm / irdft_perm.

Tolerances as for complex data: relative L2 error over the N reals of the
perm array <= 1e-14 * log2 N (float64 data), 2e-6 * log2 N (float32 data,
against the FP64 oracle on the float32-rounded input)."""
import numpy as np
import pytest

import oracle
from parity_util import TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _tdt(name):
    return torch.float64 if name == "c128" else torch.float32


def _real_input(orc, name, N, seed):
    x = orc.gen_uniform(seed, N // 2).view(np.float64).copy()  # N uniform[-1,1) reals
    if name == "c64":
        x = x.astype(np.float32).astype(np.float64)
    return x


def _check(got, ref, name, N, what=""):
    err = oracle.rel_l2(got.astype(np.complex128), ref.astype(np.complex128))
    lim = TOL[name] * max(np.log2(N), 1)
    assert err <= lim, f"{what} {name} N={N}: rel-L2 {err:.3e} > {lim:.3e}"
    s = float(np.max(np.abs(ref))) if ref.size else 0.0  # scale first: magnitudes up to 1e300
    if s > 0 and np.isfinite(s):
        rms = np.sqrt(np.mean((ref / s) ** 2))
        assert np.max(np.abs((got - ref) / s)) <= 50 * lim * rms, f"{what} {name} N={N}: outlier"


def _run(x, name, direction, flags=0):
    import paper_1409_5757_gb300 as efft
    t = torch.from_numpy(x.astype(np.float64 if name == "c128" else np.float32)).cuda()
    p = efft.Plan.real(x.size, efft.EFFT_C128 if name == "c128" else efft.EFFT_C64, direction, flags)
    p.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64), p


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("e", list(range(1, 23)))
def test_forward_every_size(orc, name, e):
    N = 1 << e
    x = _real_input(orc, name, N, 500 + e)
    got, p = _run(x, name, -1)
    _check(got, orc.rdft_perm(x), name, N, "forward")


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("e", [1, 2, 3, 4, 7, 12, 13, 17, 20])
def test_inverse_matches_oracle(orc, name, e):
    N = 1 << e
    p = _real_input(orc, name, N, 900 + e)  # an arbitrary perm spectrum
    got, _ = _run(p, name, +1)
    _check(got, orc.irdft_perm(p), name, N, "inverse")


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("e", [1, 5, 16, 21])
def test_round_trip_normalised(orc, name, e):
    import paper_1409_5757_gb300 as efft
    N = 1 << e
    x = _real_input(orc, name, N, 77 + e)
    t = torch.from_numpy(x.astype(np.float64 if name == "c128" else np.float32)).cuda()
    efft.rfft_(t)
    efft.irfft_(t, normalize=True)
    got = t.cpu().numpy().astype(np.float64)
    assert oracle.rel_l2(got.astype(np.complex128), x.astype(np.complex128)) <= 2 * TOL[name] * e


@pytest.mark.parametrize("name", ["c128", "c64"])
def test_forward_normalised(orc, name):
    import paper_1409_5757_gb300 as efft
    N = 1 << 14
    x = _real_input(orc, name, N, 3)
    got, _ = _run(x, name, -1, efft.EFFT_FLAG_NORMALIZE)
    _check(got, orc.rdft_perm(x) / N, name, N, "normalised")


REAL_MIXED = [6, 10, 14, 18, 22, 26, 30, 12, 20, 3 << 5, 5 << 9, 7 << 11, 9 << 8, 11 << 10, 13 << 7,
              15 << 12, 3 << 20]


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("N", REAL_MIXED)
def test_mixed_sizes_forward_and_inverse(orc, name, N):
    """N = M * 2^e reals (the paper's size set, Sec. 2.1): the complex plan of
    N/2 = M * 2^(e-1) points, then the mirrored pairs; N/2 odd (N = 2M) has
    no self-paired slot.  Forward and inverse against the oracle."""
    x = _real_input(orc, name, N, 1300 + N % 997)
    got, _ = _run(x, name, -1)
    _check(got, orc.rdft_perm(x), name, N, "forward")
    got, _ = _run(x, name, +1)
    _check(got, orc.irdft_perm(x), name, N, "inverse")


@pytest.mark.parametrize("name", ["c128", "c64"])
def test_mixed_round_trip_and_rules(orc, name):
    import paper_1409_5757_gb300 as efft
    N = 5 << 14
    x = _real_input(orc, name, N, 41)
    t = torch.from_numpy(x.astype(np.float64 if name == "c128" else np.float32)).cuda()
    efft.rfft_(t)
    efft.irfft_(t, normalize=False)
    got = t.cpu().numpy().astype(np.float64) / N
    assert oracle.rel_l2(got.astype(np.complex128), x.astype(np.complex128)) <= 2 * TOL[name] * 17
    code = efft.EFFT_C128 if name == "c128" else efft.EFFT_C64
    with pytest.raises(efft.EfftError) as ei:
        efft.Plan.real(N, code, efft.EFFT_REAL_FORWARD, efft.EFFT_FLAG_NORMALIZE)
    assert ei.value.status == 9  # 1/N is not exact for M > 1
    with pytest.raises(efft.EfftError) as ei:
        efft.Plan.real(2 * 17, code, efft.EFFT_REAL_FORWARD)
    assert ei.value.status == 1


@pytest.mark.parametrize("name", ["c128", "c64"])
def test_closed_forms_on_gpu(name):
    """cos(2 pi f n / N) -> R_f = N/2; (-1)^n -> R_{N/2} = N; delta -> ones.
    The phase (f n mod N) is reduced in integers first: numpy's cos of the
    unreduced argument (up to ~1e4 rad) carries phase errors of ~1e-12 that
    add up coherently across n."""
    N = 1 << 12
    n = np.arange(N)
    for f in (1, 7, N // 4, N // 2 - 1):
        got, _ = _run(np.cos(2 * np.pi * ((f * n) % N) / N), name, -1)
        want = np.zeros(N)
        want[2 * f] = N / 2
        assert np.max(np.abs(got - want)) <= TOL[name] * 12 * N, f
    got, _ = _run((-1.0) ** n, name, -1)
    want = np.zeros(N)
    want[1] = N
    assert np.max(np.abs(got - want)) <= TOL[name] * 12 * N
    d = np.zeros(N)
    d[0] = 1
    got, _ = _run(d, name, -1)
    want = np.zeros(N)
    want[0] = want[1] = 1
    want[2::2] = 1
    assert np.max(np.abs(got - want)) <= TOL[name] * 12


@pytest.mark.parametrize("name,e", [("c128", 26), ("c64", 27)])
def test_large_against_full_oracle(orc, name, e):
    N = 1 << e
    x = _real_input(orc, name, N, 2600 + e)
    got, _ = _run(x, name, -1)
    _check(got, orc.rdft_perm(x), name, N, "large")


def test_c128_extreme_magnitudes_and_nan(orc):
    N = 1 << 10
    x = _real_input(orc, "c128", N, 11)
    for scale in (1e-300, 1e300):
        got, _ = _run(x * scale, "c128", -1)
        _check(got, orc.rdft_perm(x) * scale, "c128", N, f"scale {scale}")
        got, _ = _run(orc.rdft_perm(x) * scale, "c128", +1)
        _check(got, N * x * scale, "c128", N, f"inverse scale {scale}")
    y = x.copy()
    y[5] = np.nan
    got, _ = _run(y, "c128", -1)
    assert np.all(np.isnan(got))


def test_real_plan_introspection_and_host_paths(orc):
    import paper_1409_5757_gb300 as efft
    N = 1 << 20
    p = efft.Plan.real(N, efft.EFFT_C128, -1)
    inner = efft.Plan(N // 2, efft.EFFT_C128, -1)
    assert p.radices() == inner.radices()
    assert p.info()["hbm_passes"] == inner.info()["hbm_passes"] + 1.0
    x = _real_input(orc, "c128", N, 21)
    host = x.copy()
    dev = torch.empty(N, dtype=torch.float64, device="cuda")
    p.execute_host(host.ctypes.data, dev.data_ptr(), torch.cuda.current_stream().cuda_stream)
    _check(host, orc.rdft_perm(x), "c128", N, "execute_host")
    # profiling records the complex plan's launches and the pair kernel
    p.profile(True)
    p.execute(dev.data_ptr(), torch.cuda.current_stream().cuda_stream)
    prof = p.profile_read()
    p.profile(False)
    assert "real_pair" in prof and "pass0" in prof and "range_scan" in prof


def test_real_plan_autotune(orc):
    import paper_1409_5757_gb300 as efft
    N = 1 << 21
    p = efft.Plan.real(N, efft.EFFT_C64, -1)
    scratch = torch.empty(N, dtype=torch.float32, device="cuda")
    res = p.autotune(scratch.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert p.radices() == min(res, key=lambda r: r[1])[0]
    x = _real_input(orc, "c64", N, 31)
    t = torch.from_numpy(x.astype(np.float32)).cuda()
    p.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    _check(t.cpu().numpy().astype(np.float64), orc.rdft_perm(x), "c64", N, "autotuned")
