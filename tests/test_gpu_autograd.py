"""The adjoint (conjugate-sign unnormalised transform) behind
torch.autograd: gradients of L = sum_k |w_k X_k|^2 against the closed form
2 F^H(|w|^2 X) (F^H from the oracle's radix-2 FFT with sign +1) and against
central finite differences."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _loss(X, w2):
    return torch.sum(w2 * (X.real ** 2 + X.imag ** 2))


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("e", [6, 12, 17])
def test_grad_matches_closed_form(orc, name, e):
    from paper_1409_5757_gb300.autograd import dft
    N = 1 << e
    g = np.random.default_rng(e)
    x = orc.gen_uniform(40 + e, N)
    w = g.uniform(0, 1, N)
    if name == "c64":
        x = x.astype(np.complex64).astype(np.complex128)
    tdt = torch.complex128 if name == "c128" else torch.complex64
    rdt = torch.float64 if name == "c128" else torch.float32
    xt = torch.from_numpy(x.astype(np.complex128 if name == "c128" else np.complex64)).cuda().requires_grad_(True)
    w2 = torch.from_numpy((w ** 2).astype(np.float64)).to(rdt).cuda()
    L = _loss(dft(xt, -1), w2)
    L.backward()
    got = xt.grad.cpu().numpy().astype(np.complex128)
    X = orc.dft(x, -1)
    ref = 2 * orc.dft(w ** 2 * X, +1)
    tol = (1e-14 if name == "c128" else 2e-6) * 2 * e
    assert oracle.rel_l2(got, ref) <= tol
    assert xt.grad.dtype == tdt


@pytest.mark.parametrize("sign", [-1, 1])
def test_grad_finite_differences(orc, sign):
    from paper_1409_5757_gb300.autograd import dft
    N = 1 << 10
    x = orc.gen_uniform(77, N)
    w2 = torch.from_numpy(np.random.default_rng(3).uniform(0, 1, N) ** 2).cuda()
    xt = torch.from_numpy(x.copy()).cuda().requires_grad_(True)
    L = _loss(dft(xt, sign), w2)
    L.backward()
    grad = xt.grad.cpu().numpy()
    h = 1e-3
    for j in (0, 1, 333, N - 1):
        for unit in (1.0, 1j):
            xp = torch.from_numpy(x.copy()).cuda()
            xm = torch.from_numpy(x.copy()).cuda()
            xp[j] += unit * h
            xm[j] -= unit * h
            with torch.no_grad():
                d = (_loss(dft(xp, sign), w2) - _loss(dft(xm, sign), w2)).item() / (2 * h)
            want = grad[j].real if unit == 1.0 else grad[j].imag
            assert abs(d - want) <= 1e-7 * max(1.0, abs(want)), (j, unit, d, want)


@pytest.mark.parametrize("e", [10, 16])
def test_grad_finite_differences_c64(orc, e):
    """complex64: the gradient of the FP32 transform against central
    differences of the loss evaluated in FP64 by the oracle on the FP32
    input promoted to FP64 (h = 1e-3), within the FP32 tolerance relative to
    the gradient's RMS."""
    from paper_1409_5757_gb300.autograd import dft
    N = 1 << e
    x = orc.gen_uniform(78, N).astype(np.complex64).astype(np.complex128)
    w2 = np.random.default_rng(4).uniform(0, 1, N) ** 2
    xt = torch.from_numpy(x.astype(np.complex64)).cuda().requires_grad_(True)
    L = _loss(dft(xt, -1), torch.from_numpy(w2).float().cuda())
    L.backward()
    grad = xt.grad.cpu().numpy().astype(np.complex128)
    rms = float(np.sqrt(np.mean(np.abs(grad) ** 2)))
    h = 1e-3
    for j in (0, 1, 333, N // 2, N - 1):
        for unit in (1.0, 1j):
            xp = x.copy()
            xm = x.copy()
            xp[j] += unit * h
            xm[j] -= unit * h
            d = (np.sum(w2 * np.abs(orc.dft(xp, -1)) ** 2) - np.sum(w2 * np.abs(orc.dft(xm, -1)) ** 2)) / (2 * h)
            want = grad[j].real if unit == 1.0 else grad[j].imag
            assert abs(d - want) <= 2e-6 * 2 * e * 10 * rms, (j, unit, d, want, rms)


def test_normalised_grad(orc):
    from paper_1409_5757_gb300.autograd import dft
    N = 1 << 14
    x = orc.gen_uniform(5, N)
    xt = torch.from_numpy(x.copy()).cuda().requires_grad_(True)
    L = _loss(dft(xt, -1, normalize=True), torch.ones(N, dtype=torch.float64, device="cuda"))
    L.backward()
    # L = |F x / N|^2 = sum|x|^2 / N (Parseval), so grad = 2 x / N
    assert oracle.rel_l2(xt.grad.cpu().numpy(), 2 * x / N) <= 1e-14 * 28
