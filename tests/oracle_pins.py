"""Pins for the CPU oracle: facts fixed by the paper and by mathematics.

Each pin takes an ``oracle.Oracle`` and raises AssertionError if the oracle
disagrees with something that does not come from the oracle itself:
closed forms of Eq. 1 (Sec. 1), multiple-precision brute force (mpmath),
numpy's independent FFT, invariants of the DFT (Parseval, linearity, shift,
round trip, conjugate symmetry), and the generator's published known-answer
vector.  ``test_oracle_pins.py`` runs them on the real oracle;
``test_oracle_mutants.py`` runs them on builds with a planted mistake and
requires every mistake to fail at least one pin.
"""
from __future__ import annotations

import os

import mpmath
import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _mp_dft(x, sign, dps=40):
    """Eq. 1 evaluated term by term in mpmath at `dps` digits."""
    with mpmath.workdps(dps):
        N = len(x)
        xs = [mpmath.mpc(complex(v).real, complex(v).imag) for v in x]
        out = []
        for k in range(N):
            acc = mpmath.mpc(0)
            for n in range(N):
                acc += xs[n] * mpmath.expjpi(sign * 2 * mpmath.mpf(n * k % N) / N)
            out.append(complex(acc))
    return np.array(out, dtype=np.complex128)


def _rel(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    d = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (d if d > 0 else 1.0))


def _rng(seed):
    return np.random.default_rng(seed)


def _rand_c(n, seed):
    g = _rng(seed)
    return g.uniform(-1, 1, n) + 1j * g.uniform(-1, 1, n)


# --------------------------------------------------------------------------
# Naive DFT (Eq. 1 by direct summation)
# --------------------------------------------------------------------------
def pin_naive_impulse_at_zero(o):
    """x = delta_0 gives X[k] = 1 for every k, exactly."""
    for N in (1, 2, 3, 8, 64, 1000, 4096):
        x = np.zeros(N, np.complex128)
        x[0] = 1
        for sign in (-1, 1):
            X = o.dft_naive(x, sign)
            assert np.array_equal(X, np.ones(N)), (N, sign)


def pin_naive_shifted_impulse(o):
    """x = delta_m gives X[k] = exp(sign*2*pi*i*m*k/N) (mpmath at 40 digits)."""
    for N, m in ((8, 3), (12, 5), (64, 17), (1024, 333)):
        x = np.zeros(N, np.complex128)
        x[m] = 1
        for sign in (-1, 1):
            X = o.dft_naive(x, sign)
            with mpmath.workdps(40):
                ref = np.array([complex(mpmath.expjpi(sign * 2 * mpmath.mpf(m * k % N) / N))
                                for k in range(N)])
            assert np.max(np.abs(X - ref)) <= 2e-16, (N, m, sign, np.max(np.abs(X - ref)))


def pin_naive_constant(o):
    """x = c gives X = N*c at k = 0 and 0 elsewhere."""
    c = 0.625 - 0.375j
    for N in (7, 16, 256, 4096):
        x = np.full(N, c, np.complex128)
        for sign in (-1, 1):
            X = o.dft_naive(x, sign)
            assert abs(X[0] - N * c) <= 1e-13 * N, (N, sign)
            assert np.max(np.abs(X[1:])) <= 1e-13 * N if N > 1 else True, (N, sign)


def pin_naive_single_tone(o):
    """x_n = exp(-sign*2*pi*i*f*n/N) gives N at k = f and 0 elsewhere."""
    for N, f in ((16, 3), (100, 37), (2048, 999)):
        for sign in (-1, 1):
            with mpmath.workdps(30):
                x = np.array([complex(mpmath.expjpi(-sign * 2 * mpmath.mpf(f * n % N) / N))
                              for n in range(N)])
            X = o.dft_naive(x, sign)
            ref = np.zeros(N, np.complex128)
            ref[f] = N
            assert np.max(np.abs(X - ref)) <= 1e-12 * N, (N, f, sign)


def pin_naive_brute_force(o):
    """Random inputs, any N (not only powers of two), vs mpmath term-by-term sums."""
    for i, N in enumerate((1, 2, 3, 5, 8, 12, 16, 31, 32)):
        x = _rand_c(N, 100 + i)
        for sign in (-1, 1):
            assert _rel(o.dft_naive(x, sign), _mp_dft(x, sign)) <= 1e-15, (N, sign)


def pin_naive_vs_numpy(o):
    """Naive DFT vs numpy's pocketfft: fft for sign -1, N*ifft for sign +1."""
    for e in range(0, 11):
        N = 1 << e
        x = _rand_c(N, 200 + e)
        assert _rel(o.dft_naive(x, -1), np.fft.fft(x)) <= 1e-15 * max(e, 1), e
        assert _rel(o.dft_naive(x, 1), N * np.fft.ifft(x)) <= 1e-15 * max(e, 1), e


# --------------------------------------------------------------------------
# Radix-2 FFT (Sec. 2.2, Eqs. 4-6)
# --------------------------------------------------------------------------
def pin_radix2_vs_naive(o):
    """Radix-2 equals the direct sum for every N = 2^1 .. 2^12."""
    for e in range(1, 13):
        N = 1 << e
        x = _rand_c(N, 300 + e)
        for sign in (-1, 1):
            assert _rel(o.fft_radix2(x, sign), o.dft_naive(x, sign)) <= 1e-15 * e, (e, sign)


def pin_radix2_vs_numpy(o):
    """Radix-2 vs numpy for N up to 2^18."""
    for e in (1, 2, 3, 5, 9, 13, 16, 18):
        N = 1 << e
        x = _rand_c(N, 400 + e)
        assert _rel(o.fft_radix2(x, -1), np.fft.fft(x)) <= 1e-15 * e, e
        assert _rel(o.fft_radix2(x, 1), N * np.fft.ifft(x)) <= 1e-15 * e, e


def pin_radix2_closed_forms(o):
    """Impulse, shifted impulse, constant and tone at N = 2^16."""
    N = 1 << 16
    x = np.zeros(N, np.complex128)
    x[0] = 1
    assert np.max(np.abs(o.fft_radix2(x, -1) - 1)) <= 1e-15
    x[:] = 0.5 + 0.25j
    X = o.fft_radix2(x, -1)
    assert abs(X[0] - N * (0.5 + 0.25j)) <= 1e-12 * N and np.max(np.abs(X[1:])) <= 1e-12 * N
    m = 12345
    x[:] = 0
    x[m] = 1
    k = np.arange(N)
    with mpmath.workdps(30):
        sel = [0, 1, 7, 4096, 33333, N - 1]
        ref = np.array([complex(mpmath.expjpi(-2 * mpmath.mpf(m * kk % N) / N)) for kk in sel])
    X = o.fft_radix2(x, -1)
    assert np.max(np.abs(X[sel] - ref)) <= 1e-14
    f = 4321
    x = np.exp(2j * np.pi * ((f * k) % N) / N)
    X = o.fft_radix2(x, -1)
    ref = np.zeros(N, np.complex128)
    ref[f] = N
    assert np.max(np.abs(X - ref)) <= 1e-11 * N


def pin_radix2_invariants(o):
    """Parseval, linearity, shift theorem, round trip, real-input conjugate symmetry."""
    N = 1 << 15
    x = _rand_c(N, 500)
    y = _rand_c(N, 501)
    X = o.fft_radix2(x, -1)
    Y = o.fft_radix2(y, -1)
    # Parseval: sum |X|^2 = N sum |x|^2
    assert abs(np.sum(np.abs(X) ** 2) - N * np.sum(np.abs(x) ** 2)) <= 1e-13 * N * np.sum(np.abs(x) ** 2)
    # linearity
    a, b = 0.75 - 0.5j, -1.25 + 2j
    assert _rel(o.fft_radix2(a * x + b * y, -1), a * X + b * Y) <= 1e-14
    # shift: x[n - m] -> X[k] * exp(-2*pi*i*m*k/N)
    m = 1234
    k = np.arange(N)
    ramp = np.exp(-2j * np.pi * ((m * k) % N) / N)
    assert _rel(o.fft_radix2(np.roll(x, m), -1), X * ramp) <= 1e-13
    # round trip: F+(F-(x)) / N = x
    assert _rel(o.fft_radix2(X, 1) / N, x) <= 1e-14
    # real input: X[(N-k) mod N] = conj(X[k])  (Eq. 8 read with the index N-k)
    r = x.real.copy()
    R = o.fft_radix2(r, -1)
    assert np.max(np.abs(R[(-k) % N] - np.conj(R))) <= 1e-12 * np.sqrt(N)
    assert abs(R[0].imag) <= 1e-12 and abs(R[N // 2].imag) <= 1e-12


# --------------------------------------------------------------------------
# Twiddle factors
# --------------------------------------------------------------------------
def pin_twiddle_dyadic(o):
    """exp(-2*pi*i*m/N) at the eight octant points is known in closed form."""
    h = np.sqrt(0.5)
    known = [1, h - 1j * h, -1j, -h - 1j * h, -1, -h + 1j * h, 1j, h + 1j * h]
    for N in (8, 64, 1 << 20, 1 << 33):
        for j in range(8):
            w = o.twiddle(j * N // 8, N, -1)
            assert abs(w - known[j]) <= 1.2e-16, (N, j, w)
            w = o.twiddle(j * N // 8, N, 1)
            assert abs(w - np.conj(known[j])) <= 1.2e-16, (N, j, w)


def pin_twiddle_vs_mpmath(o):
    """Random phases m/N vs mpmath at 40 digits, to about one ulp."""
    g = _rng(7)
    for _ in range(200):
        e = int(g.integers(1, 34))
        N = 1 << e
        m = int(g.integers(0, N))
        for sign in (-1, 1):
            w = o.twiddle(m, N, sign)
            with mpmath.workdps(40):
                ref = complex(mpmath.expjpi(sign * 2 * mpmath.mpf(m) / N))
            assert abs(w - ref) <= 2.3e-16, (m, N, sign)


# --------------------------------------------------------------------------
# Input generator (published SplitMix64 definition)
# --------------------------------------------------------------------------
def _kat():
    vals = []
    with open(os.path.join(GOLDEN, "splitmix64_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            a, b = line.split()
            if a == "seed":
                seed = int(b)
            else:
                vals.append((int(a), int(b)))
    return seed, vals


def pin_rng_known_answer(o):
    """SplitMix64 reproduces the generator's published known-answer vector."""
    seed, vals = _kat()
    for i, v in vals:
        assert o.splitmix64(seed, i) == v, (i, o.splitmix64(seed, i), v)


def pin_rng_uniform_mapping(o):
    """u = top 53 bits * 2^-53 and value 2u - 1, from the known-answer outputs."""
    seed, vals = _kat()
    x = o.gen_uniform(seed, 3)
    for i, v in vals[:6]:
        n, c = divmod(i, 2)
        if n < 3:
            got = x[n].real if c == 0 else x[n].imag
            assert got == 2.0 * ((v >> 11) * 2.0 ** -53) - 1.0, (i, got)
    y = o.gen_uniform(5, 1 << 16)
    assert np.all(np.abs(y.real) <= 1) and np.all(y.real < 1) and np.all(y.imag < 1)
    assert abs(np.mean(y.real)) < 0.02 and abs(np.mean(y.imag)) < 0.02
    assert abs(np.var(y.real) - 1 / 3) < 0.01
    # windows are consistent: elements n0.. of the stream
    z = o.gen_uniform(5, 100, n0=1000)
    assert np.array_equal(z, y[1000:1100])


# --------------------------------------------------------------------------
# Sampled bins
# --------------------------------------------------------------------------
def pin_bins_vs_radix2(o):
    """Direct sums at selected k equal the full transform's entries."""
    for e in (4, 11, 14):
        N = 1 << e
        ks = np.array(sorted({0, 1, N // 2, N - 1, 5 % N, (N // 3) | 1}), np.int64)
        x = o.gen_uniform(11, N)
        for sign in (-1, 1):
            full = np.fft.fft(x) if sign == -1 else N * np.fft.ifft(x)
            scale = np.linalg.norm(full) / np.sqrt(N)
            Xb = o.dft_bins_uniform(11, N, ks, sign)
            assert np.max(np.abs(Xb - full[ks])) <= 1e-14 * scale * e, (e, sign)
            Xe = o.dft_bins(x, ks, sign)
            assert np.max(np.abs(Xe - full[ks])) <= 1e-14 * scale * e, (e, sign)


def pin_bins_tone(o):
    """A pure tone at f gives N at k = f and ~0 at other sampled bins."""
    N = 1 << 16
    f = 3001
    n = np.arange(N)
    x = np.exp(2j * np.pi * ((f * n) % N) / N)
    X = o.dft_bins(x, [f, 0, 1, 777, N - 1], -1)
    assert abs(X[0] - N) <= 1e-10 * N
    assert np.max(np.abs(X[1:])) <= 1e-10 * N


def pin_bins_any_size(o):
    """Sizes N = M * 2^e (and odd N): the sampled direct sums equal numpy's
    full transform, and a tone at f gives N at k = f."""
    for N in (7, 13 * 64, 15 << 5, 5 << 7, 3 << 9):
        e = int(np.ceil(np.log2(N)))
        ks = np.array(sorted({0, 1, N // 2, N - 1, 5 % N, N // 3}), np.int64)
        x = o.gen_uniform(11, N)
        for sign in (-1, 1):
            full = np.fft.fft(x) if sign == -1 else N * np.fft.ifft(x)
            scale = np.linalg.norm(full) / np.sqrt(N)
            Xb = o.dft_bins_uniform(11, N, ks, sign)
            assert np.max(np.abs(Xb - full[ks])) <= 1e-14 * scale * e, (N, sign)
            # negative and out-of-range frequencies are taken mod N
            Xw = o.dft_bins_uniform(11, N, np.concatenate([ks - N, ks + 3 * N]), sign)
            assert np.max(np.abs(Xw - np.concatenate([full[ks], full[ks]]))) <= 1e-14 * scale * e
    N, f = 3 << 14, 4097
    n = np.arange(N)
    X = o.dft_bins(np.exp(2j * np.pi * ((f * n) % N) / N), [f, 0, 1, N - 1, N // 3], -1)
    assert abs(X[0] - N) <= 1e-10 * N
    assert np.max(np.abs(X[1:])) <= 1e-10 * N


# --------------------------------------------------------------------------
# Real data: the perm layout of Eq. 3 (Sec. 2.1)
# --------------------------------------------------------------------------
def pin_real_perm_closed_forms(o):
    """Closed forms of Eq. 1 for real inputs (phases reduced mod N in integers),
    read through the perm layout
    {R_0, R_{N/2}, R_1, I_1, ..., R_{N/2-1}, I_{N/2-1}}:
    cos(2 pi f n / N) -> R_f = N/2; sin(2 pi f n / N) -> I_f = -N/2 (sign -1);
    delta_0 -> every R_k = 1, I_k = 0; a constant c -> R_0 = N c;
    (-1)^n -> R_{N/2} = N.  Powers of two and N = M * 2^e (N/2 odd too)."""
    for N in (2, 4, 8, 64, 1024, 8192, 6, 10, 30, 12, 96, 5 << 7, 15 << 9):
        n = np.arange(N)
        tol = 1e-14 * N
        for f in range(1, N // 2):
            if f > 5 and f < N // 2 - 3:
                continue
            want = np.zeros(N)
            want[2 * f] = N / 2
            assert np.max(np.abs(o.rdft_perm(np.cos(2 * np.pi * ((f * n) % N) / N)) - want)) <= tol, (N, f, "cos")
            want = np.zeros(N)
            want[2 * f + 1] = -N / 2
            assert np.max(np.abs(o.rdft_perm(np.sin(2 * np.pi * ((f * n) % N) / N)) - want)) <= tol, (N, f, "sin")
        d = np.zeros(N)
        d[0] = 1
        want = np.zeros(N)
        want[0] = want[1] = 1
        want[2::2] = 1
        assert np.max(np.abs(o.rdft_perm(d) - want)) <= tol, (N, "delta")
        want = np.zeros(N)
        want[0] = 0.75 * N
        assert np.max(np.abs(o.rdft_perm(np.full(N, 0.75)) - want)) <= tol, (N, "constant")
        want = np.zeros(N)
        want[1] = N
        assert np.max(np.abs(o.rdft_perm((-1.0) ** n) - want)) <= tol, (N, "alternating")


def pin_real_perm_brute_force(o):
    """mpmath's Eq. 1 on random real inputs, packed by hand into Eq. 3."""
    for N, seed in ((2, 1), (4, 2), (8, 3), (16, 4), (32, 5), (6, 6), (10, 7), (12, 8), (30, 9), (24, 10)):
        x = _rng(seed).uniform(-1, 1, N)
        X = _mp_dft(x, -1)
        want = [X[0].real, X[N // 2].real]
        for k in range(1, N // 2):
            want += [X[k].real, X[k].imag]
        assert np.max(np.abs(o.rdft_perm(x) - np.array(want))) <= 1e-14 * N, N


def pin_real_perm_round_trip(o):
    """irdft_perm(rdft_perm(x)) = N x, and the conjugate-sign inverse of a
    perm spectrum equals numpy's irfft of the same spectrum times N."""
    for N in (2, 4, 16, 256, 4096, 1 << 14, 6, 14, 30, 96, 3 << 10):
        x = _rng(N).uniform(-1, 1, N)
        assert _rel(o.irdft_perm(o.rdft_perm(x)), N * x) <= 1e-14 * np.log2(N) + 1e-16, N
        p = _rng(N + 1).uniform(-1, 1, N)
        F = np.empty(N // 2 + 1, np.complex128)
        F[0], F[N // 2] = p[0], p[1]
        F[1:N // 2] = p[2::2] + 1j * p[3::2]
        assert _rel(o.irdft_perm(p), N * np.fft.irfft(F, n=N)) <= 1e-13, N


# --------------------------------------------------------------------------
# N = M * 2^e (the paper's size set, Sec. 2.1)
# --------------------------------------------------------------------------
MIXED_SMALL = (12, 20, 24, 40, 48, 96, 3 << 10, 5 << 9, 7 << 9, 9 << 8, 15 << 8)


def pin_mixed_vs_naive(o):
    """The M-way decimation equals the direct sum of Eq. 1 (itself pinned by
    mpmath and closed forms) wherever both run."""
    for N in MIXED_SMALL:
        x = _rand_c(N, N)
        for sign in (-1, 1):
            assert _rel(o.dft_mixed(x, sign), o.dft_naive(x, sign)) <= 1e-14, (N, sign)


def pin_mixed_vs_numpy(o):
    """Against numpy's pocketfft (its own mixed-radix algorithm)."""
    for N in (3 << 14, 5 << 13, 15 << 12, 7 << 14):
        x = _rand_c(N, N + 1)
        assert _rel(o.dft(x, -1), np.fft.fft(x)) <= 1e-13, N
        assert _rel(o.dft(x, +1), np.fft.ifft(x) * N) <= 1e-13, N


def pin_mixed_closed_forms(o):
    """N = M * 2^e: an impulse at m gives exp(sign*2*pi*i*m*k/N); a tone at
    f gives N at bin f; the round trip returns N x; Parseval."""
    for N in (3 << 15, 5 << 13):
        k = np.arange(N)
        for m in (1, 7, N // 3 + 1):
            x = np.zeros(N, np.complex128)
            x[m] = 1
            want = np.exp(-2j * np.pi * ((m * k) % N) / N)
            assert np.max(np.abs(o.dft(x, -1) - want)) <= 1e-14, (N, m)
        f = N // 5 + 3
        x = np.exp(2j * np.pi * ((f * k) % N) / N)
        want = np.zeros(N, np.complex128)
        want[f] = N
        assert np.max(np.abs(o.dft(x, -1) - want)) <= 1e-12 * np.log2(N) * N ** 0.5, N
        y = _rand_c(N, 3)
        Y = o.dft(y, -1)
        assert _rel(o.dft(Y, +1), N * y) <= 1e-14 * np.log2(N), N
        assert abs(np.sum(np.abs(Y) ** 2) / (N * np.sum(np.abs(y) ** 2)) - 1) <= 1e-13, N


# --------------------------------------------------------------------------
# The accuracy metric (Eq. 9, Sec. 5.3, read with complex moduli)
# --------------------------------------------------------------------------
def pin_rel_l2_hand_values(o):
    """Values computed by hand: Fe = (3, 4i), F = (3, 1 + 4i) differ by 1 in
    one component and ||Fe|| = 5, so the error is exactly 1/5; F = 0 gives 1;
    F = Fe gives 0; a difference only in the imaginary part counts."""
    Fe = np.array([3.0, 4.0j])
    assert o.rel_l2(np.array([3.0, 1.0 + 4.0j]), Fe) == 0.2
    assert o.rel_l2(np.array([3.0, 4.0j + 1.0j]), Fe) == 0.2
    assert o.rel_l2(np.zeros(2, np.complex128), Fe) == 1.0
    assert o.rel_l2(Fe.copy(), Fe) == 0.0
    # two components off: sqrt(1^2 + 2^2) / sqrt(1 + 1 + 4 + 4) = sqrt(5/10)
    Fe2 = np.array([1.0, 1.0j, 2.0, 2.0j])
    F2 = Fe2 + np.array([1.0, 0.0, 2.0j, 0.0])
    assert abs(o.rel_l2(F2, Fe2) - np.sqrt(0.5)) <= 4e-16


def pin_rel_l2_relative_perturbation(o):
    """F = Fe (1 + delta) for one complex delta gives |delta| at any size and
    any magnitude of the values (the ratio does not depend on the scale),
    including values near the binary64 limits (1e+-300)."""
    g = _rng(11)
    for N in (1, 7, 4096):
        Fe = g.uniform(-1, 1, N) + 1j * g.uniform(-1, 1, N)
        for delta in (1e-3 * (0.6 + 0.8j), 2.5e-9j, -0.125):
            want = abs(delta)
            for scale in (1.0, 1e300, 1e-300):
                got = o.rel_l2(Fe * scale * (1 + delta), Fe * scale)
                assert abs(got - want) <= 1e-12 * want + 1e-15, (N, delta, scale, got)


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
