"""Every planted mistake in the oracle must fail at least one pin.

oracle.c compiles a known mistake when built with ORACLE_MUTANT=k (a
flipped twiddle sign, a dropped term, an index off by one, swapped
real/imaginary parts, a wrong butterfly sign, a skipped reordering, a
forgotten twiddle stride, wrong generator bits or counter, a conjugated
or truncated sampled-mode twiddle, a mis-reduced octant or quadrant).
The mutants are built into a temporary directory; the shipped library is
always built with ORACLE_MUTANT=0.
"""
import numpy as np
import pytest

import oracle
from oracle_pins import ALL_PINS

MUTANTS = [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 13, 14]


@pytest.mark.parametrize("mutant", MUTANTS)
def test_mutant_is_caught(mutant, tmp_path):
    o = oracle.Oracle(mutant=mutant, outdir=str(tmp_path))
    assert o._lib.oracle_mutant() == mutant
    caught = []
    for pin in ALL_PINS:
        try:
            pin(o)
        except (AssertionError, ValueError):
            caught.append(pin.__name__)
            break
    assert caught, f"mutant {mutant} passed every pin"


def test_real_oracle_is_not_a_mutant(orc):
    assert orc._lib.oracle_mutant() == 0


# Planted mistakes in the oracle's perm packing (Eq. 3), on the CPU: each
# replaces the packing or unpacking routine of a fresh oracle object.
def _pack_swapped_ends(X):
    out = oracle.Oracle.pack_perm(X)
    out[[0, 1]] = out[[1, 0]]          # R_{N/2} first
    return out


def _pack_conjugated(X):
    out = oracle.Oracle.pack_perm(X)
    out[3::2] = -out[3::2]             # I_k of the conjugate spectrum
    return out


def _pack_shifted(X):
    X = np.asarray(X, np.complex128)
    return oracle.Oracle.pack_perm(np.roll(X, -1))  # off by one bin


def _unpack_mirror_off_by_one(p):
    F = oracle.Oracle.unpack_perm(p)
    N = F.size
    F[N // 2 + 1:] = np.conj(F[:N // 2 - 1][::-1])  # F[N-k] from F[k-1]
    return F


@pytest.mark.parametrize("mistake", [("pack_perm", _pack_swapped_ends), ("pack_perm", _pack_conjugated),
                                     ("pack_perm", _pack_shifted), ("unpack_perm", _unpack_mirror_off_by_one)],
                         ids=["swapped-ends", "conjugated", "shifted", "mirror-off-by-one"])
def test_perm_mistake_is_caught(orc, mistake):
    name, fn = mistake
    o = oracle.Oracle()
    setattr(o, name, fn)
    caught = False
    for pin in ALL_PINS:
        if "real" not in pin.__name__:
            continue
        try:
            pin(o)
        except AssertionError:
            caught = True
            break
    assert caught, f"perm mistake {fn.__name__} passed every real-data pin"


# Planted mistakes in the oracle's M-way decimation, on the CPU.
def _mixed_variant(kind):
    def dft_mixed(self, x, sign=-1):
        x = np.ascontiguousarray(np.asarray(x, np.complex128))
        N = x.size
        P = N & -N
        M = N // P
        if kind == "blocks":      # contiguous blocks instead of every M-th sample
            Y = [self.dft(x[r * P:(r + 1) * P], sign) for r in range(M)]
        else:
            Y = [self.dft(x[r::M], sign) for r in range(M)]
        k = np.arange(N, dtype=np.int64)
        X = np.zeros(N, np.complex128)
        for r in range(M):
            kk = (k % P) if kind == "phase-mod-P" else k
            sg = -sign if kind == "sign" else sign
            ang = 2.0 * np.pi * ((r * kk) % N) / N
            X += (np.cos(ang) + 1j * sg * np.sin(ang)) * Y[r][k % P]
        return X
    return dft_mixed


@pytest.mark.parametrize("kind", ["blocks", "phase-mod-P", "sign"])
def test_mixed_mistake_is_caught(orc, kind):
    import types
    o = oracle.Oracle()
    o.dft_mixed = types.MethodType(_mixed_variant(kind), o)
    caught = False
    for pin in ALL_PINS:
        if "mixed" not in pin.__name__:
            continue
        try:
            pin(o)
        except AssertionError:
            caught = True
            break
    assert caught, f"mixed-radix mistake {kind} passed every pin"


# Planted mistakes in the accuracy metric (Eq. 9), on the CPU: each replaces
# rel_l2 on a fresh oracle object and must fail a metric pin.
def _norms(F, Fe):
    F = np.asarray(F, np.complex128)
    Fe = np.asarray(Fe, np.complex128)
    return np.sum(np.abs(F - Fe) ** 2), np.sum(np.abs(Fe) ** 2), np.sum(np.abs(F) ** 2)


def _rel_squared(F, Fe):          # the ratio of the squared norms
    d, e, _ = _norms(F, Fe)
    return float(d / e)


def _rel_no_sqrt_num(F, Fe):      # sqrt dropped in the numerator
    d, e, _ = _norms(F, Fe)
    return float(d / np.sqrt(e))


def _rel_norm_of_F(F, Fe):        # normalised by ||F|| instead of ||Fe||
    d, _, f = _norms(F, Fe)
    return float(np.sqrt(d) / np.sqrt(f)) if f > 0 else float("inf")


def _rel_real_part(F, Fe):        # (F - Fe)^2 read on the real parts only
    F = np.asarray(F, np.complex128)
    Fe = np.asarray(Fe, np.complex128)
    return float(np.sqrt(np.sum((F.real - Fe.real) ** 2)) / np.sqrt(np.sum(Fe.real ** 2) + 1e-300))


def _rel_unscaled(F, Fe):         # no scaling: overflows / underflows near 1e+-300
    d, e, _ = _norms(F, Fe)
    return float(np.sqrt(d) / np.sqrt(e)) if e > 0 else float(np.sqrt(d))


@pytest.mark.parametrize("fn", [_rel_squared, _rel_no_sqrt_num, _rel_norm_of_F, _rel_real_part, _rel_unscaled],
                         ids=["squared", "no-sqrt", "norm-of-F", "real-part", "unscaled"])
def test_metric_mistake_is_caught(orc, fn):
    o = oracle.Oracle()
    o.rel_l2 = fn
    caught = False
    for pin in ALL_PINS:
        if "rel_l2" not in pin.__name__:
            continue
        try:
            with np.errstate(all="ignore"):
                pin(o)
        except AssertionError:
            caught = True
            break
    assert caught, f"metric mistake {fn.__name__} passed every pin"
