"""CPU oracle for the 1-D complex DFT (Eq. 1), as a ctypes wrapper.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline / reference legs import this package.  The product
library (paper_1409_5757_gb300) never imports it and shares no code with it.

All complex routines take and return numpy complex128 arrays (interleaved
re, im), and compute X[k] = sum_n x[n] exp(sign*2*pi*i*n*k/N) with no
normalisation.  The real-data routines (rdft_perm, irdft_perm) apply the
complex DFT to real data and pack / unpack the perm layout of Eq. 3.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_c_i64p = ctypes.POINTER(ctypes.c_int64)
_c_dp = ctypes.POINTER(ctypes.c_double)


class Oracle:
    """Handle on one build of oracle.c (mutant 0 is the real oracle)."""

    def __init__(self, mutant: int = 0, outdir: str | None = None):
        path = _build.build(mutant=mutant, outdir=outdir)
        self.path = path
        self.mutant = mutant
        lib = ctypes.CDLL(path)
        lib.oracle_version.restype = ctypes.c_int
        lib.oracle_mutant.restype = ctypes.c_int
        lib.oracle_threads.restype = ctypes.c_int
        lib.oracle_twiddle.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _c_dp, _c_dp]
        lib.oracle_dft_naive.argtypes = [_c_dp, _c_dp, ctypes.c_int64, ctypes.c_int]
        lib.oracle_dft_naive.restype = ctypes.c_int
        lib.oracle_fft_radix2.argtypes = [_c_dp, ctypes.c_int64, ctypes.c_int]
        lib.oracle_fft_radix2.restype = ctypes.c_int
        lib.oracle_gen_uniform.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, _c_dp]
        lib.oracle_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_splitmix64.restype = ctypes.c_uint64
        lib.oracle_dft_bins_uniform.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                                                _c_i64p, ctypes.c_int64, _c_dp]
        lib.oracle_dft_bins_uniform.restype = ctypes.c_int
        lib.oracle_dft_bins.argtypes = [_c_dp, ctypes.c_int64, ctypes.c_int, _c_i64p,
                                        ctypes.c_int64, _c_dp]
        lib.oracle_dft_bins.restype = ctypes.c_int
        self._lib = lib

    # -- helpers -----------------------------------------------------------
    @staticmethod
    def _c128(x) -> np.ndarray:
        return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))

    @staticmethod
    def _dp(a: np.ndarray):
        return a.ctypes.data_as(_c_dp)

    # -- API -----------------------------------------------------------------
    @property
    def version(self) -> int:
        return self._lib.oracle_version()

    @property
    def threads(self) -> int:
        return self._lib.oracle_threads()

    def twiddle(self, m: int, N: int, sign: int) -> complex:
        """exp(sign*2*pi*i*m/N) (long double, octant-reduced, rounded to double)."""
        re, im = ctypes.c_double(), ctypes.c_double()
        self._lib.oracle_twiddle(m, N, sign, ctypes.byref(re), ctypes.byref(im))
        return complex(re.value, im.value)

    def dft_naive(self, x, sign: int = -1) -> np.ndarray:
        """Direct O(N^2) evaluation of Eq. 1."""
        x = self._c128(x)
        X = np.empty_like(x)
        rc = self._lib.oracle_dft_naive(self._dp(x), self._dp(X), x.size, sign)
        if rc:
            raise ValueError(f"oracle_dft_naive failed ({rc})")
        return X

    def fft_radix2(self, x, sign: int = -1) -> np.ndarray:
        """Iterative radix-2 Cooley-Tukey (Eqs. 4-6); returns a new array."""
        X = self._c128(x).copy()
        rc = self._lib.oracle_fft_radix2(self._dp(X), X.size, sign)
        if rc:
            raise ValueError(f"oracle_fft_radix2 failed ({rc})")
        return X

    def dft(self, x, sign: int = -1) -> np.ndarray:
        """Naive DFT for N <= 4096; above, the radix-2 FFT for N a power of
        two, dft_mixed for N = M * 2^e (M odd)."""
        x = self._c128(x)
        if x.size <= 4096:
            return self.dft_naive(x, sign)
        if x.size & (x.size - 1) == 0:
            return self.fft_radix2(x, sign)
        return self.dft_mixed(x, sign)

    def dft_mixed(self, x, sign: int = -1) -> np.ndarray:
        """Eq. 1 for N = M * P, P = 2^e, M odd: the decimation identity of Eq. 4
        taken M ways instead of two,
            X[k] = sum_{r<M} exp(sign*2*pi*i*r*k/N) * Y_r[k mod P],
            Y_r = the P-point DFT of x[r], x[r+M], x[r+2M], ...
        with the Y_r from dft (radix-2 or naive) and the M-term sums
        evaluated directly; the phase r*k is reduced mod N in integers."""
        x = self._c128(x)
        N = x.size
        P = N & -N
        M = N // P
        Y = [self.dft(x[r::M], sign) for r in range(M)]
        k = np.arange(N, dtype=np.int64)
        X = np.zeros(N, dtype=np.complex128)
        for r in range(M):
            ang = 2.0 * np.pi * ((r * k) % N) / N
            X += (np.cos(ang) + 1j * sign * np.sin(ang)) * Y[r][k % P]
        return X

    def gen_uniform(self, seed: int, N: int, n0: int = 0) -> np.ndarray:
        """The oracle's own SplitMix64 uniform[-1,1) re/im input, elements n0..n0+N-1."""
        out = np.empty(N, dtype=np.complex128)
        self._lib.oracle_gen_uniform(seed & (2**64 - 1), n0, N, self._dp(out))
        return out

    def splitmix64(self, seed: int, i: int) -> int:
        return int(self._lib.oracle_splitmix64(seed & (2**64 - 1), i))

    def dft_bins_uniform(self, seed: int, N: int, ks, sign: int = -1) -> np.ndarray:
        """X[k] for the listed k with x = gen_uniform(seed, N) regenerated on the fly."""
        ks = np.ascontiguousarray(np.asarray(ks, dtype=np.int64))
        X = np.empty(ks.size, dtype=np.complex128)
        rc = self._lib.oracle_dft_bins_uniform(seed & (2**64 - 1), N, sign,
                                               ks.ctypes.data_as(_c_i64p), ks.size, self._dp(X))
        if rc:
            raise ValueError(f"oracle_dft_bins_uniform failed ({rc})")
        return X

    def dft_bins(self, x, ks, sign: int = -1) -> np.ndarray:
        """X[k] for the listed k by the direct sum of Eq. 1 over an explicit x."""
        x = self._c128(x)
        ks = np.ascontiguousarray(np.asarray(ks, dtype=np.int64))
        X = np.empty(ks.size, dtype=np.complex128)
        rc = self._lib.oracle_dft_bins(self._dp(x), x.size, sign, ks.ctypes.data_as(_c_i64p),
                                       ks.size, self._dp(X))
        if rc:
            raise ValueError(f"oracle_dft_bins failed ({rc})")
        return X


    # -- real data (the perm layout of Eq. 3, Sec. 2.1) ----------------------
    @staticmethod
    def pack_perm(X) -> np.ndarray:
        """The perm layout of Eq. 3 for the spectrum X[0..N) of real data:
        {R_0, R_{N/2}, R_1, I_1, ..., R_{N/2-1}, I_{N/2-1}} (N reals);
        X[k] for k > N/2 follows from the symmetry X[N-k] = conj(X[k])."""
        X = np.asarray(X, dtype=np.complex128)
        N = X.size
        out = np.empty(N, dtype=np.float64)
        out[0] = X[0].real
        out[1] = X[N // 2].real
        out[2::2] = X[1:N // 2].real
        out[3::2] = X[1:N // 2].imag
        return out

    @staticmethod
    def unpack_perm(p) -> np.ndarray:
        """Inverse of pack_perm: the full Hermitian spectrum F[0..N) of a
        perm array (F[N-k] = conj(F[k]); F[0], F[N/2] real)."""
        p = np.asarray(p, dtype=np.float64)
        N = p.size
        F = np.empty(N, dtype=np.complex128)
        F[0] = p[0]
        F[N // 2] = p[1]
        F[1:N // 2] = p[2::2] + 1j * p[3::2]
        F[N // 2 + 1:] = np.conj(F[1:N // 2][::-1])
        return F

    def rdft_perm(self, x, sign: int = -1) -> np.ndarray:
        """Eq. 1 for real x (N even >= 2), packed by pack_perm."""
        x = np.asarray(x, dtype=np.float64)
        return self.pack_perm(self.dft(x.astype(np.complex128), sign))

    def irdft_perm(self, p, sign: int = +1) -> np.ndarray:
        """x[n] = sum_k F[k] exp(sign*2*pi*i*n*k/N) over the Hermitian
        spectrum of the perm array p (a real result; unnormalised, so that
        irdft_perm(rdft_perm(x)) = N x)."""
        return self.dft(self.unpack_perm(p), sign).real.copy()


def rel_l2(F, Fe) -> float:
    """Relative L2 error of Eq. 9 (Sec. 5.3), read with complex moduli:
    sqrt(sum |F_k - Fe_k|^2) / sqrt(sum |Fe_k|^2)."""
    F = np.asarray(F, dtype=np.complex128)
    Fe = np.asarray(Fe, dtype=np.complex128)
    # both norms are taken of values divided by max|Fe| (the ratio is
    # unchanged) so that magnitudes near the binary64 limits do not overflow
    s = float(np.max(np.abs(Fe))) if Fe.size else 0.0
    if not np.isfinite(s) or s == 0.0:
        s = 1.0
    num = np.sqrt(np.sum(np.abs((F - Fe) / s) ** 2))
    den = np.sqrt(np.sum(np.abs(Fe / s) ** 2))
    return float(num / den) if den > 0 else float(num)


# the metric as a method as well, so that a test can replace it on one
# Oracle object (a planted mistake) without touching the module function
Oracle.rel_l2 = staticmethod(rel_l2)

_default: Oracle | None = None


def get() -> Oracle:
    """The real oracle (no planted mistake), built on first use."""
    global _default
    if _default is None:
        _default = Oracle(0)
    return _default
