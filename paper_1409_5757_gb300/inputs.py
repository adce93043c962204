"""Seeded synthetic inputs for tests and the benchmark (libefft_inputs.so).

Holds none of the transform's arithmetic.  Device generators write straight
into HBM (inputs of 2^30..2^33 elements never cross PCIe/C2C); the tone
parameters are drawn here on the host so that both the device generator and
the CPU oracle receive the same numbers as inputs.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_vp = ctypes.c_void_p

GOLDEN = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


def lib_path() -> str:
    return os.path.join(PKG, "libefft_inputs.so")


def _lib():
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run paper_1409_5757_gb300.build.build()")
        lib = ctypes.CDLL(path)
        lib.efft_gen_uniform.argtypes = [_vp, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _vp]
        lib.efft_gen_gaussian.argtypes = [_vp, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _vp]
        lib.efft_add_tones.argtypes = [_vp, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_int, _vp]
        lib.efft_diff_norms.argtypes = [_vp, _vp, ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_double), _vp]
        lib.efft_host_alloc.argtypes = [ctypes.POINTER(_vp), ctypes.c_uint64]
        lib.efft_host_free.argtypes = [_vp]
        for f in (lib.efft_gen_uniform, lib.efft_gen_gaussian, lib.efft_add_tones, lib.efft_diff_norms,
                  lib.efft_host_alloc, lib.efft_host_free):
            f.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _code(t) -> int:
    import torch
    if t.dtype == torch.complex128:
        return 1
    if t.dtype == torch.complex64:
        return 0
    raise TypeError(t.dtype)


def _stream(t):
    import torch
    return _vp(torch.cuda.current_stream(t.device).cuda_stream)


def _ok(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with CUDA error {rc}")


def fill_uniform(t, seed: int, n0: int = 0):
    """t[n] = uniform[-1,1) re/im from SplitMix64 element n0 + n."""
    _ok(_lib().efft_gen_uniform(_vp(t.data_ptr()), t.numel(), _code(t), seed & MASK64, n0, _stream(t)),
        "efft_gen_uniform")
    return t


def fill_gaussian(t, seed: int, n0: int = 0):
    _ok(_lib().efft_gen_gaussian(_vp(t.data_ptr()), t.numel(), _code(t), seed & MASK64, n0, _stream(t)),
        "efft_gen_gaussian")
    return t


def splitmix64(seed: int, i: int) -> int:
    z = (seed + (i + 1) * GOLDEN) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def tone_params(seed: int, N: int, ntones: int = 64):
    """Distinct integer frequencies f_j in [0, N) and amplitudes a_j whose real
    and imaginary parts are uniform[-1,1) dyadic rationals (exact in binary64,
    so N*a_j is exact), from a SplitMix64 stream with its own seed."""
    s = (seed * 0x100000001B3 + 0x7F4A7C15) & MASK64
    freqs, amps, seen, i = [], [], set(), 0
    while len(freqs) < ntones:
        f = splitmix64(s, i) & (N - 1)
        i += 1
        if f in seen:
            continue
        seen.add(f)
        re = 2.0 * ((splitmix64(s, i) >> 11) * 2.0 ** -53) - 1.0
        im = 2.0 * ((splitmix64(s, i + 1) >> 11) * 2.0 ** -53) - 1.0
        i += 2
        freqs.append(f)
        amps.append(complex(re, im))
    return np.array(freqs, np.int64), np.array(amps, np.complex128)


def add_tones(t, freqs, amps):
    """t[n] += sum_j a_j exp(+2*pi*i*f_j*n/N) over the whole array (synchronous)."""
    f = np.ascontiguousarray(freqs, np.int64)
    a = np.ascontiguousarray(np.asarray(amps, np.complex128).view(np.float64))
    _ok(_lib().efft_add_tones(_vp(t.data_ptr()), t.numel(), _code(t), f.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                              a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(f), _stream(t)),
        "efft_add_tones")
    return t


def diff_norms(a, b=None, scale: float = 1.0):
    """(sum |scale*a - b|^2, sum |b|^2) in FP64 on the device (synchronous)."""
    out = (ctypes.c_double * 2)()
    _ok(_lib().efft_diff_norms(_vp(a.data_ptr()), _vp(b.data_ptr() if b is not None else 0), a.numel(), _code(a),
                               float(scale), out, _stream(a)), "efft_diff_norms")
    return out[0], out[1]


class PinnedHost:
    """Page-locked host buffer from cudaHostAlloc, viewable as a CPU tensor."""

    def __init__(self, numel: int, dtype):
        import torch
        self.dtype = dtype
        self.numel = numel
        itemsize = torch.empty(0, dtype=dtype).element_size()
        self.nbytes = numel * itemsize
        p = _vp()
        _ok(_lib().efft_host_alloc(ctypes.byref(p), self.nbytes), "efft_host_alloc")
        self.ptr = p.value
        buf = (ctypes.c_uint8 * self.nbytes).from_address(self.ptr)
        self.tensor = torch.frombuffer(buf, dtype=torch.uint8).view(dtype)

    def free(self):
        if self.ptr:
            self.tensor = None
            _lib().efft_host_free(_vp(self.ptr))
            self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
