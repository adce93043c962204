"""Python binding of libefft.so: the in-place 1-D complex DFT on one GB300.

Argument marshalling only: every step of the transform runs in the CUDA
kernels of ``csrc/``.  PyTorch supplies device memory and streams.  There is
no CPU fallback: if the compiled library is missing, importing the binding's
functions raises.

    import torch, paper_1409_5757_gb300 as efft
    x = torch.randn(1 << 20, dtype=torch.complex128, device="cuda")
    efft.fft_(x)            # X[k] = sum_n x[n] exp(-2*pi*i*n*k/N), in place
    efft.fft_(x, sign=+1)   # conjugate-sign transform (x * N after both)

The C ABI is documented in include/efft.h.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))

EFFT_C64 = 0
EFFT_C128 = 1
EFFT_FLAG_DIGIT_REVERSED_OUT = 0x1
EFFT_FLAG_NORMALIZE = 0x2
EFFT_FLAG_AUTOTUNE = 0x4
EFFT_BATCH_INFLIGHT = 4
EFFT_REAL_FORWARD = -1
EFFT_REAL_INVERSE = +1
PROFILE_SLOTS = ("range_scan", "pass0", "pass1", "pass2", "pass3", "digit_swap", "direct_small", "real_pair")
EFFT_MAX_LOG2N = 33

STATUS = {
    0: "EFFT_OK", 1: "EFFT_ERR_INVALID_SIZE", 2: "EFFT_ERR_INVALID_DTYPE", 3: "EFFT_ERR_INVALID_SIGN",
    4: "EFFT_ERR_INVALID_PTR", 5: "EFFT_ERR_MISALIGNED", 6: "EFFT_ERR_ALLOC", 7: "EFFT_ERR_LAUNCH",
    8: "EFFT_ERR_TIMEOUT", 9: "EFFT_ERR_UNSUPPORTED", 10: "EFFT_ERR_INVALID_PLAN", 11: "EFFT_ERR_CUDA",
    12: "EFFT_ERR_INVALID_FLAGS",
}

# every entry point declared in include/efft.h: name -> (restype, argtypes)
_vp = ctypes.c_void_p


class EfftCandidate(ctypes.Structure):
    """efft_candidate of include/efft.h."""
    _fields_ = [("npasses", ctypes.c_int), ("radices", ctypes.c_uint64 * 4), ("wide", ctypes.c_int),
                ("fused_swap", ctypes.c_int), ("persistent", ctypes.c_int), ("tma", ctypes.c_int),
                ("ms", ctypes.c_double)]



_SIGNATURES = {
    "efft_plan_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_uint32]),
    "efft_execute": (ctypes.c_int, [_vp, _vp, _vp]),
    "efft_execute_host": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "efft_plan_destroy": (ctypes.c_int, [_vp]),
    "efft_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "efft_version": (ctypes.c_int, []),
    "efft_plan_radices": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]),
    "efft_plan_info": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)]),
    "efft_plan_profile": (ctypes.c_int, [_vp, ctypes.c_int]),
    "efft_plan_profile_read": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                              ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "efft_execute_noalloc": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, _vp]),
    "efft_execute_host_stream": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp),
                                                ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp), ctypes.c_int,
                                                _vp]),
    "efft_plan_create_with_radices": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                                     ctypes.c_uint32, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "efft_plan_autotune": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "efft_plan_autotune_candidates": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(EfftCandidate), ctypes.c_int,
                                                     ctypes.POINTER(ctypes.c_int)]),
    "efft_plan_variant": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "efft_plan_set_variant": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "efft_execute_check": (ctypes.c_int, [_vp, _vp]),
    "efft_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_uint64), ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_uint32]),
    "efft_batch_execute": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), _vp]),
    "efft_plan_schedule": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
                                          ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "efft_batch_execute_host_stream": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp),
                                                      ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp]),
    "efft_batch_info": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "efft_batch_destroy": (ctypes.c_int, [_vp]),
    "efft_plan_create_real": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_uint32]),
}


class EfftError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        name = STATUS.get(status, str(status))
        msg = _lib().efft_strerror(status).decode() if _LIB is not None else name
        super().__init__(f"{what}: {name} ({msg})" if what else f"{name} ({msg})")


_LIB = None
_LIB_LOCK = threading.Lock()


def lib_path() -> str:
    return os.path.join(PKG, "libefft.so")


def _lib():
    """Load libefft.so (built by build.py / __graft_entry__.build()); raise if absent."""
    global _LIB
    if _LIB is None:
        with _LIB_LOCK:
            if _LIB is None:
                path = lib_path()
                if not os.path.exists(path):
                    raise RuntimeError(f"{path} is missing: run paper_1409_5757_gb300.build.build() "
                                       "(there is no CPU fallback)")
                lib = ctypes.CDLL(path)
                for name, (res, args) in _SIGNATURES.items():
                    f = getattr(lib, name)
                    f.restype = res
                    f.argtypes = args
                _LIB = lib
    return _LIB


def _check(status: int, what: str):
    if status != 0:
        raise EfftError(status, what)


class Plan:
    """Owning wrapper of an efft_plan_t (efft_plan_create / efft_plan_destroy)."""

    def __init__(self, n: int, dtype: int = EFFT_C128, sign: int = -1, flags: int = 0, radices=None):
        """radices: optional explicit schedule, log2 R_0..R_{p-1}
        (efft_plan_create_with_radices); None = the built-in table, or the
        measured choice with EFFT_FLAG_AUTOTUNE."""
        self._h = _vp()
        if radices is None:
            _check(_lib().efft_plan_create(ctypes.byref(self._h), int(n), int(dtype), int(sign), int(flags)),
                   "efft_plan_create")
        else:
            r = (ctypes.c_int * max(len(radices), 1))(*[int(v) for v in radices])
            _check(_lib().efft_plan_create_with_radices(ctypes.byref(self._h), int(n), int(dtype), int(sign),
                                                        int(flags), r, len(radices)),
                   "efft_plan_create_with_radices")
        self.n, self.dtype, self.sign, self.flags = int(n), int(dtype), int(sign), int(flags)

    @classmethod
    def real(cls, n: int, precision: int = EFFT_C128, direction: int = EFFT_REAL_FORWARD, flags: int = 0):
        """Real-data plan (efft_plan_create_real): n reals <-> the perm layout
        {R_0, R_{N/2}, R_1, I_1, ...}; precision EFFT_C64 (float32 data) or
        EFFT_C128 (float64)."""
        self = cls.__new__(cls)
        self._h = _vp()
        _check(_lib().efft_plan_create_real(ctypes.byref(self._h), int(n), int(precision), int(direction),
                                            int(flags)), "efft_plan_create_real")
        self.n, self.dtype, self.sign, self.flags = int(n), int(precision), int(direction), int(flags)
        return self

    @property
    def handle(self):
        return self._h

    def execute(self, data_ptr: int, stream: int = 0) -> None:
        _check(_lib().efft_execute(self._h, _vp(data_ptr), _vp(stream)), "efft_execute")

    def execute_host(self, host_ptr: int, dev_ptr: int, stream: int = 0) -> None:
        _check(_lib().efft_execute_host(self._h, _vp(host_ptr), _vp(dev_ptr), _vp(stream)), "efft_execute_host")

    def radices(self) -> list[int]:
        arr = (ctypes.c_int * 8)()
        p = ctypes.c_int()
        _check(_lib().efft_plan_radices(self._h, arr, 8, ctypes.byref(p)), "efft_plan_radices")
        return [arr[i] for i in range(p.value)]

    def info(self) -> dict:
        hp = ctypes.c_double()
        tb = ctypes.c_uint64()
        _check(_lib().efft_plan_info(self._h, ctypes.byref(hp), ctypes.byref(tb)), "efft_plan_info")
        return {"hbm_passes": hp.value, "table_bytes": tb.value}

    def autotune(self, scratch_ptr: int, stream: int = 0) -> list[tuple[list[int], float]]:
        """efft_plan_autotune on a caller buffer of n elements (overwritten):
        [(log2 radices, median ms)] per candidate; the plan keeps the fastest."""
        cap = 16
        r = (ctypes.c_int * (4 * cap))()
        ms = (ctypes.c_double * cap)()
        nc = ctypes.c_int()
        _check(_lib().efft_plan_autotune(self._h, _vp(scratch_ptr), _vp(stream), r, ms, cap, ctypes.byref(nc)),
               "efft_plan_autotune")
        return [([v for v in r[4 * c:4 * c + 4] if v], ms[c]) for c in range(min(nc.value, cap))]

    def autotune_candidates(self, scratch_ptr: int, stream: int = 0) -> list[dict]:
        """efft_plan_autotune_candidates: every measured candidate as
        {"radices": [R_j], "wide", "fused_swap", "persistent", "ms"}, in
        measuring order; the plan keeps the fastest."""
        cap = 64
        arr = (EfftCandidate * cap)()
        nc = ctypes.c_int()
        _check(_lib().efft_plan_autotune_candidates(self._h, _vp(scratch_ptr), _vp(stream), arr, cap,
                                                    ctypes.byref(nc)), "efft_plan_autotune_candidates")
        return [{"radices": [int(arr[c].radices[j]) for j in range(arr[c].npasses)], "wide": arr[c].wide,
                 "fused_swap": arr[c].fused_swap, "persistent": arr[c].persistent, "tma": arr[c].tma,
                 "ms": arr[c].ms}
                for c in range(min(nc.value, cap))]

    def variant(self) -> dict:
        """efft_plan_variant: the kernel variant the plan runs."""
        w, f, pp, tm = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib().efft_plan_variant(self._h, ctypes.byref(w), ctypes.byref(f), ctypes.byref(pp),
                                        ctypes.byref(tm)), "efft_plan_variant")
        return {"wide": w.value, "fused_swap": f.value, "persistent": pp.value, "tma": tm.value}

    def set_variant(self, wide: int = -1, fused_swap: int = -1, persistent: int = -1, tma: int = -1) -> dict:
        """efft_plan_set_variant (-1 rule, 0 off, 1 on); returns variant()."""
        _check(_lib().efft_plan_set_variant(self._h, int(wide), int(fused_swap), int(persistent), int(tma)),
               "efft_plan_set_variant")
        return self.variant()

    def check(self, stream: int = 0) -> int:
        """efft_execute_check: synchronise `stream` and return the status of
        the plan's earlier executes' device waits (0 or EFFT_ERR_TIMEOUT)."""
        return _lib().efft_execute_check(self._h, _vp(stream))

    def profile(self, enable: bool = True) -> None:
        """Start (clearing old records) or stop per-launch CUDA-event timing."""
        _check(_lib().efft_plan_profile(self._h, 1 if enable else 0), "efft_plan_profile")

    def profile_read(self) -> dict:
        """{slot name: (total ms, launches)} for the executes since profile(True)."""
        ms = (ctypes.c_double * 8)()
        cnt = (ctypes.c_int * 8)()
        ns = ctypes.c_int()
        _check(_lib().efft_plan_profile_read(self._h, ms, cnt, 8, ctypes.byref(ns)), "efft_plan_profile_read")
        return {PROFILE_SLOTS[i]: (ms[i], cnt[i]) for i in range(min(ns.value, len(PROFILE_SLOTS))) if cnt[i]}

    def destroy(self) -> None:
        if self._h:
            _check(_lib().efft_plan_destroy(self._h), "efft_plan_destroy")
            self._h = _vp()

    def __del__(self):
        try:
            if self._h and _LIB is not None:
                _LIB.efft_plan_destroy(self._h)
        except Exception:
            pass


class Batch:
    """Owning wrapper of an efft_batch_t: `len(sizes)` in-place transforms of
    mixed sizes (N = M * 2^e), one CUDA graph launch per execute."""

    def __init__(self, sizes, dtype: int = EFFT_C64, sign: int = -1, flags: int = 0):
        self.sizes = [int(v) for v in sizes]
        self.dtype, self.sign, self.flags = int(dtype), int(sign), int(flags)
        arr = (ctypes.c_uint64 * max(len(self.sizes), 1))(*self.sizes)
        self._h = _vp()
        _check(_lib().efft_batch_create(ctypes.byref(self._h), arr, len(self.sizes), self.dtype, self.sign,
                                        self.flags), "efft_batch_create")

    def execute(self, data_ptrs, stream: int = 0) -> None:
        if len(data_ptrs) != len(self.sizes):
            raise ValueError(f"efft batch of {len(self.sizes)} transforms got {len(data_ptrs)} buffers")
        arr = (_vp * len(data_ptrs))(*[_vp(int(v)) for v in data_ptrs])
        _check(_lib().efft_batch_execute(self._h, arr, _vp(stream)), "efft_batch_execute")

    def info(self) -> dict:
        g, k = ctypes.c_int(), ctypes.c_int()
        _check(_lib().efft_batch_info(self._h, ctypes.byref(g), ctypes.byref(k)), "efft_batch_info")
        return {"groups": g.value, "kernels": k.value}

    def destroy(self) -> None:
        if self._h:
            _check(_lib().efft_batch_destroy(self._h), "efft_batch_destroy")
            self._h = _vp()

    def __del__(self):
        try:
            if self._h and _LIB is not None:
                _LIB.efft_batch_destroy(self._h)
        except Exception:
            pass


def plan_schedule(n: int, dtype: int = EFFT_C128) -> list:
    """The radices efft_plan_create chooses for (n, dtype) without the
    autotuner (whole integers; computed on the host, no device needed)."""
    arr = (ctypes.c_uint64 * 8)()
    np_ = ctypes.c_int()
    _check(_lib().efft_plan_schedule(int(n), int(dtype), arr, 8, ctypes.byref(np_)), "efft_plan_schedule")
    return [int(arr[j]) for j in range(np_.value)]


def batch_execute_host_stream(batches, host_in, host_out, dev_ptrs, stream: int = 0) -> None:
    """efft_batch_execute_host_stream: transform i copied from host_in[i] to
    dev_ptrs[i], transformed by every batch in order, copied to host_out[i];
    copies overlapped with the transforms chunk by chunk; synchronous."""
    n = len(batches[0].sizes) if batches else 0
    if not batches or any(len(b.sizes) != n for b in batches):
        raise ValueError("efft: batches of one size list expected")
    if len(host_in) != n or len(host_out) != n or len(dev_ptrs) != n:
        raise ValueError(f"efft: {n} transforms need {n} host inputs, outputs and device buffers")
    B = (_vp * len(batches))(*[b._h for b in batches])
    HI = (_vp * n)(*[_vp(int(x)) for x in host_in])
    HO = (_vp * n)(*[_vp(int(x)) for x in host_out])
    DP = (_vp * n)(*[_vp(int(x)) for x in dev_ptrs])
    _check(_lib().efft_batch_execute_host_stream(B, len(batches), HI, HO, DP, _vp(stream)),
           "efft_batch_execute_host_stream")


def execute_host_stream(plans, host_in, host_out, dev_bufs, stream: int = 0) -> None:
    """efft_execute_host_stream: host arrays (data pointers) through the plans
    in order, copies overlapped with the transforms; synchronous."""
    n = len(host_in)
    if len(host_out) != n:
        raise ValueError("host_in and host_out differ in length")
    P = (_vp * len(plans))(*[p.handle for p in plans])
    HI = (_vp * max(n, 1))(*[_vp(x) for x in host_in])
    HO = (_vp * max(n, 1))(*[_vp(x) for x in host_out])
    DB = (_vp * len(dev_bufs))(*[_vp(x) for x in dev_bufs])
    _check(_lib().efft_execute_host_stream(P, len(plans), HI, HO, n, DB, len(dev_bufs), _vp(stream)),
           "efft_execute_host_stream")


_PLANS: dict = {}
_PLANS_LOCK = threading.Lock()


def get_plan(n: int, dtype: int, sign: int = -1, flags: int = 0) -> Plan:
    """Cached plan for (device, N, dtype, sign, flags)."""
    import torch
    key = (torch.cuda.current_device(), int(n), int(dtype), int(sign), int(flags))
    with _PLANS_LOCK:
        p = _PLANS.get(key)
        if p is None:
            p = Plan(n, dtype, sign, flags)
            _PLANS[key] = p
    return p


_BATCHES: dict = {}


def get_batch(sizes, dtype: int, sign: int = -1, flags: int = 0) -> Batch:
    """Cached batch for (device, sizes, dtype, sign, flags)."""
    import torch
    key = (torch.cuda.current_device(), tuple(int(v) for v in sizes), int(dtype), int(sign), int(flags))
    with _PLANS_LOCK:
        b = _BATCHES.get(key)
        if b is None:
            b = Batch(sizes, dtype, sign, flags)
            _BATCHES[key] = b
    return b


def clear_plans() -> None:
    with _PLANS_LOCK:
        for p in _PLANS.values():
            p.destroy()
        _PLANS.clear()
        for b in _BATCHES.values():
            b.destroy()
        _BATCHES.clear()
        for p in _RPLANS.values():
            p.destroy()
        _RPLANS.clear()


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.complex128:
        return EFFT_C128
    if t.dtype == torch.complex64:
        return EFFT_C64
    raise TypeError(f"efft: unsupported dtype {t.dtype} (complex64 or complex128)")


def fft_(t, sign: int = -1, flags: int = 0, stream=None):
    """In-place DFT of a contiguous 1-D CUDA complex tensor; returns t."""
    import torch
    if not t.is_cuda:
        raise ValueError("efft.fft_: tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("efft.fft_: tensor must be contiguous")
    code = _dtype_code(t)
    with torch.cuda.device(t.device):
        plan = get_plan(t.numel(), code, sign, flags)
        s = stream if stream is not None else torch.cuda.current_stream(t.device)
        plan.execute(t.data_ptr(), s.cuda_stream)
    return t


def fft_batch_(tensors, sign: int = -1, flags: int = 0, stream=None):
    """In-place DFTs of a list of contiguous 1-D CUDA complex tensors of one
    dtype and device (supported lengths, not overlapping) by one batch
    execute; returns the list."""
    import torch
    if not tensors:
        return tensors
    code = _dtype_code(tensors[0])
    dev = tensors[0].device
    for t in tensors:
        if not t.is_cuda or t.device != dev:
            raise ValueError("efft.fft_batch_: tensors must be on one CUDA device")
        if not t.is_contiguous():
            raise ValueError("efft.fft_batch_: tensors must be contiguous")
        if _dtype_code(t) != code:
            raise ValueError("efft.fft_batch_: tensors must share one dtype")
    with torch.cuda.device(dev):
        b = get_batch([t.numel() for t in tensors], code, sign, flags)
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        b.execute([t.data_ptr() for t in tensors], s.cuda_stream)
    return tensors


_RPLANS: dict = {}


def _real_code(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return EFFT_C128
    if t.dtype == torch.float32:
        return EFFT_C64
    raise TypeError(f"efft: unsupported real dtype {t.dtype} (float32 or float64)")


def _real_execute(t, direction: int, flags: int, stream):
    import torch
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("efft: real transforms take a contiguous CUDA tensor")
    code = _real_code(t)
    with torch.cuda.device(t.device):
        key = (torch.cuda.current_device(), t.numel(), code, direction, int(flags))
        with _PLANS_LOCK:
            p = _RPLANS.get(key)
            if p is None:
                p = Plan.real(t.numel(), code, direction, flags)
                _RPLANS[key] = p
        s = stream if stream is not None else torch.cuda.current_stream(t.device)
        p.execute(t.data_ptr(), s.cuda_stream)
    return t


def rfft_(t, flags: int = 0, stream=None):
    """In-place real-data DFT of a contiguous 1-D CUDA float32/float64 tensor
    of N = M * 2^e reals (e >= 1, M odd <= 15): afterwards t holds the perm layout
    {R_0, R_{N/2}, R_1, I_1, ..., R_{N/2-1}, I_{N/2-1}} (Eq. 3)."""
    return _real_execute(t, EFFT_REAL_FORWARD, flags, stream)


def irfft_(t, normalize: bool = True, stream=None):
    """In place, the inverse of rfft_: a perm array back to N reals
    (divided by N when normalize, else N times the original data)."""
    return _real_execute(t, EFFT_REAL_INVERSE, EFFT_FLAG_NORMALIZE if normalize else 0, stream)


def fft(t, sign: int = -1):
    """Out-of-place convenience: clone then fft_."""
    return fft_(t.clone(), sign)


def version() -> int:
    return _lib().efft_version()


__all__ = ["Plan", "Batch", "EfftError", "fft_", "fft", "fft_batch_", "rfft_", "irfft_", "get_plan", "get_batch",
           "clear_plans", "version", "EFFT_REAL_FORWARD", "EFFT_REAL_INVERSE",
           "lib_path", "execute_host_stream", "batch_execute_host_stream", "plan_schedule", "EFFT_C64", "EFFT_C128", "EFFT_FLAG_DIGIT_REVERSED_OUT",
           "EFFT_FLAG_NORMALIZE", "EFFT_FLAG_AUTOTUNE"]
