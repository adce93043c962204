"""Helpers shared by the GPU parity tests: tolerances, seeded inputs, the
element-wise check and the list of radix schedules the planner accepts."""
import numpy as np

import oracle

# relative L2 error (Eq. 9, Sec. 5.3) per log2 N
TOL = {"c128": 1e-14, "c64": 2e-6}


def host_input(o, name, N, seed):
    """The seeded uniform[-1,1) input; for c64 the FP32-rounded values (what
    the GPU sees), promoted back to FP64 for the oracle."""
    x = o.gen_uniform(seed, N)
    if name == "c64":
        x = x.astype(np.complex64).astype(np.complex128)
    return x


def check(got, ref, name, N, what=""):
    err = oracle.rel_l2(got, ref)
    lim = TOL[name] * max(np.log2(N), 1)
    assert err <= lim, f"{what} {name} N={N}: rel-L2 {err:.3e} > {lim:.3e}"
    s = float(np.max(np.abs(ref))) if ref.size else 0.0  # scale first: magnitudes up to 1e300
    if s > 0 and np.isfinite(s):
        rms = np.sqrt(np.mean(np.abs(ref / s) ** 2))
        assert np.max(np.abs((got - ref) / s)) <= 50 * lim * rms, f"{what} {name} N={N}: outlier"
    return err


def schedule_candidates(e):
    """Every radix schedule (log2 R_j) the planner accepts for N = 2^e: none
    for N <= 8; one pass of 2^4..2^11; two or three passes of 2^4..2^11,
    symmetric."""
    if e <= 3:
        return [[]]
    c = []
    if e <= 11:
        c.append([e])
    if e % 2 == 0 and 4 <= e // 2 <= 11:
        c.append([e // 2, e // 2])
    for a in range(4, 12):
        b = e - 2 * a
        if 4 <= b <= 11:
            c.append([a, b, a])
    return c
