"""Host models of the index decompositions the kernels use, checked against
the oracle on the CPU (no GPU, no library call).  They restate the mapping
in numpy so that a change to the kernels' index arithmetic has a reference
that runs without a device; the GPU parity tests check the kernels
themselves.

- The two-stage column DFT of the mixed-radix middle pass for R = P1 * 16,
  P1 = 3 * 2^c (Sec. 2.1's N = M * 2^s with M = 3): n = n2 + 16 n1,
  k = k1 + P1 k2; stage A the P1-point DFT over n1 (a radix-3 butterfly over
  n1 = j, j + Q, j + 2Q with Q = P1 / 3, the twiddle exp(-2 pi i j q / P1),
  a radix-Q decimation in frequency) times exp(-2 pi i n2 k1 / R); stage B
  the 16-point DFT over n2.
- The digit reversal of a three-pass (A, B, A) schedule and its in-place
  tile-pair swap (Sec. 3.2's scatter): position q0 B A + q1 A + q2 holds
  X[q0 + A q1 + A B q2], and swapping the outer digits restores natural
  order.
"""
import numpy as np
import pytest

import oracle


def _bitrev(v, bits):
    r = 0
    for b in range(bits):
        r |= ((v >> b) & 1) << (bits - 1 - b)
    return r


def _dif(v, log2n):
    """In-place radix-2 decimation in frequency of a list of 2^log2n values;
    entry u ends up holding output bitrev(u)."""
    half = (1 << log2n) // 2
    while half >= 1:
        for blk in range(0, 1 << log2n, 2 * half):
            for j in range(half):
                a, b = v[blk + j], v[blk + j + half]
                v[blk + j] = a + b
                v[blk + j + half] = (a - b) * np.exp(-2j * np.pi * j / (2 * half))
        half //= 2


def _two_stage_column(x, p1):
    q = p1 // 3
    c = q.bit_length() - 1
    r = p1 * 16
    tile = np.zeros((p1, 16), dtype=complex)  # [k1][n2], the exchange buffer
    for n2 in range(16):
        v = [x[n2 + 16 * n1] for n1 in range(p1)]
        y = [[0j] * q for _ in range(3)]
        for j in range(q):
            a, b, d = v[j], v[j + q], v[j + 2 * q]
            t1 = b + d
            t2 = a - 0.5 * t1
            t3 = -1j * (np.sqrt(3.0) / 2.0) * (b - d)
            y[0][j] = a + t1
            y[1][j] = (t2 + t3) * np.exp(-2j * np.pi * j / p1)
            y[2][j] = (t2 - t3) * np.exp(-2j * np.pi * 2 * j / p1)
        for qq in range(3):
            w = list(y[qq])
            if c:
                _dif(w, c)
            for u in range(q):
                k1 = qq + 3 * (_bitrev(u, c) if c else 0)
                tile[k1][n2] = w[u] * np.exp(-2j * np.pi * n2 * k1 / r)
    out = np.zeros(r, dtype=complex)
    for k1 in range(p1):
        v = list(tile[k1])
        _dif(v, 4)
        for u in range(16):
            out[k1 + p1 * _bitrev(u, 4)] = v[u]
    return out


@pytest.mark.parametrize("p1", [3, 6, 12])
def test_two_stage_column_dft_matches_oracle(orc, p1):
    r = p1 * 16
    x = orc.gen_uniform(300 + p1, r)
    got = _two_stage_column(x, p1)
    want = orc.dft(x, -1)
    assert oracle.rel_l2(got, want) <= 1e-15 * np.log2(r) * 4


def test_two_stage_column_index_map_is_a_bijection():
    for p1 in (3, 6, 12):
        seen = set()
        for k1 in range(p1):
            for u in range(16):
                seen.add(k1 + p1 * _bitrev(u, 4))
        assert seen == set(range(16 * p1))


@pytest.mark.parametrize("a,b", [(3, 2), (4, 5), (5, 3)])
def test_digit_reversal_and_tile_swap_model(orc, a, b):
    A, B = 1 << a, 3 << b
    n = A * B * A
    x = orc.gen_uniform(400 + a, n)
    X = orc.dft(x, -1)
    # the three-pass output before the swap: position q0 B A + q1 A + q2
    # holds X[q0 + A q1 + A B q2]
    p = np.arange(n)
    q0, q1, q2 = p // (B * A), (p // A) % B, p % A
    dr = X[q0 + A * q1 + A * B * q2]
    # in-place swap of (q0, q1, q2) with (q2, q1, q0), tile pair by tile pair
    # (T x T tiles, I <= J), as the swap kernel does
    y = dr.copy()
    T = min(32, A)
    nt = A // T
    for i1 in range(B):
        for J in range(nt):
            for I in range(J + 1):
                r = np.arange(T)
                rows0 = (I * T + r)[:, None] * (B * A) + i1 * A + (J * T + r)[None, :]
                rows1 = (J * T + r)[:, None] * (B * A) + i1 * A + (I * T + r)[None, :]
                t0, t1 = y[rows0].copy(), y[rows1].copy()
                y[rows1] = t0.T
                if I != J:
                    y[rows0] = t1.T
    assert np.array_equal(y, X)
