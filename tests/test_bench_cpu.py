"""Host-side logic of bench.py (no GPU): the double-float operation count of
the ALU roofline, the traffic table lookup, and workload scaling."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _walk_pass_ops(log2r: int, kind: str) -> float:
    """FP32 operations per element of one double-float pass, counted by
    walking the radix-16 (then radix 2^(log2r mod 4)) decimation-in-frequency
    butterflies level by level as the pass kernels run them: every pair
    (a, b) costs an add and a subtract, its second output a multiply by
    exp(-2*pi*i*e/16) (e = j*8/half: 0 and 4 free, 2 and 6 the
    exp(-2*pi*i/8) product, odd e a general constant product); every stage
    but the last multiplies 15 of each 16 values by an internal twiddle;
    strided passes apply the pass twiddle as two products and renormalise."""
    add, mul, w8, norm = 16, 32, 24, 6
    stages = [4] * (log2r // 4) + ([log2r % 4] if log2r % 4 else [])
    total = 0.0
    for st, lg in enumerate(stages):
        n = 1 << lg
        ops = 0.0
        half = n // 2
        while half >= 1:
            for blk in range(0, n, 2 * half):
                for j in range(half):
                    ops += 2 * add  # a + b, a - b
                    e = j * (8 // half)
                    if e in (2, 6):
                        ops += w8
                    elif e % 2 == 1:
                        ops += mul
            half //= 2
        total += ops / n  # per element
        if st < len(stages) - 1:
            total += 15.0 / 16.0 * mul
    if kind in ("FIRST", "MID"):
        total += 2 * mul + norm
    return total


@pytest.mark.parametrize("log2r", [8, 9, 10, 11])
@pytest.mark.parametrize("kind", ["FIRST", "MID", "LAST"])
def test_df_ops_per_element_matches_butterfly_walk(log2r, kind):
    assert bench.df_ops_per_element(log2r, kind) == pytest.approx(_walk_pass_ops(log2r, kind))


def test_df_ops_known_values():
    # the figures quoted for the complex128 passes
    assert bench.df_ops_per_element(10, "FIRST") == 324
    assert bench.df_ops_per_element(10, "LAST") == 254
    assert bench.df_ops_per_element(11, "FIRST") == 346
    assert bench.FP32_PEAK_OPS == pytest.approx(152 * 128 * 2.07e9)


def test_traffic_lookup_by_kernel_family(tmp_path, monkeypatch):
    fp = {f: bench.kernel_fingerprint(f) for f in ("c128", "c64", "mixed")}
    assert len(set(fp.values())) == 3
    table = tmp_path / "profiles"
    table.mkdir()
    (table / "dram_traffic.txt").write_text(
        "# header\n"
        f"c2 30 pass0 1.0e9 60.0 40.0 {fp['c128']} src a\n"
        f"c4 31 pass1 2.0e9 - - {fp['c64']} src b\n"
        f"m1 30 pass1 3.0e9 - - {fp['mixed']} src c\n"
        f"c4 31 pass0 4.0e9 1 2 {fp['c128']} wrong family\n")
    # the table under a temporary root; the fingerprints stay those of the sources
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_fingerprint", lambda family: fp[family])
    t = bench.measured_traffic("c2", 30, "pass0")
    assert t["bytes"] == 1.0e9 and t["fma_pipe_pct"] == 60.0 and t["source"] == "src a"
    t = bench.measured_traffic("c4", 31, "pass1")
    assert t["bytes"] == 2.0e9 and t["fma_pipe_pct"] is None and t["issue_pct"] is None
    assert bench.measured_traffic("m1", 30, "pass1")["bytes"] == 3.0e9
    assert bench.measured_traffic("c4", 31, "pass0") is None  # fingerprint of another family
    assert bench.measured_traffic("c3", 33, "pass0") is None  # no entry


def test_scale_workload():
    m1 = bench.WORKLOADS["m1"]
    s = bench.scale_workload(m1, 28)
    assert s["n"] == 3 << 26 and s["log2n"] == 28
    assert "3*2^26" in s["desc"] and "3 GiB" in s["desc"]
    assert m1["n"] == 3 << 28  # the table itself is untouched
    c4 = bench.scale_workload(bench.WORKLOADS["c4"], 28)
    assert c4["log2n"] == 28 and "n" not in c4 and "2^28" in c4["desc"]
