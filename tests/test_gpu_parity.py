"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (relative L2 error of Eq. 9, Sec. 5.3, with complex moduli):
  complex128 (double-float butterflies): 1e-14 * log2 N
  complex64  (FP32 butterflies)        : 2e-6  * log2 N, against the FP64
             oracle applied to the FP32-rounded input promoted to FP64.
Inputs are the seeded uniform[-1,1) re/im stream regenerated by the oracle's
own SplitMix64 (bit-identical to the device generator, checked below).
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-14, "c64": 2e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _tdtype(name):
    return torch.complex128 if name == "c128" else torch.complex64


def gpu_fft(x_host, name, sign=-1, flags=0):
    import paper_1409_5757_gb300 as efft
    t = torch.from_numpy(np.ascontiguousarray(x_host.astype(np.complex128 if name == "c128" else np.complex64)))
    t = t.cuda()
    efft.fft_(t, sign=sign, flags=flags)
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def host_input(o, name, N, seed):
    x = o.gen_uniform(seed, N)
    if name == "c64":
        x = x.astype(np.complex64).astype(np.complex128)  # the values the GPU sees
    return x


def check(got, ref, name, N, what=""):
    err = oracle.rel_l2(got, ref)
    lim = TOL[name] * max(np.log2(N), 1)
    assert err <= lim, f"{what} {name} N={N}: rel-L2 {err:.3e} > {lim:.3e}"
    # element-wise: no single output far off (relative to the RMS output)
    s = float(np.max(np.abs(ref))) if ref.size else 0.0  # scale first: magnitudes up to 1e300
    if s > 0 and np.isfinite(s):
        rms = np.sqrt(np.mean(np.abs(ref / s) ** 2))
        assert np.max(np.abs((got - ref) / s)) <= 50 * lim * rms, f"{what} {name} N={N}: outlier"
    return err


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("sign", [-1, 1])
@pytest.mark.parametrize("e", list(range(0, 23)))
def test_parity_every_size(orc, name, sign, e):
    N = 1 << e
    x = host_input(orc, name, N, seed=1000 + e)
    got = gpu_fft(x, name, sign)
    check(got, orc.dft(x, sign), name, N)


def test_device_generator_matches_oracle_generator(orc):
    from paper_1409_5757_gb300 import inputs
    for N, seed, n0 in ((1, 3, 0), (1000, 1, 0), (4096, 77, 123456789)):
        t = torch.empty(N, dtype=torch.complex128, device="cuda")
        inputs.fill_uniform(t, seed, n0)
        assert np.array_equal(t.cpu().numpy(), orc.gen_uniform(seed, N, n0=n0))
        t = torch.empty(N, dtype=torch.complex64, device="cuda")
        inputs.fill_uniform(t, seed, n0)
        assert np.array_equal(t.cpu().numpy(), orc.gen_uniform(seed, N, n0=n0).astype(np.complex64))


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("e", [12, 13, 16, 19, 20, 21, 22, 23])
def test_digit_reversed_output(orc, name, e):
    import paper_1409_5757_gb300 as efft
    N = 1 << e
    radices = efft.Plan(N, efft.EFFT_C128 if name == "c128" else efft.EFFT_C64, -1,
                        efft.EFFT_FLAG_DIGIT_REVERSED_OUT).radices()
    x = host_input(orc, name, N, seed=7)
    got = gpu_fft(x, name, -1, efft.EFFT_FLAG_DIGIT_REVERSED_OUT)
    X = orc.dft(x, -1)
    # position P = sum_j q_j s_j holds X[q_0 + R_0 q_1 + R_0 R_1 q_2 + ...]
    R = [1 << r for r in radices]
    P = np.arange(N)
    k = np.zeros(N, np.int64)
    s = N
    mult = 1
    for j, Rj in enumerate(R):
        s //= Rj
        q = (P // s) % Rj
        k += q * mult
        mult *= Rj
    check(got, X[k], name, N, "digit-reversed")


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("e", [5, 11, 16, 21])
def test_round_trip(orc, name, e):
    import paper_1409_5757_gb300 as efft
    N = 1 << e
    x = host_input(orc, name, N, seed=9)
    t = torch.from_numpy(x.astype(np.complex128 if name == "c128" else np.complex64)).cuda()
    efft.fft_(t, -1)
    efft.fft_(t, 1)
    got = t.cpu().numpy().astype(np.complex128) / N
    err = oracle.rel_l2(got, x)
    assert err <= 2 * TOL[name] * e


@pytest.mark.parametrize("name", ["c128", "c64"])
def test_special_inputs(orc, name):
    N = 1 << 14
    k = np.arange(N)
    cases = {
        "zeros": np.zeros(N, np.complex128),
        "impulse0": (k == 0).astype(np.complex128),
        "impulse_m": (k == 1234).astype(np.complex128),
        "constant": np.full(N, 0.375 - 0.625j),
        "tone": np.exp(2j * np.pi * ((777 * k) % N) / N),
    }
    for label, x in cases.items():
        if name == "c64":
            x = x.astype(np.complex64).astype(np.complex128)
        got = gpu_fft(x, name, -1)
        ref = orc.fft_radix2(x, -1)
        if label == "zeros":
            assert np.all(got == 0)
        else:
            check(got, ref, name, N, label)


@pytest.mark.parametrize("scale", [1e300, 1e-300, 2.0 ** -1000, 1e150])
def test_c128_extreme_magnitudes(orc, scale):
    """The double-float path carries a power-of-two scale: magnitudes far
    outside the binary32 range keep full accuracy."""
    N = 1 << 16
    x = orc.gen_uniform(21, N) * scale
    got = gpu_fft(x, "c128", -1)
    check(got, orc.fft_radix2(x, -1), "c128", N, f"scale {scale}")


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("e", [3, 10, 16, 21])
def test_nan_input_gives_nan(orc, name, e):
    N = 1 << e
    x = orc.gen_uniform(5, N)
    x[N // 3] = complex(np.nan, 0.0)
    got = gpu_fft(x, name, -1)
    assert np.all(np.isnan(got.real) | np.isnan(got.imag))


def test_c128_inf_input_gives_nan(orc):
    N = 1 << 16
    x = orc.gen_uniform(5, N)
    x[17] = complex(np.inf, 1.0)
    got = gpu_fft(x, "c128", -1)
    assert np.all(np.isnan(got.real))


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("e", [24, 26])
def test_parity_large_full_oracle(orc, name, e):
    N = 1 << e
    x = host_input(orc, name, N, seed=2000 + e)
    got = gpu_fft(x, name, -1)
    check(got, orc.fft_radix2(x, -1), name, N)


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("sign", [-1, 1])
def test_parity_2p28_wide_first_pass(orc, name, sign):
    """2^28 = 2^10 * 2^8 * 2^10: from 2^28 on the first pass runs on wide
    tiles (complex128: 8192 elements; complex64: the radix-32 kernel on
    16384 elements, 16 columns); against the full oracle."""
    import paper_1409_5757_gb300 as efft
    N = 1 << 28
    code = efft.EFFT_C128 if name == "c128" else efft.EFFT_C64
    assert efft.Plan(N, code, sign).radices() == [10, 8, 10]
    x = host_input(orc, name, N, seed=2828)
    got = gpu_fft(x, name, sign)
    check(got, orc.fft_radix2(x, sign), name, N)


@pytest.mark.parametrize("sign", [-1, 1])
def test_parity_2p28_wide_first_pass_2p11_c128(orc, sign):
    """complex128 2^28 with the schedule 2^11 * 2^6 * 2^11: the first pass is
    the wide 2^11-row kernel (8192-element tiles, 4 columns, one 512-thread
    CTA per SM) at a power-of-two stride, the kernel variant that the 2^33
    schedule 2^11 * 2^11 * 2^11 runs; element by element against the full
    oracle."""
    import paper_1409_5757_gb300 as efft
    N = 1 << 28
    x = host_input(orc, "c128", N, seed=2811)
    t = torch.from_numpy(x).cuda()
    p = efft.Plan(N, efft.EFFT_C128, sign, radices=[11, 6, 11])
    assert p.radices() == [11, 6, 11]
    p.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = t.cpu().numpy()
    del t
    p.destroy()
    check(got, orc.fft_radix2(x, sign), "c128", N)


def test_parity_c64_2p29_middle_pass_2p11(orc):
    """complex64 2^29 with the schedule 2^9 * 2^11 * 2^9: from 2^28 on the
    2^11-row middle pass runs on 8-column tiles (16384 elements, one
    1024-thread CTA per SM); against the full oracle."""
    import paper_1409_5757_gb300 as efft
    N = 1 << 29
    x = host_input(orc, "c64", N, seed=2929)
    t = torch.from_numpy(x.astype(np.complex64)).cuda()
    p = efft.Plan(N, efft.EFFT_C64, -1, radices=[9, 11, 9])
    assert p.radices() == [9, 11, 9]
    p.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = t.cpu().numpy().astype(np.complex128)
    del t
    check(got, orc.fft_radix2(x, -1), "c64", N)


def test_execute_host_entry_point(orc):
    import paper_1409_5757_gb300 as efft
    N = 1 << 18
    x = orc.gen_uniform(4, N)
    host = torch.from_numpy(x.copy()).pin_memory()
    dev = torch.empty(N, dtype=torch.complex128, device="cuda")
    p = efft.Plan(N, efft.EFFT_C128, -1)
    p.execute_host(host.data_ptr(), dev.data_ptr(), torch.cuda.current_stream().cuda_stream)
    check(host.numpy(), orc.fft_radix2(x, -1), "c128", N, "execute_host")


def test_execute_rejects_bad_buffers():
    import paper_1409_5757_gb300 as efft
    p = efft.Plan(1 << 10, efft.EFFT_C128, -1)
    with pytest.raises(efft.EfftError) as ei:
        p.execute(0)
    assert ei.value.status == 4
    t = torch.zeros(2048 + 1, dtype=torch.complex64, device="cuda")
    with pytest.raises(efft.EfftError) as ei:
        p.execute(t.data_ptr() + 8)  # 8-byte aligned only, complex128 needs 16
    assert ei.value.status == 5
    h = torch.zeros(1024, dtype=torch.complex128)
    with pytest.raises(efft.EfftError) as ei:
        p.execute(h.data_ptr())  # host memory
    assert ei.value.status == 4
    p.destroy()
    with pytest.raises(efft.EfftError) as ei:
        efft._check(efft._lib().efft_execute(p.handle, None, None), "x")


def test_fault_injection_is_host_side(monkeypatch):
    import paper_1409_5757_gb300 as efft
    monkeypatch.setenv("EFFT_FAULT_INJECT", "alloc")
    with pytest.raises(efft.EfftError) as ei:
        efft.Plan(1 << 12)
    assert ei.value.status == 6
    monkeypatch.setenv("EFFT_FAULT_INJECT", "launch")
    p = efft.Plan(1 << 12)
    t = torch.zeros(1 << 12, dtype=torch.complex128, device="cuda")
    with pytest.raises(efft.EfftError) as ei:
        p.execute(t.data_ptr())
    assert ei.value.status == 7
    monkeypatch.delenv("EFFT_FAULT_INJECT")
    p.execute(t.data_ptr())
    torch.cuda.synchronize()


@pytest.mark.parametrize("e", [10, 20])
def test_c128_output_just_below_a_power_of_two(e):
    """x = v * delta_0 gives X[k] = v for every k.  With v = +-(2^k - 2^(k-30))
    the double-float value is (2^k, -2^(k-30)): a power-of-two high part
    with an opposite-sign low part, whose sum lies in the binade below --
    the binary64 conversion must still return v exactly."""
    N = 1 << e
    for k in (0, 9, 40, -20):
        for sgn in (1.0, -1.0):
            v = sgn * (2.0 ** k - 2.0 ** (k - 30))
            x = np.zeros(N, np.complex128)
            x[0] = v + 1j * v
            got = gpu_fft(x, "c128", -1)
            assert np.max(np.abs(got - (v + 1j * v))) <= 1e-15 * abs(v), (k, sgn)


@pytest.mark.parametrize("e", [11, 16, 20, 24])
@pytest.mark.parametrize("pattern", ["element", "column"])
def test_c128_tiles_of_different_scales(orc, e, pattern):
    """The complex128 scale is found per first-pass tile and reconciled in
    the second pass: inputs whose binary exponents vary by up to 2^+-48
    between elements, or between column groups (so that whole tiles differ),
    still match the oracle."""
    N = 1 << e
    n = np.arange(N)
    shift = ((n * 7919) % 97) - 48 if pattern == "element" else ((n % 4096) >> 6) % 97 - 48
    x = orc.gen_uniform(60 + e, N) * np.ldexp(1.0, shift)
    got = gpu_fft(x, "c128", -1)
    check(got, orc.dft(x, -1), "c128", N, pattern)


@pytest.mark.parametrize("radices,sign,flags", [
    ([9, 8, 9], -1, 0), ([9, 8, 9], 1, 2), ([9, 10, 9], -1, 0), ([10, 8, 10], 1, 0), ([9, 8, 9], -1, 1)],
    ids=["9-8-9", "9-8-9-inv-norm", "9-10-9", "10-8-10-inv", "9-8-9-digit-reversed"])
def test_parity_fused_digit_swap(orc, radices, sign, flags):
    """complex128 three-pass schedules (a, b, a) with a in 9..11 and b in
    {8, 10, 11} from 2^26 on: the middle pass swaps the outer digits itself
    (pairs of column tiles on the two CTAs of a cluster) and the last pass is
    strided, so no digit-swap sweep runs (efft_plan_info counts 3.5 sweeps).
    Element by element against the full oracle; with
    EFFT_FLAG_DIGIT_REVERSED_OUT the unfused passes run and the output is the
    digit-reversed order of the oracle's."""
    import paper_1409_5757_gb300 as efft
    e = sum(radices)
    N = 1 << e
    x = host_input(orc, "c128", N, seed=4000 + e + radices[0])
    t = torch.from_numpy(x).cuda()
    p = efft.Plan(N, efft.EFFT_C128, sign, flags, radices=radices)
    fused = not (flags & efft.EFFT_FLAG_DIGIT_REVERSED_OUT)
    # 3 passes + the half sweep of the range scan (an unfused natural-order
    # plan would add the swap sweep: 4.5)
    assert p.info()["hbm_passes"] == 3.5
    p.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = t.cpu().numpy()
    del t
    p.destroy()
    ref = orc.fft_radix2(x, sign)
    if flags & efft.EFFT_FLAG_NORMALIZE:
        ref = ref / N
    if not fused:
        a, b = radices[0], radices[1]
        P = np.arange(N, dtype=np.int64)
        q0, q1, q2 = P >> (a + b), (P >> a) & ((1 << b) - 1), P & ((1 << a) - 1)
        ref = ref[q0 + (q1 << a) + (q2 << (a + b))]
    check(got, ref, "c128", N)


def test_fused_digit_swap_in_a_batch_is_bit_identical():
    """Two 2^28 transforms (default schedule 10 * 8 * 10, fused swap) in one
    batch launch (grid.y selects the transform, clusters along x) equal
    single-plan executes bit for bit."""
    import paper_1409_5757_gb300 as efft
    from paper_1409_5757_gb300 import inputs
    N = 1 << 28
    p = efft.Plan(N, efft.EFFT_C128, -1)
    assert p.radices() == [10, 8, 10] and p.info()["hbm_passes"] == 3.5
    xs = [torch.empty(N, dtype=torch.complex128, device="cuda") for _ in range(2)]
    for i, x in enumerate(xs):
        inputs.fill_uniform(x, seed=60 + i)
    want = []
    for x in xs:
        y = x.clone()
        p.execute(y.data_ptr(), torch.cuda.current_stream().cuda_stream)
        want.append(y)
    b = efft.Batch([N, N], efft.EFFT_C128, -1)
    b.execute([x.data_ptr() for x in xs], torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for x, w in zip(xs, want):
        assert torch.equal(x, w)
    b.destroy()
    p.destroy()
    del want, xs


@pytest.mark.parametrize("radices,flags,variant", [
    ([8, 11, 8], 0, (-1, -1, 1)), ([9, 9, 9], 0, (-1, -1, 1)), ([8, 10, 8], 0, (-1, -1, 1)),
    ([10, 8, 10], 1, (1, -1, 1)), ([9, 11, 9], 0, (-1, 1, 1)), ([10, 8, 10], 0, (1, 1, 1)),
    ([10, 8, 10], 0, (0, 0, 0)), ([9, 8, 9], 0, (1, 1, 0))],
    ids=["8-11-8-pf", "9-9-9-pf", "8-10-8-pf", "10-8-10-wide-pf-digit-reversed", "9-11-9-fused-pf",
         "10-8-10-all", "10-8-10-none", "9-8-9-wide-fused"])
def test_parity_persistent_passes(orc, radices, flags, variant):
    """complex128 from 2^26 on, every kernel variant set through
    efft_plan_set_variant: the persistent strided passes that copy the next
    tile's inputs into shared memory while the current tile finishes (every
    middle-pass radix 2^8..2^11 on 4096-element tiles, the wide first pass,
    the swapping and the strided last passes), the folded digit swap and the
    wide first-pass tiles, on and off; against the full oracle, in natural or
    digit-reversed order."""
    import paper_1409_5757_gb300 as efft
    e = sum(radices)
    N = 1 << e
    x = host_input(orc, "c128", N, seed=4100 + e + radices[1])
    t = torch.from_numpy(x).cuda()
    p = efft.Plan(N, efft.EFFT_C128, -1, flags, radices=radices)
    got_v = p.set_variant(*variant)
    for k, want in zip(("wide", "fused_swap", "persistent"), variant):
        if want == 0:
            assert got_v[k] == 0, (k, got_v)
    if variant[2] == 1:
        assert got_v["persistent"] == 1
    p.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = t.cpu().numpy()
    del t
    p.destroy()
    ref = orc.fft_radix2(x, -1)
    if flags & efft.EFFT_FLAG_DIGIT_REVERSED_OUT:
        a, b = radices[0], radices[1]
        P = np.arange(N, dtype=np.int64)
        q0, q1, q2 = P >> (a + b), (P >> a) & ((1 << b) - 1), P & ((1 << a) - 1)
        ref = ref[q0 + (q1 << a) + (q2 << (a + b))]
    check(got, ref, "c128", N)


@pytest.mark.parametrize("e,sign", [(28, -1), (28, 1), (20, -1), (24, 1)])
def test_parity_c64_tma_first_pass(orc, e, sign):
    """complex64: the wide first pass of 2^10 rows (16 columns) as the
    persistent kernel fed by TMA copies (efft_plan_set_variant, tma = 1; at
    2^20 and 2^24 with the wide tiles forced, fewer tiles than SMs at 2^20):
    against the full oracle, bit for bit against the kernel that loads its
    own tiles (the same arithmetic), and no expired device wait."""
    import paper_1409_5757_gb300 as efft
    N = 1 << e
    x = host_input(orc, "c64", N, seed=5100 + e)
    runs = {}
    for tma in (0, 1):
        # a first pass of 2^10 rows: the table's schedule at 2^20 and 2^28,
        # 2^10 * 2^4 * 2^10 at 2^24
        p = efft.Plan(N, efft.EFFT_C64, sign, radices=[10, 4, 10] if e == 24 else None)
        v = p.set_variant(1, -1, -1, tma)
        assert v["tma"] == tma and v["wide"] == 1
        t = torch.from_numpy(x.astype(np.complex64)).cuda()
        p.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert p.check(torch.cuda.current_stream().cuda_stream) == 0
        runs[tma] = t
        p.destroy()
    assert torch.equal(runs[0], runs[1])
    got = runs[1].cpu().numpy().astype(np.complex128)
    del runs
    check(got, orc.fft_radix2(x, sign), "c64", N)


def test_tma_wait_expiry_is_reported(orc, monkeypatch):
    """The bounded device wait of the TMA-fed first pass, made to run out on
    purpose: with EFFT_FAULT_INJECT=tma_wait the kernel arms its barrier
    without issuing copies, gives up after 1024 polls, records the timeout
    and returns; efft_execute_check reports EFFT_ERR_TIMEOUT once, and the
    context stays usable (the next execute is correct)."""
    import paper_1409_5757_gb300 as efft
    N = 1 << 20  # schedule 2^10 * 2^10: a first pass of 2^10 rows
    x = host_input(orc, "c64", N, seed=52)
    p = efft.Plan(N, efft.EFFT_C64, -1)
    assert p.set_variant(1, -1, -1, 1)["tma"] == 1
    sp = torch.cuda.current_stream().cuda_stream
    t = torch.from_numpy(x.astype(np.complex64)).cuda()
    monkeypatch.setenv("EFFT_FAULT_INJECT", "tma_wait")
    p.execute(t.data_ptr(), sp)
    monkeypatch.delenv("EFFT_FAULT_INJECT")
    assert p.check(sp) == 8  # EFFT_ERR_TIMEOUT
    assert p.check(sp) == 0  # the record was cleared
    t = torch.from_numpy(x.astype(np.complex64)).cuda()
    p.execute(t.data_ptr(), sp)
    assert p.check(sp) == 0
    check(t.cpu().numpy().astype(np.complex128), orc.fft_radix2(x, -1), "c64", N)
    p.destroy()


@pytest.mark.parametrize("radices,sign", [([9, 11, 9], -1), ([4, 11, 4], 1), ([6, 11, 6], -1)])
def test_parity_c64_tma_middle_pass(orc, radices, sign):
    """complex64: the wide middle pass of 2^11 rows (8 columns, 1024 threads)
    as the persistent kernel fed by TMA copies (3-D boxes: column, row,
    block), at the 2^29 default schedule and with the wide tiles forced at
    2^19 and 2^23 (16 and 64 columns per block): against the full oracle,
    bit for bit against the middle pass that loads its own tiles, and no
    expired device wait."""
    import paper_1409_5757_gb300 as efft
    e = sum(radices)
    N = 1 << e
    x = host_input(orc, "c64", N, seed=5300 + e)
    runs = {}
    for tma in (0, 1):
        p = efft.Plan(N, efft.EFFT_C64, sign, radices=radices)
        v = p.set_variant(1, -1, -1, tma)
        assert v["tma"] == tma and v["wide"] == 1, v
        t = torch.from_numpy(x.astype(np.complex64)).cuda()
        p.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert p.check(torch.cuda.current_stream().cuda_stream) == 0
        runs[tma] = t
        p.destroy()
    assert torch.equal(runs[0], runs[1])
    got = runs[1].cpu().numpy().astype(np.complex128)
    del runs
    check(got, orc.fft_radix2(x, sign), "c64", N)


def test_tma_wait_expiry_is_reported_middle_pass(orc, monkeypatch):
    """The TMA-fed complex64 middle pass with its wait made to run out
    (EFFT_FAULT_INJECT=tma_wait): EFFT_ERR_TIMEOUT, then a correct execute."""
    import paper_1409_5757_gb300 as efft
    N = 1 << 19
    x = host_input(orc, "c64", N, seed=54)
    p = efft.Plan(N, efft.EFFT_C64, -1, radices=[4, 11, 4])
    assert p.set_variant(1, -1, -1, 1)["tma"] == 1
    sp = torch.cuda.current_stream().cuda_stream
    t = torch.from_numpy(x.astype(np.complex64)).cuda()
    monkeypatch.setenv("EFFT_FAULT_INJECT", "tma_wait")
    p.execute(t.data_ptr(), sp)
    monkeypatch.delenv("EFFT_FAULT_INJECT")
    assert p.check(sp) == 8
    assert p.check(sp) == 0
    t = torch.from_numpy(x.astype(np.complex64)).cuda()
    p.execute(t.data_ptr(), sp)
    assert p.check(sp) == 0
    check(t.cpu().numpy().astype(np.complex128), orc.fft_radix2(x, -1), "c64", N)
    p.destroy()
