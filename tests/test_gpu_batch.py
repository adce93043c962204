"""Explicit radix schedules, the autotuner and batched transforms of mixed
sizes (one CUDA graph launch) against the CPU oracle.

A batch runs the same kernels with the same schedule as single plans, so
its results must be bit-identical to theirs; the single-plan path is in turn
checked against the oracle here and in test_gpu_parity.py."""
import numpy as np
import pytest

import oracle
from parity_util import TOL, check, host_input, schedule_candidates

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _code(name):
    import paper_1409_5757_gb300 as efft
    return efft.EFFT_C128 if name == "c128" else efft.EFFT_C64


def _np(name):
    return np.complex128 if name == "c128" else np.complex64


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("e", list(range(0, 25)))
def test_every_schedule_matches_oracle(orc, name, e):
    """Every accepted radix schedule, through efft_plan_create_with_radices."""
    import paper_1409_5757_gb300 as efft
    N = 1 << e
    x = host_input(orc, name, N, seed=3000 + e)
    X = orc.dft(x, -1)
    for r in schedule_candidates(e):
        plan = efft.Plan(N, _code(name), -1, 0, radices=r)
        assert plan.radices() == r
        t = torch.from_numpy(x.astype(_np(name))).cuda()
        plan.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
        check(t.cpu().numpy().astype(np.complex128), X, name, N, f"radices {r}")
        plan.destroy()


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("e", [13, 20])
def test_every_schedule_inverse_normalised(orc, name, e):
    import paper_1409_5757_gb300 as efft
    N = 1 << e
    x = host_input(orc, name, N, seed=17)
    X = orc.dft(x, +1) / N
    for r in schedule_candidates(e):
        t = torch.from_numpy(x.astype(_np(name))).cuda()
        efft.Plan(N, _code(name), 1, efft.EFFT_FLAG_NORMALIZE, radices=r).execute(
            t.data_ptr(), torch.cuda.current_stream().cuda_stream)
        check(t.cpu().numpy().astype(np.complex128), X, name, N, f"radices {r}")


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("e", [4, 12, 19, 24])
def test_autotune_scans_every_candidate(orc, name, e):
    import paper_1409_5757_gb300 as efft
    N = 1 << e
    plan = efft.Plan(N, _code(name), -1)
    scratch = torch.empty(N, dtype=torch.complex128 if name == "c128" else torch.complex64, device="cuda")
    res = plan.autotune(scratch.data_ptr(), torch.cuda.current_stream().cuda_stream)
    ns = len(schedule_candidates(e))
    # every accepted schedule first, then the fastest schedule's variants
    assert [r for r, _ in res[:ns]] == schedule_candidates(e)
    best_schedule = min(res[:ns], key=lambda t: t[1])[0]
    assert all(r == best_schedule for r, _ in res[ns:])
    assert all(ms > 0 for _, ms in res)
    best = min(res, key=lambda t: t[1])[0]
    assert plan.radices() == best
    # the tuned plan still computes the DFT
    x = host_input(orc, name, N, seed=55)
    t = torch.from_numpy(x.astype(_np(name))).cuda()
    plan.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    check(t.cpu().numpy().astype(np.complex128), orc.dft(x, -1), name, N, "autotuned")
    # later plans with the flag reuse the cached choice
    assert efft.Plan(N, _code(name), 1, efft.EFFT_FLAG_AUTOTUNE).radices() == best


@pytest.mark.parametrize("name,e", [("c128", 26), ("c64", 26), ("c128", 16), ("c64", 21)])
def test_autotune_scans_variants(orc, name, e):
    """The tuner's second stage: for the fastest schedule each kernel
    variant switched the other way where it changes the launches (the wide
    strided tiles; complex128 from 2^26 also the folded digit swap and the
    persistent passes); the plan ends on the fastest candidate and still
    computes the DFT."""
    import paper_1409_5757_gb300 as efft
    N = 1 << e
    plan = efft.Plan(N, _code(name), -1)
    scratch = torch.empty(N, dtype=torch.complex128 if name == "c128" else torch.complex64, device="cuda")
    res = plan.autotune_candidates(scratch.data_ptr(), torch.cuda.current_stream().cuda_stream)
    ns = len(schedule_candidates(e))
    assert [[int(r).bit_length() - 1 for r in c["radices"]] for c in res[:ns]] == schedule_candidates(e)
    best = min(res, key=lambda c: c["ms"])
    assert plan.radices() == [int(r).bit_length() - 1 for r in best["radices"]]
    assert plan.variant() == {k: best[k] for k in ("wide", "fused_swap", "persistent", "tma")}
    # each variant candidate differs from the others (a knob that changes no
    # launch of the fastest schedule is not measured)
    keys = [(c["wide"], c["fused_swap"], c["persistent"], c["tma"]) for c in res[ns:]]
    assert len(set(keys)) == len(keys) <= 4
    if name == "c128" and e >= 26 and best["radices"][0] in (512, 1024, 2048) and len(best["radices"]) == 3:
        assert any(c["fused_swap"] != res[0]["fused_swap"] for c in res) or len(keys) >= 2
    x = host_input(orc, name, N, seed=56)
    t = torch.from_numpy(x.astype(_np(name))).cuda()
    plan.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    check(t.cpu().numpy().astype(np.complex128), orc.dft(x, -1) if N <= (1 << 22) else orc.fft_radix2(x, -1),
          name, N, "tuned variant")


@pytest.mark.parametrize("name,n", [("c128", 3 << 20), ("c64", 5 << 18), ("c128", 15 << 14)])
def test_autotune_mixed_sizes_scans_outer_radix(orc, name, n):
    """N = M * 2^e: the tuner times every outer radix 2^a of the
    (2^a, M 2^b, 2^a) schedule the kernels accept (and one pass when
    N <= 2048), keeps the fastest, and later plans with EFFT_FLAG_AUTOTUNE
    reuse it."""
    import paper_1409_5757_gb300 as efft
    plan = efft.Plan(n, _code(name), -1)
    scratch = torch.empty(n, dtype=torch.complex128 if name == "c128" else torch.complex64, device="cuda")
    res = plan.autotune_candidates(scratch.data_ptr(), torch.cuda.current_stream().cuda_stream)
    outer = [c["radices"][0] for c in res]
    # the schedule scan (distinct outer radices), then at most one record of
    # the fastest schedule with the first pass's tile width switched
    k = len(set(outer))
    assert k >= 3 and len(outer[:k]) == len(set(outer[:k])) and len(res) <= k + 1
    for c in res:
        A, B = c["radices"][0], c["radices"][1]
        assert c["radices"][2] == A and A * B * A == n and A <= 2048 and B <= 2048
    if len(res) == k + 1:
        first = min(res[:k], key=lambda c: c["ms"])
        assert res[k]["radices"] == first["radices"] and res[k]["wide"] == 1 - first["wide"]
    best = min(res, key=lambda c: c["ms"])
    assert best["ms"] > 0
    # a plan created with the flag reuses the measured choice
    tuned = efft.Plan(n, _code(name), -1, efft.EFFT_FLAG_AUTOTUNE)
    assert tuned.radices() == [int(R & -R).bit_length() - 1 for R in best["radices"]]
    assert tuned.variant()["wide"] == best["wide"]
    x = host_input(orc, name, n, seed=57)
    t = torch.from_numpy(x.astype(_np(name))).cuda()
    tuned.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    check(t.cpu().numpy().astype(np.complex128), orc.dft(x, -1), name, n, "tuned mixed")


@pytest.mark.parametrize("name,n", [("c128", 3 << 24), ("c64", 3 << 26)])
def test_mixed_first_pass_tile_width_knob(orc, name, n):
    """N = M * 2^e with outer radix 2^10: the `wide` knob switches the first
    pass (2^10 rows at the odd stride 3 * 2^(e-10)) between its two tile
    widths; both give the oracle's transform, and the tuner's flip of the
    knob is a candidate of the same schedule."""
    import paper_1409_5757_gb300 as efft
    plan = efft.Plan(n, _code(name), -1)
    assert plan.radices()[0] == 10
    x = host_input(orc, name, n, seed=58)
    ref = orc.dft(x, -1)
    seen = set()
    for w in (1, 0):
        assert plan.set_variant(w, -1, -1)["wide"] == w
        seen.add(plan.variant()["wide"])
        t = torch.from_numpy(x.astype(_np(name))).cuda()
        plan.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        check(t.cpu().numpy().astype(np.complex128), ref, name, n, f"wide={w}")
    assert seen == {0, 1}
    with pytest.raises(efft.EfftError) as ei:
        plan.set_variant(-1, 1, -1)
    assert ei.value.status == 9


@pytest.mark.parametrize("name", ["c128", "c64"])
def test_autotune_flag_at_creation(orc, name):
    import paper_1409_5757_gb300 as efft
    N = 1 << 18
    plan = efft.Plan(N, _code(name), -1, efft.EFFT_FLAG_AUTOTUNE)
    assert plan.radices() in schedule_candidates(18)
    x = host_input(orc, name, N, seed=8)
    t = torch.from_numpy(x.astype(_np(name))).cuda()
    plan.execute(t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    check(t.cpu().numpy().astype(np.complex128), orc.dft(x, -1), name, N, "autotune flag")


def _batch_inputs(orc, name, es, seed):
    xs = [host_input(orc, name, 1 << e, seed + i) for i, e in enumerate(es)]
    ts = [torch.from_numpy(x.astype(_np(name))).cuda() for x in xs]
    return xs, ts


@pytest.mark.parametrize("name", ["c128", "c64"])
@pytest.mark.parametrize("sign,flags", [(-1, 0), (1, 0x2), (-1, 0x1)])
def test_batch_mixed_sizes(orc, name, sign, flags):
    """Sizes 2^0..2^20 with repeats, in shuffled order: each result equals the
    single-plan result bit for bit, and the oracle within tolerance."""
    import paper_1409_5757_gb300 as efft
    rng = np.random.default_rng(21)
    es = list(range(0, 21)) + [12, 12, 3, 16, 16, 16, 20, 7, 0]
    rng.shuffle(es)
    xs, ts = _batch_inputs(orc, name, es, 400)
    refs = [t.clone() for t in ts]
    b = efft.Batch([t.numel() for t in ts], _code(name), sign, flags)
    info = b.info()
    assert info["groups"] == len(set(es))
    assert info["kernels"] > 0
    b.execute([t.data_ptr() for t in ts], torch.cuda.current_stream().cuda_stream)
    for r in refs:
        efft.fft_(r, sign, flags)
    torch.cuda.synchronize()
    for e, x, t, r in zip(es, xs, ts, refs):
        assert torch.equal(t, r), f"batch differs from the single plan at N=2^{e}"
        if not (flags & 0x1):
            want = orc.dft(x, sign) / ((1 << e) if flags & 0x2 else 1)
            check(t.cpu().numpy().astype(np.complex128), want, name, 1 << e, "batch")
    b.destroy()


@pytest.mark.parametrize("name", ["c128", "c64"])
def test_batch_reexecute_new_buffers(orc, name):
    """More executes back to back than the staging ring holds, each on other
    buffers: the device pointer array follows every call."""
    import paper_1409_5757_gb300 as efft
    es = [14, 9, 14, 17, 3, 12]
    b = efft.Batch([1 << e for e in es], _code(name), -1)
    rounds = []
    for k in range(2 * efft.EFFT_BATCH_INFLIGHT + 1):
        xs, ts = _batch_inputs(orc, name, es, 1000 + 10 * k)
        b.execute([t.data_ptr() for t in ts], torch.cuda.current_stream().cuda_stream)
        rounds.append((xs, ts))
    torch.cuda.synchronize()
    for xs, ts in rounds:
        for e, x, t in zip(es, xs, ts):
            check(t.cpu().numpy().astype(np.complex128), orc.dft(x, -1), name, 1 << e, "re-execute")


def test_batch_argument_errors():
    import paper_1409_5757_gb300 as efft
    base = torch.zeros(3 << 12, dtype=torch.complex64, device="cuda")
    b = efft.Batch([1 << 12, 1 << 12], efft.EFFT_C64, -1)
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(ValueError):
        b.execute([base.data_ptr()], s)
    with pytest.raises(efft.EfftError) as ei:  # overlapping buffers
        b.execute([base.data_ptr(), base.data_ptr() + 8 * 100], s)
    assert ei.value.status == 4
    with pytest.raises(efft.EfftError) as ei:  # misaligned
        b.execute([base.data_ptr(), base.data_ptr() + (1 << 15) + 4], s)
    assert ei.value.status == 5
    with pytest.raises(efft.EfftError) as ei:  # host memory
        h = torch.zeros(1 << 12, dtype=torch.complex64)
        b.execute([base.data_ptr(), h.data_ptr()], s)
    assert ei.value.status == 4
    b.execute([base.data_ptr(), base.data_ptr() + (1 << 15)], s)  # adjacent is fine
    torch.cuda.synchronize()
    h = b._h
    b.destroy()
    assert efft._lib().efft_batch_destroy(h) == 10


@pytest.mark.parametrize("name", ["c128", "c64"])
def test_batch_fault_injection(monkeypatch, name):
    import paper_1409_5757_gb300 as efft
    t = torch.zeros(1 << 10, dtype=torch.complex128 if name == "c128" else torch.complex64, device="cuda")
    b = efft.Batch([1 << 10], _code(name), -1)
    monkeypatch.setenv("EFFT_FAULT_INJECT", "launch")
    with pytest.raises(efft.EfftError) as ei:
        b.execute([t.data_ptr()], 0)
    assert ei.value.status == 7
    with pytest.raises(efft.EfftError) as ei:
        efft.Batch([1 << 11, 1 << 10], _code(name), -1)
    assert ei.value.status == 7
    monkeypatch.setenv("EFFT_FAULT_INJECT", "alloc")
    with pytest.raises(efft.EfftError) as ei:
        efft.Batch([1 << 9], _code(name), -1)
    assert ei.value.status == 6
    monkeypatch.delenv("EFFT_FAULT_INJECT")
    b.execute([t.data_ptr()], 0)
    torch.cuda.synchronize()


@pytest.mark.parametrize("name", ["c128", "c64"])
def test_batch_host_stream_chain(orc, name):
    """efft_batch_execute_host_stream: host arrays through a chain of batches,
    chunk by chunk (ten 2^22 transforms make several chunks of one group).
    A one-batch chain equals single plans bit for bit; forward then the
    normalised inverse returns the input; mismatched batches are rejected."""
    import paper_1409_5757_gb300 as efft
    from paper_1409_5757_gb300 import inputs
    es = [22] * 10 + [0, 3, 12, 16, 16, 20, 12]
    sizes = [1 << e for e in es]
    tdt = torch.complex128 if name == "c128" else torch.complex64
    offs = np.concatenate([[0], np.cumsum(sizes)])
    total = int(offs[-1])
    hin = inputs.PinnedHost(total, tdt)
    hout = inputs.PinnedHost(total, tdt)
    for i, n in enumerate(sizes):
        inputs_t = torch.empty(n, dtype=tdt, device="cuda")
        inputs.fill_uniform(inputs_t, 7100 + i)
        hin.tensor[offs[i]:offs[i + 1]].copy_(inputs_t.cpu())
    esz = hin.tensor.element_size()
    dev = torch.empty(total, dtype=tdt, device="cuda")
    hp_in = [hin.ptr + int(o) * esz for o in offs[:-1]]
    hp_out = [hout.ptr + int(o) * esz for o in offs[:-1]]
    dp = [dev.data_ptr() + int(o) * esz for o in offs[:-1]]
    fwd = efft.Batch(sizes, _code(name), -1)
    inv = efft.Batch(sizes, _code(name), +1, efft.EFFT_FLAG_NORMALIZE)
    s = torch.cuda.current_stream().cuda_stream
    efft.batch_execute_host_stream([fwd], hp_in, hp_out, dp, s)
    for i, n in enumerate(sizes):
        ref = hin.tensor[offs[i]:offs[i + 1]].cuda()
        efft.fft_(ref, -1)
        assert torch.equal(hout.tensor[offs[i]:offs[i + 1]], ref.cpu()), f"N=2^{es[i]}"
    efft.batch_execute_host_stream([fwd, inv], hp_in, hp_out, dp, s)
    for i, n in enumerate(sizes):
        got = hout.tensor[offs[i]:offs[i + 1]].numpy().astype(np.complex128)
        x = hin.tensor[offs[i]:offs[i + 1]].numpy().astype(np.complex128)
        assert oracle.rel_l2(got, x) <= 2 * TOL[name] * max(es[i], 1), f"round trip N=2^{es[i]}"
    other = efft.Batch(sizes[:-1] + [1 << 13], _code(name), -1)
    with pytest.raises(efft.EfftError) as ei:
        efft.batch_execute_host_stream([fwd, other], hp_in, hp_out, dp, s)
    assert ei.value.status == 1
    for b in (fwd, inv, other):
        b.destroy()
    hin.free()
    hout.free()


@pytest.mark.parametrize("flags", [0, 0x4], ids=["table", "autotuned"])
def test_batch_of_256_uneven_c64(orc, flags):
    """256 complex64 transforms, N = 2^e with e uniform in {12..24} (seed 5),
    with the table's schedules and with EFFT_FLAG_AUTOTUNE (the benchmark's
    setting): bit-identical to single plans of the same flags for all, the
    oracle for the smallest and largest sampled."""
    import paper_1409_5757_gb300 as efft
    from paper_1409_5757_gb300 import inputs
    es = np.random.default_rng(5).integers(12, 25, 256)
    ts = [torch.empty(1 << int(e), dtype=torch.complex64, device="cuda") for e in es]
    for i, t in enumerate(ts):
        inputs.fill_uniform(t, 5000 + i)
    refs = [t.clone() for t in ts]
    efft.fft_batch_(ts, -1, flags)
    for r in refs:
        efft.fft_(r, -1, flags)
    torch.cuda.synchronize()
    for e, t, r in zip(es, ts, refs):
        assert torch.equal(t, r), f"N=2^{e}"
    for i in (int(np.argmin(es)), int(np.argmax(es))):
        N = 1 << int(es[i])
        x = orc.gen_uniform(5000 + i, N).astype(np.complex64).astype(np.complex128)
        check(ts[i].cpu().numpy().astype(np.complex128), orc.dft(x, -1), "c64", N, "256-batch")


@pytest.mark.parametrize("name", ["c128", "c64"])
def test_batch_grad_matches_closed_form(orc, name):
    """L = sum_t sum_k |w_tk X_tk|^2 over a batch of sizes 2^4..2^14:
    grad x_t = 2 F^H(|w_t|^2 X_t) per transform."""
    from paper_1409_5757_gb300.autograd import dft_batch
    es = [4, 9, 14, 9, 11]
    g = np.random.default_rng(99)
    xs = [host_input(orc, name, 1 << e, 70 + i) for i, e in enumerate(es)]
    ws = [g.uniform(0, 1, 1 << e) for e in es]
    rdt = torch.float64 if name == "c128" else torch.float32
    xt = [torch.from_numpy(x.astype(_np(name))).cuda().requires_grad_(True) for x in xs]
    Xs = dft_batch(xt, -1)
    L = sum(torch.sum(torch.from_numpy(w ** 2).to(rdt).cuda() * (X.real ** 2 + X.imag ** 2)) for w, X in zip(ws, Xs))
    L.backward()
    for e, x, w, t in zip(es, xs, ws, xt):
        ref = 2 * orc.dft(w ** 2 * orc.dft(x, -1), +1)
        assert oracle.rel_l2(t.grad.cpu().numpy().astype(np.complex128), ref) <= TOL[name] * 2 * e


def test_batch_grad_finite_differences(orc):
    from paper_1409_5757_gb300.autograd import dft_batch
    es = [6, 10]
    xs = [orc.gen_uniform(90 + i, 1 << e) for i, e in enumerate(es)]
    w2 = [torch.from_numpy(np.random.default_rng(e).uniform(0, 1, 1 << e) ** 2).cuda() for e in es]

    def loss(ts):
        return sum(torch.sum(w * (X.real ** 2 + X.imag ** 2)) for w, X in zip(w2, dft_batch(ts, 1)))

    xt = [torch.from_numpy(x.copy()).cuda().requires_grad_(True) for x in xs]
    loss(xt).backward()
    h = 1e-3
    for ti, j in ((0, 0), (0, 63), (1, 5), (1, 1023)):
        for unit in (1.0, 1j):
            xp = [torch.from_numpy(x.copy()).cuda() for x in xs]
            xm = [torch.from_numpy(x.copy()).cuda() for x in xs]
            xp[ti][j] += unit * h
            xm[ti][j] -= unit * h
            with torch.no_grad():
                d = (loss(xp) - loss(xm)).item() / (2 * h)
            gj = xt[ti].grad[j].item()
            want = gj.real if unit == 1.0 else gj.imag
            assert abs(d - want) <= 1e-7 * max(1.0, abs(want)), (ti, j, unit, d, want)


def test_batch_grad_256_uneven_c64_at_config_scale(orc):
    """The batched, differentiated configuration at full scale: 256 complex64
    transforms of 2^e points, e uniform in {12..24} (numpy default_rng(5)),
    inputs the seed-5 uniform stream laid end to end, one graph launch
    forward and one backward through autograd.dft_batch; loss
    L = sum_t sum_k w_tk^2 |X_tk|^2 with w uniform[0,1).
    For the smallest and the largest member: the gradient against the closed
    form 2 F^H(|w|^2 X) (F, F^H from the FP64 oracle on the FP32 input
    promoted to FP64), and central finite differences of L evaluated by the
    FP64 oracle (h = 1e-3) at sampled coordinates, real and imaginary."""
    from paper_1409_5757_gb300 import inputs
    from paper_1409_5757_gb300.autograd import dft_batch
    es = [int(e) for e in np.random.default_rng(5).integers(12, 25, 256)]
    offs = np.concatenate([[0], np.cumsum([1 << e for e in es])]).astype(np.int64)
    arena = torch.empty(int(offs[-1]), dtype=torch.complex64, device="cuda")
    inputs.fill_uniform(arena, 5)
    xt = [arena[int(offs[i]):int(offs[i + 1])].clone().requires_grad_(True) for i in range(256)]
    del arena
    g = np.random.default_rng(55)
    ws = [g.uniform(0, 1, 1 << e) for e in es]
    w2t = [torch.from_numpy(w ** 2).float().cuda() for w in ws]
    Xs = dft_batch(xt, -1)
    L = sum(torch.sum(w2.double() * (X.real.double() ** 2 + X.imag.double() ** 2)) for w2, X in zip(w2t, Xs))
    L.backward()
    del Xs, w2t
    for i in (int(np.argmin(es)), int(np.argmax(es))):
        N = 1 << es[i]
        x = orc.gen_uniform(5, N, n0=int(offs[i])).astype(np.complex64).astype(np.complex128)
        assert np.array_equal(x, xt[i].detach().cpu().numpy().astype(np.complex128)), "input stream"
        w2 = ws[i] ** 2
        X = orc.fft_radix2(x, -1)
        ref = 2 * orc.fft_radix2(w2 * X, +1)
        got = xt[i].grad.cpu().numpy().astype(np.complex128)
        assert oracle.rel_l2(got, ref) <= TOL["c64"] * 2 * es[i], (N, oracle.rel_l2(got, ref))
        # central differences of the FP64 loss, coordinate by coordinate
        rms = float(np.sqrt(np.mean(np.abs(ref) ** 2)))
        h = 1e-3
        for j in (0, 1, N // 2 + 1, N - 1):
            for unit in (1.0, 1j):
                xp = x.copy()
                xm = x.copy()
                xp[j] += unit * h
                xm[j] -= unit * h
                lp = float(np.sum(w2 * np.abs(orc.fft_radix2(xp, -1)) ** 2))
                lm = float(np.sum(w2 * np.abs(orc.fft_radix2(xm, -1)) ** 2))
                d = (lp - lm) / (2 * h)
                want = got[j].real if unit == 1.0 else got[j].imag
                assert abs(d - want) <= TOL["c64"] * 2 * es[i] * 10 * rms, (N, j, unit, d, want, rms)
