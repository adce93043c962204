"""The boundary's concurrency rules (include/efft.h): executes of one plan on
different buffers may run concurrently on unordered streams, and an execute
captured into a CUDA graph may be replayed while eager executes of the same
plan run.  Every execute has a state word of its own (the largest binary64
exponent of its complex128 input); a shared word would give a buffer the
scale of another one, and with inputs 10^400 apart in magnitude that would
flush the smaller buffer's values to zero.  Results are compared bit for bit
with the same executes run one after the other (the kernels are
deterministic)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _inputs(N):
    from paper_1409_5757_gb300 import inputs
    a = torch.empty(N, dtype=torch.complex128, device="cuda")
    b = torch.empty(N, dtype=torch.complex128, device="cuda")
    inputs.fill_uniform(a, seed=41)
    inputs.fill_uniform(b, seed=42)
    a.mul_(1e200)
    b.mul_(1e-200)
    return a, b


def _sequential(plan, x):
    y = x.clone()
    plan.execute(y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return y


@pytest.mark.parametrize("e", [12, 20, 24])
def test_one_plan_two_streams_two_buffers(e):
    import paper_1409_5757_gb300 as efft
    N = 1 << e
    plan = efft.Plan(N, efft.EFFT_C128, -1)
    a0, b0 = _inputs(N)
    want_a, want_b = _sequential(plan, a0), _sequential(plan, b0)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    # 40 rounds: more executes than the plan's ring of state words holds
    for _ in range(20):
        a, b = a0.clone(), b0.clone()
        torch.cuda.synchronize()
        for _ in range(2):  # forward twice on each buffer, the streams unordered
            plan.execute(a.data_ptr(), s1.cuda_stream)
            plan.execute(b.data_ptr(), s2.cuda_stream)
        torch.cuda.synchronize()
        wa, wb = _sequential(plan, want_a), _sequential(plan, want_b)
        assert torch.equal(a, wa)
        assert torch.equal(b, wb)
    assert float(torch.abs(want_b).max()) > 0
    plan.destroy()


def test_captured_execute_replays_beside_eager_executes():
    import paper_1409_5757_gb300 as efft
    N = 1 << 18
    plan = efft.Plan(N, efft.EFFT_C128, -1)
    a0, b0 = _inputs(N)
    want_a, want_b = _sequential(plan, a0), _sequential(plan, b0)
    xa = a0.clone()
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap):
        with torch.cuda.graph(g, stream=cap, capture_error_mode="relaxed"):
            plan.execute(xa.data_ptr(), cap.cuda_stream)
    other = torch.cuda.Stream()
    for _ in range(3):
        xa.copy_(a0)
        xb = b0.clone()
        torch.cuda.synchronize()
        g.replay()  # on the current stream
        plan.execute(xb.data_ptr(), other.cuda_stream)
        torch.cuda.synchronize()
        assert torch.equal(xa, want_a)
        assert torch.equal(xb, want_b)
    del g
    plan.destroy()


def test_destroy_waits_for_executes_in_flight():
    import paper_1409_5757_gb300 as efft
    N = 1 << 22
    a0, _ = _inputs(N)
    plan = efft.Plan(N, efft.EFFT_C128, -1)
    want = _sequential(plan, a0)
    plan2 = efft.Plan(N, efft.EFFT_C128, -1)
    x = a0.clone()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    plan2.execute(x.data_ptr(), s.cuda_stream)
    plan2.destroy()  # returns after the execute's launches finished with its state
    torch.cuda.synchronize()
    assert torch.equal(x, want)
    plan.destroy()
    assert np.isfinite(float(torch.abs(x).max()))
