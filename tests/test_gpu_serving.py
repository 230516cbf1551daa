"""Serving (continuous batching under a memory budget): every request's result is the same
alone and in a mix of concurrent requests, equals a direct gdsw_solve, and admission never
exceeds the memory budget."""
import numpy as np
import pytest

from paper_2606_01433_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_01433_gb300 import gdsw
    gdsw.load()
    return gdsw


def _mix():
    return [I.carreau_cube(8, 0.5, 1e-3, seed=11), I.carreau_cube(12, 0.7, 1e-2, seed=12),
            I.carreau_cube(16, 0.3, 1e-4, seed=13), I.carreau_cube(20, 0.9, 3e-3, seed=14),
            I.carreau_cube(8, 0.4, 2e-2, seed=15)]


def test_alone_equals_mix_and_direct(lib):
    probs = _mix()
    srv = lib.Server(max_slots=4, mem_budget_bytes=32 << 30)
    t = srv.gdsw_server_submit(probs[0])
    st, x_alone = srv.gdsw_server_wait(t)
    assert st.state == lib.REQ_DONE and st.status == 0 and st.relres <= 1e-8
    tickets = [srv.gdsw_server_submit(p) for p in probs[1:3]]
    t0 = srv.gdsw_server_submit(probs[0])
    tickets += [srv.gdsw_server_submit(p) for p in probs[3:]]
    st0, x_mix = srv.gdsw_server_wait(t0)
    others = [srv.gdsw_server_wait(t) for t in tickets]
    assert st0.state == lib.REQ_DONE and all(s.state == lib.REQ_DONE and s.relres <= 1e-8 for s, _ in others)
    assert np.array_equal(x_alone, x_mix)
    stats = srv.gdsw_server_stats_read()
    assert stats.completed == 6 and stats.peak_running >= 2
    srv.close()
    ctx = lib.Context(probs[0], precision=("fp32",) * 3, phi_precision="fp32", tol=1e-8)
    b = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    ctx.gdsw_rhs_lift(b)
    x = torch.zeros_like(b)
    ctx.gdsw_solve(b, x)
    torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), x_alone)
    ctx.close()


def test_memory_admission(lib):
    probs = _mix()
    ana = lib.Context(probs[3], analyze_only=True, precision=("fp32",) * 3, phi_precision="fp32")
    one = ana.sizes.device_bytes + 16 * ana.n + (64 << 20)   # the server's admission estimate
    budget = int(one * 1.5)                 # room for one of these requests, not for two
    srv = lib.Server(max_slots=4, mem_budget_bytes=budget)
    ts = [srv.gdsw_server_submit(probs[3]) for _ in range(3)]
    res = [srv.gdsw_server_wait(t) for t in ts]
    stats = srv.gdsw_server_stats_read()
    assert all(s.state == lib.REQ_DONE for s, _ in res)
    assert stats.peak_used_bytes <= budget
    assert stats.peak_running == 1
    assert all(np.array_equal(res[0][1], x) for _, x in res[1:])
    srv.close()


def test_request_too_large_fails(lib):
    srv = lib.Server(max_slots=2, mem_budget_bytes=1 << 20)
    t = srv.gdsw_server_submit(I.carreau_cube(8, 0.5, 1e-3, seed=1))
    st, _ = srv.gdsw_server_wait(t)
    assert st.state == lib.REQ_FAILED and st.status == lib.GDSW_ERR_OOM
    srv.close()
