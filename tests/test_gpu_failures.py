"""Failure detection, injected on the host (no GPU fault, trap or hang): a non-finite
right-hand side, an iteration cap, a problem whose coarse operator is singular (pure Neumann
data: translations and the pressure constant are in the kernel), and a device wait that can
never be met (the persistent sweep's bounded wait).  Each returns its status code and leaves
the context usable."""
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


def test_nan_rhs_and_iteration_cap(lib):
    p = I.box_problem(4, 4, 4, (2, 2, 2), levels=2, form="symmetric", uk_seed=3, lam=1.0, n=0.5, nu_inf=1e-3)
    ctx = lib.Context(p, tol=1e-10, max_it=3)
    b = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    ctx.gdsw_rhs_lift(b)
    x = torch.zeros_like(b)
    info = ctx.gdsw_solve(b, x)                       # capped: not converged, best x returned
    assert info.status == lib.GDSW_ERR_NOT_CONVERGED and info.iterations == 3
    assert np.isfinite(x.cpu().numpy()).all() and 0 < info.relres < 1
    bn = b.clone()
    bn[7] = float("nan")
    with pytest.raises(lib.GdswError) as e:
        ctx.gdsw_solve(bn, torch.zeros_like(b))
    assert e.value.code == lib.GDSW_ERR_NAN
    ctx2 = lib.Context(p, tol=1e-10)                  # the library is still healthy
    x2 = torch.zeros_like(b)
    assert ctx2.gdsw_solve(b, x2).status == 0
    ctx.close()
    ctx2.close()


def test_singular_coarse_operator(lib):
    p = I.box_problem(4, 4, 4, (2, 2, 2), levels=2, bc="neumann")
    with pytest.raises(lib.GdswError) as e:
        lib.Context(p)
    assert e.value.code == lib.GDSW_ERR_SINGULAR


def test_persistent_sweep_wait_limit(lib):
    """A dependency of the persistent level sweep that its producers never signal: the wait ends
    after its 1 s limit, every CTA returns, the call reports GDSW_ERR_TIMEOUT, and the same
    context then solves normally."""
    import time
    p = I.box_problem(4, 4, 4, (2, 2, 2), levels=2, form="symmetric", uk_seed=3, lam=1.0, n=0.5, nu_inf=1e-3)
    ctx = lib.Context(p, tol=1e-10, precision=("fp32",) * 3, phi_precision="fp32")
    t0 = time.perf_counter()
    with pytest.raises(lib.GdswError) as e:
        ctx.gdsw_sweep_wait_selftest()
    elapsed = time.perf_counter() - t0
    assert e.value.code == lib.GDSW_ERR_TIMEOUT
    assert 0.9 <= elapsed < 60.0, elapsed
    ctx.gdsw_set_local_sweep(True, 0)
    b = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    ctx.gdsw_rhs_lift(b)
    x = torch.zeros_like(b)
    info = ctx.gdsw_solve(b, x)
    assert info.status == 0 and info.relres <= 1e-10
    ctx.close()
