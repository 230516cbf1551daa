"""GPU parity of the geometric multigrid whose coarse solver is the multilevel GDSW method
(Section 3), through the C ABI, against the oracle's multigrid (oracle/mg.py) on the same
seeded nested grids.

Tolerances: transfers are the same sparse products (<= 1e-14 relative); an FP64 smoothing
sweep uses FP64 patch inverses (explicit inverse against the oracle's numpy inverse, <= 1e-10);
one V-cycle with an essentially exact coarse solve (coarse FGMRES to 1e-13) <= 1e-9; the
V-cycle-preconditioned FGMRES with the paper's 1e-1 coarse solve reaches the direct solution
to 1e-8 (FP32 and FP64 smoothing), its iteration count within +-2 of the oracle's (FP64)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = {
    "two_grid_newtonian": lambda: I.mg_hierarchy(8, 2, parts=(2, 2, 2), groups=(), levels=2, carreau=False),
    "two_grid_carreau": lambda: I.mg_hierarchy(8, 2, parts=(2, 2, 2), groups=(), levels=2, carreau=True),
    "three_grid_carreau": lambda: I.mg_hierarchy(16, 3, parts=(2, 2, 2), groups=(), levels=2, carreau=True),
}


@pytest.mark.parametrize("name,symmetric", [("two_grid_newtonian", False), ("three_grid_carreau", False),
                                            ("three_grid_carreau", True)])
def test_mg_components(lib, name, symmetric):
    from oracle import mg
    probs = CASES[name]()
    M = mg.Multigrid(probs, pre=2, post=2, coarse_tol=1e-13, symmetric=symmetric)
    G = lib.Multigrid(probs, pre=2, post=2, smoother="fp64", coarse_tol=1e-13, coarse_precision=("fp64",) * 3,
                      coarse_phi="fp64", symmetric=symmetric)
    rng = np.random.default_rng(11)
    for l in range(len(probs) - 1):
        nf, nc = M.A[l].shape[0], M.A[l + 1].shape[0]
        xc = rng.standard_normal(nc)
        z = torch.zeros(nf, dtype=torch.float64, device="cuda")
        G.gdsw_mg_prolong(l, dev(xc), z)
        assert rel(host(z), M.P[l] @ xc) <= 1e-14
        rf = rng.standard_normal(nf)
        rc = torch.zeros(nc, dtype=torch.float64, device="cuda")
        G.gdsw_mg_restrict(l, dev(rf), rc)
        assert rel(host(rc), M.R[l] @ rf) <= 1e-14
        b = rng.standard_normal(nf)
        x = torch.zeros(nf, dtype=torch.float64, device="cuda")
        G.gdsw_mg_smooth(l, dev(b), x, 1)
        assert rel(host(x), M.smoothers[l].smooth(b, np.zeros(nf), 1)) <= 1e-10, l
    r = rng.standard_normal(M.A[0].shape[0])
    z = torch.zeros_like(dev(r))
    G.gdsw_mg_vcycle(dev(r), z)
    assert rel(host(z), M.vcycle(r)) <= 1e-9
    G.close()


@pytest.mark.parametrize("name", ["two_grid_newtonian", "two_grid_carreau"])
@pytest.mark.parametrize("smoother", ["fp32", "fp64"])
def test_mg_solve(lib, name, smoother):
    from oracle import fgmres, mg
    probs = CASES[name]()
    M = mg.Multigrid(probs, pre=2, post=2, coarse_tol=1e-1)
    A = M.A[0]
    b = I.random_rhs(A.shape[0], 4)
    _, io = fgmres.fgmres(lambda v: A @ v, b, M.vcycle, tol=1e-8)
    xd = spla.spsolve(A.tocsc(), b)
    G = lib.Multigrid(probs, pre=2, post=2, smoother=smoother, coarse_tol=1e-1, tol=1e-8)
    x = torch.zeros(G.n, dtype=torch.float64, device="cuda")
    info = G.solve(dev(b), x)
    assert info.status == 0 and info.relres <= 1e-8
    assert abs(info.iterations - io["iterations"]) <= 2, (info.iterations, io["iterations"])
    st = G.gdsw_mg_stats()
    assert st["cycles"] >= info.iterations and st["coarse_solves"] == st["cycles"]
    G.close()
    G = lib.Multigrid(probs, pre=2, post=2, smoother=smoother, coarse_tol=1e-1, tol=1e-12)
    x = torch.zeros(G.n, dtype=torch.float64, device="cuda")
    info = G.solve(dev(b), x)
    assert info.status == 0
    assert rel(host(x), xd) <= 1e-8
    G.close()


def test_mg_rejects_bad_grids(lib):
    """Grids that are not nested, or a fine grid with a Schwarz preconditioner, are refused
    with GDSW_ERR_INVALID_ARG and a reason."""
    probs = I.mg_hierarchy(8, 2, parts=(2, 2, 2), groups=(), levels=2, carreau=False)
    other = I.mg_hierarchy(6, 2, parts=(2, 2, 2), groups=(), levels=2, carreau=False)
    with pytest.raises(lib.GdswError) as e:
        lib.Multigrid([probs[0], other[1]])
    assert e.value.code == lib.GDSW_ERR_INVALID_ARG and "nested" in str(e.value)


@pytest.mark.parametrize("smoother", ["fp32", "fp64"])
def test_mg_launch_chain_is_bitwise_neutral(lib, smoother):
    """The chained launches of the smoother, transfers and Krylov kernels change no number:
    V-cycles and the preconditioned solve are bitwise equal with the chain on and off."""
    probs = CASES["three_grid_carreau"]()
    b = None
    out = []
    try:
        for on in (True, False):
            lib.set_launch_overlap(on)
            G = lib.Multigrid(probs, pre=2, post=2, smoother=smoother, coarse_tol=1e-1, tol=1e-10, symmetric=True)
            if b is None:
                b = I.random_rhs(G.n, 6)
            z = torch.zeros(G.n, dtype=torch.float64, device="cuda")
            G.gdsw_mg_vcycle(dev(b), z)
            x = torch.zeros_like(z)
            info = G.solve(dev(b), x)
            assert info.status == 0
            out.append((host(z), info.iterations, host(x)))
            G.close()
    finally:
        lib.set_launch_overlap(True)
    (z1, i1, x1), (z2, i2, x2) = out
    assert np.array_equal(z1, z2) and i1 == i2 and np.array_equal(x1, x2)
