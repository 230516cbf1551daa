"""GPU parity of the Q2 / P1-disc variant (the paper's element pair, Section 2) with its
two- to four-level GDSW coarse spaces, through the C ABI, against the FP64 CPU oracle.

The pressure is discontinuous (four dofs per fluid element); no pressure dof lies on the
interface, so the coarse space holds the entity translations plus one pressure column per
subdomain (the constant on the subdomain's elements), and every coarse level one per part.
Tolerances as in the Q2/Q1 parity tests: single FP64 steps <= 1e-12 (operator <= 1e-14),
apply <= 1e-11, FP64 solve <= 1e-10 with iterations +-1, mixed FP32 / BF16 local factors
forward error <= 1e-8.
"""
import numpy as np
import pytest

from paper_2606_01433_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32 = (("fp32", "fp32", "fp32"), "fp32")
BF16 = (("bf16", "fp32", "fp32"), "fp32")


def _p1(p):
    p.pressure = "p1disc"
    return p


PROBLEMS = {
    "box6_carreau": lambda: _p1(I.box_problem(6, 6, 6, (3, 2, 2), levels=2, form="symmetric", uk_seed=3, lam=1.0,
                                              n=0.5, nu_inf=1e-3)),
    "channel16_obstacles": lambda: _p1(I.channel(16, parts=(4, 4, 4), groups=(), levels=2)),
    "die_rcb": lambda: _p1(I.die(16, 16, 32, nparts=16, per_group=4, levels=2)),
    "channel12_3lvl": lambda: _p1(I.channel(12, parts=(4, 4, 4), groups=((2, 2, 2),), levels=3)),
    "die_rcb_4lvl": lambda: _p1(I.die(16, 16, 32, nparts=32, per_group=4, levels=4)),
}

_cache = {}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_01433_gb300 import gdsw
    gdsw.load()
    return gdsw


def oracle_for(name, weighting="pou"):
    from oracle import fem, gdsw as og
    key = (name, weighting)
    if key not in _cache:
        p = PROBLEMS[name]()
        S = fem.assemble(p)
        _cache[key] = (p, S, og.GDSW(S, p, weighting=weighting))
    return _cache[key]


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_p1disc_operator(lib, name):
    """Section 2 assembly with the element pressure (B rows 4 f + k), SpMV and lifting."""
    from oracle import fem
    p, S, P = oracle_for(name)
    ctx = lib.Context(p)
    assert ctx.sizes.n_p == 4 * S["mesh"].elems.size
    Ag = ctx.gdsw_matrix_csr()
    assert abs(Ag - S["A"]).max() <= 1e-14 * abs(S["A"]).max()
    x = np.random.default_rng(0).standard_normal(ctx.n)
    y = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    ctx.gdsw_spmv(dev(x), y)
    assert rel(host(y), S["A"] @ x) <= 1e-14
    b = torch.full_like(y, float("nan"))
    ctx.gdsw_rhs_lift(b)
    assert rel(host(b), fem.lifted_rhs(S)) <= 1e-13
    ctx.close()


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("weighting", ["pou", "plain"])
def test_p1disc_level_steps(lib, name, weighting):
    """Sections 2.1 / 2.2 with the P1-disc sets on every level: local branch (the element
    pressure of Omega_i' kept away from its rim; a coarse part's own pressure columns only),
    Phi^T r, Phi x (per-part pressure columns) and A_0."""
    p, S, P = oracle_for(name, weighting)
    ctx = lib.Context(p, weighting=weighting)
    rng = np.random.default_rng(1)
    for l, lev in enumerate(P.levels):
        assert int(ctx.sizes.n_coarse[l]) == lev.n0
        r = rng.standard_normal(lev.n)
        z = torch.zeros(lev.n, dtype=torch.float64, device="cuda")
        ctx.gdsw_apply_local(l, dev(r), z)
        assert rel(host(z), lev.apply_local(r, weighting)) <= 1e-12, (l, "local")
        r0 = torch.zeros(lev.n0, dtype=torch.float64, device="cuda")
        ctx.gdsw_restrict(l, dev(r), r0)
        assert rel(host(r0), lev.Phi.T @ r) <= 1e-12, (l, "restrict")
        x0 = rng.standard_normal(lev.n0)
        z2 = torch.zeros(lev.n, dtype=torch.float64, device="cuda")
        ctx.gdsw_prolong(l, dev(x0), z2)
        assert rel(host(z2), lev.Phi @ x0) <= 1e-12, (l, "prolong")
        assert rel(ctx.gdsw_coarse_matrix(l), P.A0[l + 1]) <= 1e-12, (l, "A0")
    ctx.close()


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_p1disc_apply_and_solve(lib, name):
    """Two- to four-level apply and FP64 FGMRES: solution within 1e-10 of the oracle's, iterations
    +-1; then FP32 and BF16 local factors reach the FP64 solution to 1e-8."""
    from oracle import fem, fgmres
    p, S, P = oracle_for(name)
    ctx = lib.Context(p, tol=1e-10)
    r = np.random.default_rng(2).standard_normal(ctx.n)
    z = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    ctx.gdsw_apply(dev(r), z)
    assert rel(host(z), P.apply(r)) <= 1e-11
    b = fem.lifted_rhs(S) if p.rhs_seed is None else I.random_rhs(ctx.n, p.rhs_seed)
    xo, io = fgmres.fgmres(lambda v: S["A"] @ v, b, P.apply, tol=1e-10)
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    info = ctx.gdsw_solve(dev(b), x)
    assert info.status == 0 and abs(info.iterations - io["iterations"]) <= 1
    assert rel(host(x), xo) <= 1e-10
    ctx.close()
    x13, _ = fgmres.fgmres(lambda v: S["A"] @ v, b, P.apply, tol=1e-13)
    for prec in (FP32, BF16):
        cm = lib.Context(p, precision=prec[0], phi_precision=prec[1], tol=1e-12)
        x = torch.zeros(cm.n, dtype=torch.float64, device="cuda")
        info = cm.gdsw_solve(dev(b), x)
        assert info.status == 0 and rel(host(x), x13) <= 1e-8, prec
        cm.close()


def test_p1disc_poiseuille_and_degenerate_cases(lib):
    """Closed form on the GPU (Poiseuille's linear pressure is in P1-disc) and one subdomain
    (empty coarse space, one FGMRES step)."""
    from oracle import fem
    p = I.poiseuille(4, parts=(2, 2, 2), pressure="p1disc")
    S = fem.assemble(p)
    ctx = lib.Context(p, tol=1e-13)
    b = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    ctx.gdsw_rhs_lift(b)
    x = torch.zeros_like(b)
    info = ctx.gdsw_solve(b, x)
    assert info.status == 0
    u, pc = fem.full_solution(S, host(x))
    ue, _ = I.poiseuille_exact(p)
    m = S["mesh"]
    assert np.abs(u[m.active] - ue[m.active]).max() < 1e-11
    ctr = I.element_centers(p.nx, p.ny, p.nz, p.h, p.origin)[m.elems]
    assert np.abs(pc[:, 0] - (1.0 - ctr[:, 0])).max() < 1e-10
    assert np.abs(pc[:, 1] + 0.5 * p.h).max() < 1e-10 and np.abs(pc[:, 2:]).max() < 1e-10
    ctx.close()
    p1 = I.box_problem(3, 3, 3, (1, 1, 1), form="symmetric", uk_seed=7, lam=1.0, n=0.5, nu_inf=1e-3,
                       pressure="p1disc")
    c1 = lib.Context(p1, tol=1e-10)
    assert int(c1.sizes.n_coarse[0]) == 0
    r = I.random_rhs(c1.n, 4)
    x = torch.zeros(c1.n, dtype=torch.float64, device="cuda")
    info = c1.gdsw_solve(dev(r), x)
    assert info.status == 0 and info.iterations == 1
    c1.close()
