"""Pins of the oracle's Q2 / P1-disc variant (the paper's own element pair, Section 2) and of
its two- to four-level GDSW coarse spaces.

The pressure is discontinuous: per fluid element the coefficients of 1, xi, eta, zeta in the
element's reference coordinates.  No pressure dof lies on the subdomain interface, so the
pressure part of the null space enters the coarse space as one column per subdomain (the
constant pressure on the subdomain's elements, Section 2.1's remark that the pressure
coupling has to be supplied), and each overlapping subdomain keeps the pressure dofs of the
elements that do not touch its artificial boundary.  The tests use closed forms, brute-force
geometric counts, special cases and invariants, as the Q2/Q1 pins do.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from paper_2606_01433_gb300 import inputs as I
from oracle import fem, fgmres, gdsw


def _exact_p1disc_pressure(p, mesh, G=1.0):
    """p = G (1 - x) per element: x = x_c + (h/2) xi, so the coefficients are
    (G (1 - x_c), -G h / 2, 0, 0)."""
    ctr = I.element_centers(p.nx, p.ny, p.nz, p.h, p.origin)[mesh.elems]
    out = np.zeros((mesh.elems.size, 4))
    out[:, 0] = G * (1.0 - ctr[:, 0])
    out[:, 1] = -0.5 * G * p.h
    return out


# --------------------------------------------------------------------------- closed form
@pytest.mark.parametrize("parts", [(1, 1, 1), (2, 2, 2), (2, 1, 2)])
def test_p1disc_poiseuille_closed_form(parts):
    """Section 2 weak form with the Q2 / P1-disc pair: Poiseuille's velocity is quadratic and
    its pressure linear, so both lie in the discrete spaces and the discrete solution equals
    the analytic one to rounding -- by a direct solve and by two-level GDSW-FGMRES."""
    p = I.poiseuille(4, parts=parts, pressure="p1disc")
    S = fem.assemble(p)
    mesh = S["mesh"]
    assert mesh.np_ == 4 * mesh.elems.size
    b = fem.lifted_rhs(S)
    ue, _ = I.poiseuille_exact(p)
    pe = _exact_p1disc_pressure(p, mesh)
    x = spla.spsolve(S["A"].tocsc(), b)
    u, pc = fem.full_solution(S, x)
    assert np.abs(u[mesh.active] - ue[mesh.active]).max() < 1e-11
    assert np.abs(pc - pe).max() < 1e-10
    P = gdsw.GDSW(S, p)
    x2, info = fgmres.fgmres(lambda v: S["A"] @ v, b, P.apply, tol=1e-13)
    u2, pc2 = fem.full_solution(S, x2)
    assert info["converged"]
    assert np.abs(u2[mesh.active] - ue[mesh.active]).max() < 1e-11
    assert np.abs(pc2 - pe).max() < 1e-10


def test_p1disc_divergence_closed_form():
    """The divergence rows -int_e psi_k div u for u = (x^2, y z, 0), which is in Q2: div u =
    2x + z, so with x = x_c + (h/2) xi and z = z_c + (h/2) zeta on the element of centre c
    and edge h the four rows are -(2 x_c + z_c) h^3, -h^4 / 3, 0 and -h^4 / 6."""
    p = I.box_problem(3, 2, 2, (1, 1, 1), bc="neumann", pressure="p1disc")
    S = fem.assemble(p)
    mesh = S["mesh"]
    assert mesh.dnodes.size == 0
    x = p.node_coords()
    u = np.zeros((p.n_nodes, 3))
    u[:, 0] = x[:, 0] ** 2
    u[:, 1] = x[:, 1] * x[:, 2]
    xv = u[mesh.vnodes].ravel()
    Bu = (S["A"][mesh.nu:, :mesh.nu] @ xv).reshape(-1, 4)
    h = p.h
    ctr = I.element_centers(p.nx, p.ny, p.nz, h, p.origin)[mesh.elems]
    expect = np.stack([-(2 * ctr[:, 0] + ctr[:, 2]) * h ** 3, np.full(len(ctr), -h ** 4 / 3),
                       np.zeros(len(ctr)), np.full(len(ctr), -h ** 4 / 6)], axis=1)
    assert np.abs(Bu - expect).max() < 1e-15
    # the pressure-pressure block is zero (no stabilisation)
    assert abs(S["A"][mesh.nu:, mesh.nu:]).max() == 0


# --------------------------------------------------------------------------- overlap sets
def _box_p1disc_kept(p, parts):
    """Pressure dofs of every overlapping subdomain of a box partition of an uncarved box,
    counted axis by axis: the part's element range [lo, hi) grows by one layer to
    [lo', hi'); element a keeps its four pressure dofs when none of its nodes lies on the
    grown box's artificial boundary, i.e. (a > lo' or a = lo' = 0) and
    (a + 1 < hi' or a + 1 = hi' = m) on every axis."""
    dims = (p.nx, p.ny, p.nz)
    n_vel = 3 * int(((p.tags != I.TAG_WALL) & (p.tags != I.TAG_INFLOW)).sum())
    out = []
    for bz in range(parts[2]):
        for by in range(parts[1]):
            for bx in range(parts[0]):
                keep = []
                for b, q, m in zip((bx, by, bz), parts, dims):
                    lo, hi = b * m // q, (b + 1) * m // q
                    lo2, hi2 = max(lo - 1, 0), min(hi + 1, m)
                    keep.append([a for a in range(m)
                                 if (a > lo2 or a == lo2 == 0) and (a + 1 < hi2 or a + 1 == hi2 == m)])
                els = sorted(a + p.nx * (b + p.ny * c) for c in keep[2] for b in keep[1] for a in keep[0])
                out.append(np.array([n_vel + 4 * e + k for e in els for k in range(4)], dtype=np.int64))
    return out


@pytest.mark.parametrize("m,parts", [(6, (3, 3, 3)), (4, (2, 2, 2)), (6, (2, 3, 1))])
def test_p1disc_overlap_pressure_sets(m, parts):
    """Section 2.1 homogeneous Dirichlet data on the artificial boundary, for the element
    pressure: the oracle's local dof sets hold exactly the pressure dofs of the elements of
    Omega_i' that do not touch its artificial boundary (box-geometric count), plus the same
    velocity dofs as with Q1 pressure."""
    p = I.unit_cube(m, parts=parts)
    p.pressure = "p1disc"
    S = fem.assemble(p)
    nu = S["mesh"].nu
    got = gdsw.overlapping_dofs(S, p)
    lev, _ = gdsw.build_level1(S, p)
    pq = I.unit_cube(m, parts=parts)
    vel = gdsw.overlapping_dofs(fem.assemble(pq), pq)
    expect = _box_p1disc_kept(p, parts)
    assert len(got) == len(expect)
    for a, c, e, v in zip(got, lev.dofs, expect, vel):
        assert np.array_equal(a, c)
        assert np.array_equal(a[a >= nu], e)
        assert np.array_equal(a[a < nu], v[v < nu])


# --------------------------------------------------------------------------- special cases
def test_p1disc_one_subdomain_is_direct_solve():
    """One subdomain: no interface, an empty coarse space, A_1 = A, so B = A^{-1} and FGMRES
    takes one iteration."""
    p = I.box_problem(3, 3, 3, (1, 1, 1), form="symmetric", uk_seed=7, lam=1.0, n=0.5, nu_inf=1e-3,
                      pressure="p1disc")
    S = fem.assemble(p)
    P = gdsw.GDSW(S, p)
    assert P.levels[0].n0 == 0
    r = np.random.default_rng(0).standard_normal(S["A"].shape[0])
    zd = spla.spsolve(S["A"].tocsc(), r)
    assert np.linalg.norm(P.apply(r) - zd) <= 1e-12 * np.linalg.norm(zd)
    x, info = fgmres.fgmres(lambda v: S["A"] @ v, r, P.apply, tol=1e-10)
    assert info["iterations"] == 1


def test_p1disc_pressure_columns_and_translations():
    """Section 2.1 null space: on the all-wall cavity every subdomain's pressure column is the
    constant pressure on that subdomain's elements (zero velocity, zero linear coefficients),
    since -B^T 1 vanishes on velocity dofs that are zero on the subdomain's boundary; on the
    pure-Neumann operator the sum of the translation-c columns is the constant field e_c."""
    p = I.box_problem(4, 4, 4, (2, 2, 2), bc="cavity", pressure="p1disc")
    S = fem.assemble(p)
    mesh = S["mesh"]
    lev, _ = gdsw.build_level1(S, p)
    N = 8
    n_ent = sum(len(d) for (s, d, m) in lev.coarse_nodes if len(s) >= 2)
    assert lev.n0 == n_ent + N
    assert [tuple(s) for (s, d, m) in lev.coarse_nodes if len(s) == 1] == [(i,) for i in range(N)]
    sub = p.part[mesh.elems]
    for i in range(N):
        v = lev.Phi[:, n_ent + i].toarray().ravel()
        expect = np.zeros(lev.n)
        expect[mesh.nu + 4 * np.nonzero(sub == i)[0]] = 1.0
        assert np.abs(v - expect).max() < 1e-12
    pn = I.box_problem(4, 4, 4, (2, 2, 2), bc="neumann", pressure="p1disc")
    Sn = fem.assemble(pn)
    levn, _ = gdsw.build_level1(Sn, pn)
    for c in range(3):
        cols = [d[m.index(c)] for (s, d, m) in levn.coarse_nodes if c in m]
        e = np.zeros(levn.n0); e[cols] = 1.0
        expect = np.zeros(levn.n); expect[c:Sn["mesh"].nu:3] = 1.0
        assert np.abs(levn.Phi @ e - expect).max() < 1e-12


def test_p1disc_extension_and_invertibility():
    """Section 2.1 extension Phi_I = -A_II^{-1} A_IGamma Phi_Gamma: (A Phi)_I = 0; Gamma (the
    interface velocity dofs and the element constants) and the interiors (interior velocity
    and the linear pressure dofs of each subdomain's elements) partition the free dofs; every
    local matrix and every A_II is invertible (smallest singular value), and so is A_0."""
    p = I.box_problem(4, 4, 2, (2, 2, 1), form="symmetric", uk_seed=3, lam=1.0, n=0.5, nu_inf=1e-2,
                      pressure="p1disc")
    S = fem.assemble(p)
    A = S["A"]
    nu = S["mesh"].nu
    lev, A0 = gdsw.build_level1(S, p)
    AP = (A @ lev.Phi).toarray()
    inter = np.concatenate(lev.interior)
    assert np.abs(AP[inter]).max() < 1e-12 * np.abs(AP).max()
    G = np.nonzero(lev.gamma)[0]
    assert G.size + inter.size == lev.n and np.union1d(G, inter).size == lev.n
    assert np.array_equal(G[G >= nu], nu + 4 * np.arange(S["mesh"].elems.size))
    assert np.array_equal(np.sort(inter[inter >= nu]),
                          np.setdiff1d(nu + np.arange(4 * S["mesh"].elems.size), G[G >= nu]))
    for d in list(lev.dofs) + list(lev.interior):
        s = np.linalg.svd(A[d][:, d].toarray(), compute_uv=False)
        assert s[-1] > 1e-10 * s[0]
    s = np.linalg.svd(A0, compute_uv=False)
    assert s[-1] > 1e-10 * s[0]


@pytest.mark.parametrize("weighting", ["plain", "pou"])
def test_p1disc_brute_force_dense(weighting):
    """Section 2.1 two-level preconditioner written out with dense numpy inverses of every
    local matrix and of A_0 = Phi^T A Phi; the oracle's apply equals it column by column, the
    plain form is symmetric, and FGMRES reaches the dense solution."""
    p = I.box_problem(3, 2, 2, (3, 2, 1), form="symmetric", uk_seed=5, lam=1.0, n=0.5, nu_inf=1e-3,
                      pressure="p1disc")
    S = fem.assemble(p)
    A = S["A"].toarray()
    P = gdsw.GDSW(S, p, weighting=weighting)
    lev = P.levels[0]
    n = A.shape[0]
    B = np.zeros((n, n))
    for d, w in zip(lev.dofs, lev.weights):
        Dw = np.diag(w) if weighting == "pou" else np.eye(d.size)
        B[np.ix_(d, d)] += Dw @ np.linalg.inv(A[np.ix_(d, d)])
    Phi = lev.Phi.toarray()
    B += Phi @ np.linalg.inv(Phi.T @ A @ Phi) @ Phi.T
    for j in np.random.default_rng(2).choice(n, size=40, replace=False):
        e = np.zeros(n); e[j] = 1.0
        assert np.abs(P.apply(e) - B[:, j]).max() <= 1e-12 * max(1.0, np.abs(B).max())
    if weighting == "plain":
        assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    b = I.random_rhs(n, 3)
    x, info = fgmres.fgmres(lambda v: S["A"] @ v, b, P.apply, tol=1e-12)
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


def _brute_force(P, level=0):
    """Section 2.2 recursion written out with dense numpy inverses (plain weighting)."""
    lev = P.levels[level]
    A = P.A0[level].toarray() if hasattr(P.A0[level], "toarray") else P.A0[level]
    B = np.zeros((lev.n, lev.n))
    for d in lev.dofs:
        B[np.ix_(d, d)] += np.linalg.inv(A[np.ix_(d, d)])
    if lev.n0 == 0:
        return B
    Phi = lev.Phi.toarray() if hasattr(lev.Phi, "toarray") else lev.Phi
    inner = np.linalg.inv(P.A0[level + 1]) if level + 1 == len(P.levels) else _brute_force(P, level + 1)
    return B + Phi @ inner @ Phi.T


@pytest.mark.parametrize("L", [3, 4])
def test_p1disc_multilevel_brute_force(L):
    """Section 2.2 four-level equation with the P1-disc coarse spaces: on every coarse level a
    part's pressure column is a coarse node of that part alone, so the next level adds one
    pressure column per part; the oracle's apply equals the dense recursion built with numpy
    inverses, the plain form is symmetric, every local and interior matrix is invertible, and
    FGMRES reaches the dense solution."""
    groups = ((2, 2, 1),) if L == 3 else ((2, 2, 1), (2, 1, 1))
    p = I.box_problem(4, 4, 2, (4, 4, 2), groups=groups, levels=L, form="symmetric", uk_seed=1, lam=1.0, n=0.5,
                      nu_inf=1e-3, pressure="p1disc")
    S = fem.assemble(p)
    P = gdsw.GDSW(S, p, weighting="plain")
    n = S["A"].shape[0]
    B = _brute_force(P)
    for j in np.random.default_rng(4).choice(n, size=30, replace=False):
        e = np.zeros(n); e[j] = 1.0
        assert np.abs(P.apply(e) - B[:, j]).max() <= 1e-11 * max(1.0, np.abs(B).max())
    assert np.abs(B - B.T).max() <= 1e-11 * np.abs(B).max()
    for l, lev in enumerate(P.levels):
        A = P.A0[l].toarray() if hasattr(P.A0[l], "toarray") else P.A0[l]
        for d in list(lev.dofs) + [i for i in lev.interior if i.size]:
            s = np.linalg.svd(A[np.ix_(d, d)], compute_uv=False)
            assert s[-1] > 1e-10 * s[0]
    b = I.random_rhs(n, 3)
    x, info = fgmres.fgmres(lambda v: S["A"] @ v, b, P.apply, tol=1e-12)
    xd = spla.spsolve(S["A"].tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


def test_p1disc_coarse_pressure_columns_by_hand():
    """The coarse-level readings written out for a 4 x 4 x 2 box of 32 one-element subdomains
    grouped 2 x 2 x 1 into 8 parts (all-wall cavity): (a) a level-2 local set holds the
    pressure columns of its own part's four subdomains and no other; (b) the level-2 pressure
    column of part J, carried down through both bases, is the constant pressure on the elements
    of J's subdomains (zero velocity, zero slopes); (c) it is a one-part coarse node of the
    next level."""
    p = I.box_problem(4, 4, 2, (4, 4, 2), groups=((2, 2, 1),), levels=3, bc="cavity", pressure="p1disc")
    S = fem.assemble(p)
    mesh = S["mesh"]
    P = gdsw.GDSW(S, p)
    lev1, lev2 = P.levels
    n_ent1 = sum(len(d) for (s, d, m) in lev1.coarse_nodes if len(s) >= 2)
    assert lev1.n0 == n_ent1 + 32
    group = np.asarray(p.groups[0])
    for J in range(8):
        pcol = n_ent1 + np.arange(32)
        mine = np.intersect1d(lev2.dofs[J], pcol)
        assert np.array_equal(mine, np.sort(n_ent1 + np.nonzero(group == J)[0]))
    n_ent2 = sum(len(d) for (s, d, m) in lev2.coarse_nodes if len(s) >= 2)
    assert lev2.n0 == n_ent2 + 8
    assert [tuple(s) for (s, d, m) in lev2.coarse_nodes if len(s) == 1] == [(J,) for J in range(8)]
    Phi1 = lev1.Phi.toarray()
    sub = p.part[mesh.elems]
    for J in range(8):
        e2 = np.zeros(lev2.n0); e2[n_ent2 + J] = 1.0
        v = Phi1 @ (lev2.Phi @ e2)
        expect = np.zeros(lev1.n)
        expect[mesh.nu + 4 * np.nonzero(np.isin(sub, np.nonzero(group == J)[0]))[0]] = 1.0
        assert np.abs(v - expect).max() < 1e-11
