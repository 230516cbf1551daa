"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

Each test names the passage it checks.  None of them re-derives the oracle's own formula:
they use closed forms, special cases that reduce to a direct solve, invariants of the
construction, brute-force dense matrices and textbook optimality.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from paper_2606_01433_gb300 import inputs as I
from oracle import fem, gdsw, fgmres


def _solve_poiseuille(parts, m=4, levels=2, groups=None):
    p = I.poiseuille(m, parts=parts, groups=groups, levels=levels)
    S = fem.assemble(p)
    return p, S, fem.lifted_rhs(S)


# --------------------------------------------------------------------------- P1
@pytest.mark.parametrize("parts", [(1, 1, 1), (2, 2, 2), (2, 1, 2)])
def test_poiseuille_closed_form(parts):
    """Section 2 weak form (gradient form, do-nothing outflow): the Poiseuille flow
    u = (G/2) y (1-y) e_x, p = G (1-x) lies in Q2/Q1, so the discrete solution equals it
    to rounding -- by a direct solve and by GDSW-preconditioned FGMRES."""
    p, S, b = _solve_poiseuille(parts)
    ue, pe = I.poiseuille_exact(p)
    mesh = S["mesh"]
    x = spla.spsolve(S["A"].tocsc(), b)
    u, pr = fem.full_solution(S, x)
    assert np.abs(u[mesh.active] - ue[mesh.active]).max() < 1e-11
    assert np.abs(pr[mesh.pnodes] - pe[mesh.pnodes]).max() < 1e-10
    P = gdsw.GDSW(S, p)
    x2, info = fgmres.fgmres(lambda v: S["A"] @ v, b, P.apply, tol=1e-13)
    u2, pr2 = fem.full_solution(S, x2)
    assert info["converged"]
    assert np.abs(u2[mesh.active] - ue[mesh.active]).max() < 1e-11
    assert np.abs(pr2[mesh.pnodes] - pe[mesh.pnodes]).max() < 1e-10


# --------------------------------------------------------------------------- operator pins
def test_stiffness_closed_forms():
    """Section 2 / 3 bilinear forms on a pure-Neumann box (no Dirichlet dof):
    u = x e_x gives u^T A u = nu |Omega| (gradient form) and 2 nu |Omega| (symmetric form,
    2 D:D = 2); translations are in the kernel of both; rotations only in the kernel of the
    symmetric form; and sum_P (B u)_P = -int div u = -|Omega|."""
    for form, expect in (("gradient", 1.0), ("symmetric", 2.0)):
        p = I.box_problem(3, 2, 2, (1, 1, 1), form=form, bc="neumann", nu0=1.7)
        S = fem.assemble(p)
        mesh = S["mesh"]
        A = S["A"]
        x = p.node_coords()[mesh.vnodes]
        vol = (3 * p.h) * (2 * p.h) * (2 * p.h)
        u = np.zeros((mesh.vnodes.size, 3)); u[:, 0] = x[:, 0]
        z = np.concatenate([u.ravel(), np.zeros(mesh.np_)])
        Az = A @ z
        assert abs(z[:mesh.nu] @ Az[:mesh.nu] - expect * 1.7 * vol) < 1e-12
        assert abs(Az[mesh.nu:].sum() + vol) < 1e-12
        for c in range(3):
            t = np.zeros((mesh.vnodes.size, 3)); t[:, c] = 1.0
            zt = np.concatenate([t.ravel(), np.zeros(mesh.np_)])
            assert np.abs((A @ zt)[:mesh.nu]).max() < 1e-12
        rot = np.zeros((mesh.vnodes.size, 3)); rot[:, 0] = -x[:, 1]; rot[:, 1] = x[:, 0]
        zr = np.concatenate([rot.ravel(), np.zeros(mesh.np_)])
        r = np.abs((A @ zr)[:mesh.nu]).max()
        if form == "symmetric":
            assert r < 1e-12
        else:
            assert r > 1e-3


# --------------------------------------------------------------------------- P9
def test_carreau_closed_form():
    """Section 3 Carreau law: for the linear field u = (y, 0, 0) (simple shear, gamma_dot = 1)
    and u = (x, -y, 0) (extension, gamma_dot = 2) the Q2 interpolant is exact, so nu at every
    Gauss point equals nu_inf + (nu0 - nu_inf)(1 + lambda^2 gamma_dot^2)^((n-1)/2)."""
    nu0, nu_inf, lam, n = 3.0, 0.25, 2.0, 0.5
    p = I.box_problem(2, 2, 2, (1, 1, 1), form="symmetric", bc="neumann",
                      nu0=nu0, nu_inf=nu_inf, lam=lam, n=n)
    x = p.node_coords()
    mesh = fem.Mesh(p)
    tabs = fem.reference_tables()
    p.uk = np.zeros_like(x); p.uk[:, 0] = x[:, 1]
    nu = fem.quadrature_viscosity(mesh, tabs)
    assert np.allclose(nu, nu_inf + (nu0 - nu_inf) * 5.0 ** -0.25, rtol=0, atol=1e-13)
    p.uk = np.zeros_like(x); p.uk[:, 0] = x[:, 0]; p.uk[:, 1] = -x[:, 1]
    nu = fem.quadrature_viscosity(mesh, tabs)
    assert np.allclose(nu, nu_inf + (nu0 - nu_inf) * 17.0 ** -0.25, rtol=0, atol=1e-13)
    # n = 1 (or lambda = 0) is the Newtonian symmetric form with nu0
    p.n_carreau = 1.0
    A1 = fem.assemble(p)["A"]
    p.uk = None
    A0 = fem.assemble(p)["A"]
    assert abs(A1 - A0).max() < 1e-13


# --------------------------------------------------------------------------- P2
def test_one_subdomain_is_direct_solve():
    """Section 2.1 additive sum with N = 1: Gamma is empty and A_1 = A, so B = A^{-1} and
    FGMRES converges in one iteration."""
    p = I.box_problem(3, 3, 3, (1, 1, 1), form="symmetric", uk_seed=7, lam=1.0, n=0.5, nu_inf=1e-3)
    S = fem.assemble(p)
    P = gdsw.GDSW(S, p)
    assert P.levels[0].n0 == 0
    r = np.random.default_rng(0).standard_normal(S["A"].shape[0])
    z = P.apply(r)
    zd = spla.spsolve(S["A"].tocsc(), r)
    assert np.linalg.norm(z - zd) <= 1e-12 * np.linalg.norm(zd)
    x, info = fgmres.fgmres(lambda v: S["A"] @ v, r, P.apply, tol=1e-10)
    assert info["iterations"] == 1


# --------------------------------------------------------------------------- P3
def test_partition_of_unity():
    """The 'pou' weights sum to one: sum_i R_i^T D_i R_i 1 = 1 exactly, on the first
    level and on a coarse level."""
    p = I.box_problem(4, 4, 4, (2, 2, 2), groups=((2, 2, 1),), levels=3)
    S = fem.assemble(p)
    P = gdsw.GDSW(S, p)
    for lev in P.levels:
        s = np.zeros(lev.n)
        for d, w in zip(lev.dofs, lev.weights):
            s[d] += w
        assert np.array_equal(s, np.ones(lev.n))


# --------------------------------------------------------------------------- entity count
@pytest.mark.parametrize("m,parts,n0", [(4, (2, 2, 2), 76), (8, (4, 4, 4), 1116)])
def test_coarse_dimension_box(m, parts, n0):
    """Section 2.1 entities for a box partition of a cube: 3 q^2 (q-1) faces,
    3 (q-1)^2 q edge segments... gives 19 entities (2x2x2) and 279 (4x4x4), each with
    three translations and one pressure constant."""
    p = I.unit_cube(m, parts=parts)
    S = fem.assemble(p)
    lev, A0 = gdsw.build_level1(S, p)
    q = parts[0]
    faces = 3 * q * q * (q - 1)
    edges = 3 * (q - 1) ** 2 * q
    verts = (q - 1) ** 3
    assert len(lev.entities) == faces + edges + verts
    assert lev.n0 == n0 == 4 * (faces + edges + verts)


# --------------------------------------------------------------------------- P4
def test_constants_reproduced():
    """Section 2.1: Phi_Gamma carries the null space (translations, pressure constants), and
    the saddle-point extension reproduces it: on the pure-Neumann operator the sum of all
    translation-c columns is the constant field e_c (also on the next level, since
    A_0 1_c = Phi^T A e_c = 0); on the all-wall cavity the sum of the pressure columns is
    (u, p) = (0, 1)."""
    p = I.box_problem(4, 4, 4, (2, 2, 2), groups=((2, 1, 1),), levels=3, bc="neumann")
    S = fem.assemble(p)
    mesh = S["mesh"]
    lev, A0 = gdsw.build_level1(S, p)
    for c in range(3):
        cols = [d[m.index(c)] for (s, d, m) in lev.coarse_nodes if c in m]
        e = np.zeros(lev.n0); e[cols] = 1.0
        v = lev.Phi @ e
        expect = np.zeros(lev.n); expect[c:mesh.nu:3] = 1.0
        assert np.abs(v - expect).max() < 1e-12
        lev2, _ = gdsw.build_coarse_level(A0, lev.coarse_nodes, p.groups[0])
        cols2 = [d[m.index(c)] for (s, d, m) in lev2.coarse_nodes if c in m]
        e2 = np.zeros(lev2.n0); e2[cols2] = 1.0
        assert np.abs(lev2.Phi @ e2 - e).max() < 1e-12
    pc = I.box_problem(4, 4, 4, (2, 2, 2), bc="cavity")
    Sc = fem.assemble(pc)
    levc, _ = gdsw.build_level1(Sc, pc)
    cols = [d[m.index(3)] for (s, d, m) in levc.coarse_nodes if 3 in m]
    e = np.zeros(levc.n0); e[cols] = 1.0
    v = levc.Phi @ e
    nu = Sc["mesh"].nu
    assert np.abs(v[:nu]).max() < 1e-12 and np.abs(v[nu:] - 1.0).max() < 1e-12


# --------------------------------------------------------------------------- P5
def test_extension_property():
    """Section 2.1: Phi_I = -A_II^{-1} A_IGamma Phi_Gamma means (A Phi)_I = 0; Phi_Gamma is
    block diagonal (velocity dofs -> velocity columns, pressure dofs -> pressure columns)
    with one unit entry per interface row."""
    p = I.box_problem(4, 4, 4, (2, 2, 2), form="symmetric", uk_seed=3, lam=1.0, n=0.5, nu_inf=1e-2)
    S = fem.assemble(p)
    lev, A0 = gdsw.build_level1(S, p)
    AP = (S["A"] @ lev.Phi).toarray()
    interior = np.concatenate(lev.interior)
    assert np.abs(AP[interior]).max() < 1e-12 * np.abs(AP).max()
    PG = lev.PhiGamma.tocsr()
    G = np.nonzero(lev.gamma)[0]
    assert np.array_equal(np.diff(PG.indptr)[G], np.ones(G.size, dtype=int))
    mode = {}
    for (s, d, m) in lev.coarse_nodes:
        for dd, mm in zip(d, m):
            mode[dd] = mm
    nu = S["mesh"].nu
    for r in G:
        col = PG.indices[PG.indptr[r]]
        assert (mode[col] == 3) == (r >= nu)
        if r < nu:
            assert mode[col] == r % 3
    # Gamma and the interiors partition the free dofs
    assert G.size + interior.size == lev.n


# --------------------------------------------------------------------------- P6
def _brute_force(P, level=0):
    """Section 2.2 four-level equation written out with explicit dense inverses."""
    lev = P.levels[level]
    n = lev.n
    B = np.zeros((n, n))
    A = P.A0[level].toarray() if hasattr(P.A0[level], "toarray") else P.A0[level]
    for d, w in zip(lev.dofs, lev.weights):
        Ai = np.linalg.inv(A[np.ix_(d, d)])
        Dw = np.diag(w) if P.weighting == "pou" else np.eye(d.size)
        B[np.ix_(d, d)] += Dw @ Ai
    if lev.n0 == 0:
        return B
    Phi = lev.Phi.toarray() if hasattr(lev.Phi, "toarray") else lev.Phi
    if level + 1 == len(P.levels):
        inner = np.linalg.inv(P.A0[level + 1])
    else:
        inner = _brute_force(P, level + 1)
    return B + Phi @ inner @ Phi.T


@pytest.mark.parametrize("case", ["2lvl", "3lvl", "4lvl"])
@pytest.mark.parametrize("weighting", ["plain", "pou"])
def test_brute_force_dense(case, weighting):
    """Section 2.2 four-level equation (and its two/three-level truncations): the oracle's
    recursive apply equals the preconditioner built densely with numpy inverses, column by
    column; FGMRES with it reaches the dense solution."""
    if case == "2lvl":
        p = I.box_problem(2, 2, 2, (2, 2, 2), levels=2)
    elif case == "3lvl":
        p = I.box_problem(4, 4, 2, (4, 4, 2), groups=((2, 2, 1),), levels=3)
    else:
        p = I.box_problem(4, 4, 2, (4, 4, 2), groups=((2, 2, 1), (2, 1, 1)), levels=4)
    S = fem.assemble(p)
    P = gdsw.GDSW(S, p, weighting=weighting)
    Bd = _brute_force(P)
    n = S["A"].shape[0]
    cols = np.random.default_rng(1).choice(n, size=min(n, 40), replace=False)
    for j in cols:
        e = np.zeros(n); e[j] = 1.0
        z = P.apply(e)
        assert np.abs(z - Bd[:, j]).max() <= 1e-12 * max(1.0, np.abs(Bd).max())
    b = I.random_rhs(n, 3)
    x, info = fgmres.fgmres(lambda v: S["A"] @ v, b, P.apply, tol=1e-12)
    xd = np.linalg.solve(S["A"].toarray(), b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


# --------------------------------------------------------------------------- P7
def test_level_collapse():
    """Section 2.2 recursion: with one part on the last Schwarz level the next coarse space
    is empty and that level's local solve is the exact inverse, so four levels with
    N^(3) = 1 equal three levels, and three levels with N^(2) = 1 equal two levels."""
    p4 = I.box_problem(4, 4, 2, (4, 4, 2), groups=((2, 2, 1), (2, 2, 2)), levels=4)
    p3 = I.box_problem(4, 4, 2, (4, 4, 2), groups=((2, 2, 1),), levels=3)
    S = fem.assemble(p4)
    P4 = gdsw.GDSW(S, p4)
    P3 = gdsw.GDSW(S, p3)
    assert P4.levels[2].N == 1
    q3 = I.box_problem(4, 4, 2, (4, 4, 2), groups=((4, 4, 2),), levels=3)
    q2 = I.box_problem(4, 4, 2, (4, 4, 2), levels=2)
    Q3 = gdsw.GDSW(S, q3)
    Q2 = gdsw.GDSW(S, q2)
    rng = np.random.default_rng(5)
    for _ in range(3):
        r = rng.standard_normal(S["A"].shape[0])
        a, b = P4.apply(r), P3.apply(r)
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
        a, b = Q3.apply(r), Q2.apply(r)
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


# --------------------------------------------------------------------------- P8
def test_plain_preconditioner_symmetric():
    """Section 2.1/2.2: with the paper's plain additive sum every term R^T A_i^{-1} R and
    Phi (.) Phi^T of a symmetric operator is symmetric, so x^T B y = y^T B x."""
    p = I.box_problem(4, 4, 4, (2, 2, 2), groups=((2, 1, 1),), levels=3, form="symmetric",
                      uk_seed=2, lam=1.0, n=0.5, nu_inf=1e-3)
    S = fem.assemble(p)
    P = gdsw.GDSW(S, p, weighting="plain")
    rng = np.random.default_rng(2)
    for _ in range(3):
        x, y = rng.standard_normal((2, S["A"].shape[0]))
        a, b = x @ P.apply(y), y @ P.apply(x)
        assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))


# --------------------------------------------------------------------------- P10
def test_fgmres_least_squares_optimal():
    """FGMRES (Section 3): after k steps x_k minimises ||b - A (x0 + Z_k y)|| over y; the
    oracle's x equals the dense least-squares minimiser and its residual."""
    p = I.box_problem(3, 3, 3, (3, 3, 1), levels=2)
    S = fem.assemble(p)
    A = S["A"]
    P = gdsw.GDSW(S, p)
    b = I.random_rhs(A.shape[0], 4)
    for k in (1, 4, 9):
        x, info = fgmres.fgmres(lambda v: A @ v, b, P.apply, tol=0.0, max_it=k, restart=k,
                                keep_basis=True)
        Z = info["Z"]
        AZ = np.column_stack([A @ z for z in Z])
        y, *_ = np.linalg.lstsq(AZ, b, rcond=None)
        xs = Z.T @ y
        assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
        assert abs(info["relres"] - np.linalg.norm(b - A @ xs) / np.linalg.norm(b)) < 1e-12


def test_local_matrices_invertible():
    """Section 2.1: every local saddle-point matrix A_i is invertible (homogeneous Dirichlet
    data on the artificial boundary); checked by the smallest singular value on a tiny
    mesh, on every level."""
    p = I.box_problem(4, 4, 2, (4, 4, 2), groups=((2, 2, 1), (2, 1, 1)), levels=4,
                      form="symmetric", uk_seed=1, lam=1.0, n=0.5, nu_inf=1e-3)
    S = fem.assemble(p)
    P = gdsw.GDSW(S, p)
    for l, lev in enumerate(P.levels):
        A = P.A0[l].toarray() if hasattr(P.A0[l], "toarray") else P.A0[l]
        for d in lev.dofs:
            s = np.linalg.svd(A[np.ix_(d, d)], compute_uv=False)
            assert s[-1] > 1e-10 * s[0]
    s = np.linalg.svd(P.A0[-1], compute_uv=False)
    assert s[-1] > 1e-10 * s[0]


def test_picard_pins():
    """Section 3 Picard iteration in the oracle: with n = 1 (Newtonian Carreau limit) nu does
    not depend on u, so every iterate is the same Stokes solution; for a shear-thinning fluid
    the increments shrink (a contraction on this mildly nonlinear case) and the last iterate
    satisfies the nonlinear system A(nu(u)) x = b(nu(u)) to the size of the last increment."""
    import numpy as np
    from oracle import fem
    from paper_2606_01433_gb300 import inputs as I
    p1 = I.box_problem(3, 3, 3, (1, 1, 1), form="symmetric", uk_seed=4, lam=1.0, n=1.0, nu_inf=0.0)
    xs = fem.picard(p1, 2)
    assert np.linalg.norm(xs[1] - xs[0]) <= 1e-12 * np.linalg.norm(xs[0])
    p = I.box_problem(3, 3, 3, (1, 1, 1), form="symmetric", uk_seed=4, lam=1.0, n=0.6, nu_inf=1e-2)
    xs = fem.picard(p, 6)
    inc = [np.linalg.norm(xs[k + 1] - xs[k]) / np.linalg.norm(xs[k + 1]) for k in range(5)]
    assert all(inc[k + 1] < inc[k] for k in range(4)), inc
    S0 = fem.assemble(p)
    u, _ = fem.full_solution(S0, xs[-1])
    import copy
    q = copy.copy(p)
    q.uk = u
    S = fem.assemble(q)
    res = np.linalg.norm(S["A"] @ xs[-1] - fem.lifted_rhs(S)) / np.linalg.norm(fem.lifted_rhs(S))
    assert res <= 10 * inc[-1], (res, inc)


def test_rotation_modes_pin():
    """Rotations in the coarse null space (the variant Section 2.1 leaves out): with the three
    rigid rotations per entity about its centroid, a global rigid rotation of the pure-Neumann
    symmetric-form problem lies exactly in the range of Phi (it is in the kernel of A, so its
    discrete extension reproduces it); without them it does not.  The default coarse space is
    unchanged by the option."""
    import numpy as np
    from oracle import fem, gdsw as og
    from paper_2606_01433_gb300 import inputs as I
    p = I.box_problem(4, 4, 4, (2, 2, 2), levels=2, form="symmetric", bc="neumann")
    S = fem.assemble(p)
    m = S["mesh"]
    nid = m.vnodes
    xyz = np.stack([nid % m.nxn, (nid // m.nxn) % m.nyn, nid // (m.nxn * m.nyn)], axis=1) * 0.5 * p.h
    r = np.zeros(S["A"].shape[0])
    d = xyz - np.array([0.37, 0.52, 0.41])
    r[:m.nu] = np.cross(np.array([0.3, -0.5, 0.8])[None, :], d).ravel()   # rigid rotation, p = 0
    assert np.linalg.norm(S["A"] @ r) <= 1e-10 * np.linalg.norm(r)          # in the kernel of A
    rot, _ = og.build_level1(S, p, rotations=True)
    plain, _ = og.build_level1(S, p)
    # the default space: per entity three translations if it holds a free velocity node and
    # one pressure constant if it holds a Q1 node, all as 0/1 indicators
    expect = sum(3 * int((m.vindex[nodes] >= 0).any()) + int((m.pindex[nodes] >= 0).any())
                 for _, nodes in plain.entities)
    assert plain.n0 == expect and np.all(plain.PhiGamma.data == 1.0)
    assert rot.n0 > plain.n0
    for lev, ok in ((rot, True), (plain, False)):
        Phi = lev.Phi.toarray()
        c = np.linalg.lstsq(Phi, r, rcond=None)[0]
        res = np.linalg.norm(Phi @ c - r) / np.linalg.norm(r)
        assert (res <= 1e-10) if ok else (res >= 1e-3), (ok, res)


# --------------------------------------------------------------------------- overlap depth
def _box_overlap_dofs(p, parts):
    """Free dofs of every overlapping subdomain of a box partition of an uncarved box,
    counted axis by axis: the part's element range [lo, hi) grows by one element layer to
    [max(lo-1, 0), min(hi+1, m)); a Q2 node index i along that axis is kept when it lies
    strictly inside the grown range (2 lo' < i < 2 hi'), or on the physical boundary
    (i = 0 or i = 2m) that the grown range reaches.  Dof numbering as documented for the
    inputs: free velocity nodes (tags other than wall/inflow) in node order, three
    components each, then the Q1 (all-even index) nodes in node order."""
    dims = (p.nx, p.ny, p.nz)
    nxn, nyn = 2 * p.nx + 1, 2 * p.ny + 1
    free_v = np.nonzero((p.tags != I.TAG_WALL) & (p.tags != I.TAG_INFLOW))[0]
    vnum = -np.ones(p.n_nodes, dtype=np.int64)
    vnum[free_v] = np.arange(free_v.size)
    nid = np.arange(p.n_nodes)
    ijk = np.stack([nid % nxn, (nid // nxn) % nyn, nid // (nxn * nyn)], axis=1)
    q1 = np.nonzero((ijk % 2 == 0).all(axis=1))[0]
    pnum = -np.ones(p.n_nodes, dtype=np.int64)
    pnum[q1] = np.arange(q1.size)
    nu = 3 * free_v.size
    out = []
    for bz in range(parts[2]):
        for by in range(parts[1]):
            for bx in range(parts[0]):
                keep = []
                for b, q, m in zip((bx, by, bz), parts, dims):
                    lo, hi = b * m // q, (b + 1) * m // q
                    lo2, hi2 = max(lo - 1, 0), min(hi + 1, m)
                    idx = [i for i in range(2 * m + 1)
                           if 2 * lo2 < i < 2 * hi2 or (i == 0 and lo2 == 0) or (i == 2 * m and hi2 == m)]
                    keep.append(np.array(idx))
                k3, j3, i3 = np.meshgrid(keep[2], keep[1], keep[0], indexing="ij")
                nodes = np.sort((i3 + nxn * (j3 + nyn * k3)).ravel())
                v = vnum[nodes]
                v = v[v >= 0]
                pp = pnum[nodes]
                out.append(np.sort(np.concatenate([(3 * v[:, None] + np.arange(3)).ravel(), nu + pp[pp >= 0]])))
    return out


@pytest.mark.parametrize("m,parts", [(8, (4, 4, 4)), (6, (2, 3, 1)), (4, (2, 2, 2))])
def test_overlap_one_element_layer(m, parts):
    """Section 3 'one layer of overlap' with Section 2.1's homogeneous Dirichlet data on the
    artificial boundary: for box partitions of an uncarved cube (corner, edge, face and
    interior parts) the oracle's overlapping dof sets equal the box-geometric count of one
    element layer with the rim of the grown box dropped -- and differ from zero or two
    layers."""
    p = I.unit_cube(m, parts=parts)
    S = fem.assemble(p)
    got = gdsw.overlapping_dofs(S, p)
    lev, _ = gdsw.build_level1(S, p)
    expect = _box_overlap_dofs(p, parts)
    assert len(got) == len(expect) == parts[0] * parts[1] * parts[2]
    for a, b, c in zip(got, expect, lev.dofs):
        assert np.array_equal(a, b) and np.array_equal(c, b)
    for k in (0, 2):
        other = gdsw.overlapping_dofs(S, p, overlap=k)
        assert any(not np.array_equal(a, b) for a, b in zip(other, expect))


def test_coarse_overlap_chain_by_hand():
    """Section 2.2 coarse levels with one layer of overlap, written out by hand on a chain:
    eight one-element parts along x (faces F1..F7 between parts k-1 and k, each one entity
    with ux, uy, uz, p), grouped in pairs {0,1}, {2,3}, {4,5}, {6,7}.  Face F_k lies in the
    closure of group J when one of its parts belongs to J; coarse nodes couple when their
    sharing sets meet (F_k with F_k-1 and F_k+1), so with one graph layer
    Omega_0' = F1..F3, Omega_1' = F1..F5, Omega_2' = F3..F7, Omega_3' = F5..F7."""
    p = I.box_problem(8, 1, 1, (8, 1, 1), groups=((2, 1, 1),), levels=3)
    S = fem.assemble(p)
    P = gdsw.GDSW(S, p)
    lev1, lev2 = P.levels
    assert [tuple(s) for s, nodes in lev1.entities] == [(k - 1, k) for k in range(1, 8)]
    assert lev1.n0 == 28
    F = lambda a, b: np.arange(4 * (a - 1), 4 * b)        # dofs of faces F_a .. F_b
    expect = [F(1, 3), F(1, 5), F(3, 7), F(5, 7)]
    assert len(lev2.dofs) == 4
    for got, exp in zip(lev2.dofs, expect):
        assert np.array_equal(got, exp), (got, exp)
    # level-2 interface: the faces shared by two groups, F2, F4, F6
    assert [tuple(s) for s, nodes in lev2.entities] == [(0, 1), (1, 2), (2, 3)]
    assert [list(nodes) for s, nodes in lev2.entities] == [[1], [3], [5]]


def test_fgmres_restart_cycles():
    """Restarted FGMRES (Section 3): with restart 5 on a case that needs more than 15
    iterations, (a) the residual estimates never increase, (b) the run reaches the dense
    solution, (c) a restart continues from the cycle's iterate exactly as a fresh run started
    there, and (d) the second cycle's update is the least-squares minimiser of the residual
    of that iterate over span(A Z) of the cycle."""
    p = I.box_problem(4, 4, 4, (2, 2, 2), levels=2, form="symmetric", uk_seed=3, lam=1.0, n=0.5, nu_inf=1e-3)
    S = fem.assemble(p)
    A = S["A"]
    P = gdsw.GDSW(S, p)
    b = I.random_rhs(A.shape[0], 8)
    mv = lambda v: A @ v
    x, info = fgmres.fgmres(mv, b, P.apply, tol=1e-12, restart=5, max_it=400)
    assert info["converged"] and info["iterations"] > 15
    h = np.array(info["history"])
    assert np.all(h[1:] <= h[:-1] * (1 + 1e-12))
    xd = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    x5, _ = fgmres.fgmres(mv, b, P.apply, tol=0.0, restart=5, max_it=5)
    x10, i10 = fgmres.fgmres(mv, b, P.apply, tol=0.0, restart=5, max_it=10, keep_basis=True)
    y10, _ = fgmres.fgmres(mv, b, P.apply, tol=0.0, restart=5, max_it=5, x0=x5)
    assert np.linalg.norm(x10 - y10) <= 1e-13 * np.linalg.norm(x10)
    AZ = np.column_stack([A @ z for z in i10["Z"]])
    y, *_ = np.linalg.lstsq(AZ, b - A @ x5, rcond=None)
    assert np.linalg.norm(x10 - (x5 + i10["Z"].T @ y)) <= 1e-10 * np.linalg.norm(x10)


# --------------------------------------------------------------------------- mixed emulation
def test_rounding_functions():
    """The two roundings of the mixed-precision emulation against hand-worked ties and the
    conversions of two libraries: binary32 (Python's struct packing, a C float cast) and
    bfloat16 (PyTorch's float32 -> bfloat16 conversion, round to nearest even)."""
    import struct
    one = 1.0
    # binary32: 24-bit significand, ties to even
    assert gdsw.round_fp32(one + 2.0 ** -24) == one
    assert gdsw.round_fp32(one + 3 * 2.0 ** -24) == one + 2.0 ** -22
    x = np.random.default_rng(0).standard_normal(2000) * np.exp(np.random.default_rng(1).uniform(-30, 30, 2000))
    ref = np.array([struct.unpack("f", struct.pack("f", v))[0] for v in x])
    assert np.array_equal(gdsw.round_fp32(x), ref)
    # bfloat16: 8-bit significand, ties to even
    assert gdsw.round_bf16(one + 2.0 ** -8) == one
    assert gdsw.round_bf16(one + 3 * 2.0 ** -8) == one + 2.0 ** -6
    assert gdsw.round_bf16(one + 2.0 ** -8 + 2.0 ** -20) == one + 2.0 ** -7
    assert gdsw.round_bf16(-(one + 2.0 ** -8)) == -one and gdsw.round_bf16(0.0) == 0.0
    assert gdsw.round_bf16(255.5) == 256.0 and gdsw.round_bf16(3.0) == 3.0
    torch = pytest.importorskip("torch")
    x32 = gdsw.round_fp32(x)
    ref = torch.from_numpy(x32.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(gdsw.round_bf16(x32), ref)


def test_mixed_emulation_effect():
    """The emulation perturbs the preconditioner by the unit roundoff of its precision
    (FP32 ~ 1e-7, BF16 ~ 4e-3, relative) and the FP64 flexible GMRES still reaches the
    FP64 solution, with iteration counts close to the FP64 preconditioner's."""
    p = I.box_problem(4, 4, 4, (2, 2, 2), groups=((2, 2, 1),), levels=3, form="symmetric", uk_seed=3,
                      lam=1.0, n=0.5, nu_inf=1e-3)
    S = fem.assemble(p)
    A = S["A"]
    P64 = gdsw.GDSW(S, p)
    P32 = gdsw.GDSW(S, p, local_precision=("fp32", "fp32"))
    P16 = gdsw.GDSW(S, p, local_precision=("bf16", "fp32"))
    r = np.random.default_rng(3).standard_normal(A.shape[0])
    z64 = P64.apply(r)
    e32 = np.linalg.norm(P32.apply(r) - z64) / np.linalg.norm(z64)
    e16 = np.linalg.norm(P16.apply(r) - z64) / np.linalg.norm(z64)
    assert 1e-10 < e32 < 1e-5 and 1e-5 < e16 < 1e-1 and e32 < e16, (e32, e16)
    b = fem.lifted_rhs(S)
    xd = spla.spsolve(A.tocsc(), b)
    its = {}
    for name, P in (("fp64", P64), ("fp32", P32), ("bf16", P16)):
        x, info = fgmres.fgmres(lambda v: A @ v, b, P.apply, tol=1e-11)
        assert info["converged"]
        assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
        its[name] = info["iterations"]
    assert abs(its["fp32"] - its["fp64"]) <= 1 and its["bf16"] >= its["fp64"], its
