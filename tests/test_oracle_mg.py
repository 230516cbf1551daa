"""Pins of the oracle's geometric multigrid (Section 3: the Schwarz method as the coarse-grid
solver of a geometric multigrid method) against facts that nested finite-element spaces and
the textbook multigrid components fix: the Galerkin identity of rediscretised nested
operators, exact interpolation of the coarse spaces, the vanishing restricted residual after
an exact coarse-grid correction, the colour classes sharing no dof, the smoother converging
on its own, and convergence to the direct solution."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from paper_2606_01433_gb300 import inputs as I
from oracle import fem, fgmres, mg


def _pair(m, carreau=False, form=None):
    ps = I.mg_hierarchy(m, 2, parts=(1, 1, 1), groups=(), levels=2, carreau=carreau)
    if form is not None:
        for p in ps:
            p.form = form
    return ps, [fem.assemble(p) for p in ps]


@pytest.mark.parametrize("form", ["gradient", "symmetric"])
def test_galerkin_identity_nested_grids(form):
    """Nested Q2/Q1 spaces: every coarse basis function is a fine-grid function, and 3x3x3
    Gauss integrates both grids' Newtonian bilinear forms exactly, so P^T A_f P equals the
    operator assembled on the coarse grid (velocity, divergence and their couplings)."""
    ps, S = _pair(8, form=form)
    P = mg.prolongation(S[0], S[1])
    G = (P.T @ S[0]["A"] @ P).toarray()
    Ac = S[1]["A"].toarray()
    assert np.abs(G - Ac).max() <= 1e-12 * np.abs(Ac).max()


def test_prolongation_reproduces_coarse_space():
    """P interpolates exactly: a velocity in Q2 on the coarse grid (degree <= 2 per axis,
    zero on the walls and the inflow) and a trilinear pressure are reproduced at the fine
    nodes."""
    ps, S = _pair(8)
    P = mg.prolongation(S[0], S[1])

    def dofs(Sx):
        m = Sx["mesh"]
        x = m.p.node_coords()
        u = np.zeros((m.vnodes.size, 3))
        xv = x[m.vnodes]
        u[:, 0] = xv[:, 0] * xv[:, 1] * (1 - xv[:, 1]) * xv[:, 2] * (1 - xv[:, 2])
        u[:, 1] = xv[:, 1] * (1 - xv[:, 1]) * xv[:, 2] * (1 - xv[:, 2]) * xv[:, 0] * (1.5 - xv[:, 0])
        u[:, 2] = -2.0 * xv[:, 0] * xv[:, 1] * (1 - xv[:, 1]) * xv[:, 2] * (1 - xv[:, 2])
        xp = x[m.pnodes]
        pr = 1.0 + xp[:, 0] - 2.0 * xp[:, 1] + xp[:, 0] * xp[:, 2] - 0.5 * xp[:, 0] * xp[:, 1] * xp[:, 2]
        return np.concatenate([u.ravel(), pr])
    uf, uc = dofs(S[0]), dofs(S[1])
    assert np.abs(P @ uc - uf).max() <= 1e-13 * np.abs(uf).max()


def test_exact_coarse_correction_annihilates_restricted_residual():
    """With the Galerkin identity, one exact coarse-grid correction x = P A_c^{-1} P^T b leaves
    a residual whose restriction vanishes: P^T (b - A_f x) = 0."""
    ps, S = _pair(8)
    A = S[0]["A"]
    P = mg.prolongation(S[0], S[1])
    b = I.random_rhs(A.shape[0], 2)
    x = P @ spla.spsolve(S[1]["A"].tocsc(), P.T @ b)
    assert np.linalg.norm(P.T @ (b - A @ x)) <= 1e-11 * np.linalg.norm(P.T @ b)


def test_vanka_colours_disjoint_and_smoothing_contracts():
    """The patches of one colour (parity of the voxel indices) share no dof, every free dof
    lies in some patch, and the multiplicative sweep is a convergent iteration on its own
    (block Gauss-Seidel over the colour classes with exact patch solves): 40 sweeps shrink
    the error to the direct solution by two orders of magnitude on a Newtonian 4^3 channel."""
    ps, S = _pair(4)
    A = S[0]["A"]
    V = mg.Vanka(S[0])
    covered = np.zeros(A.shape[0], dtype=int)
    for c in range(8):
        seen = np.zeros(A.shape[0], dtype=int)
        for e in np.nonzero(V.colour == c)[0]:
            seen[V.dofs[e]] += 1
        assert seen.max() <= 1
        covered += seen
    assert covered.min() >= 1
    b = I.random_rhs(A.shape[0], 3)
    xd = spla.spsolve(A.tocsc(), b)
    x = V.smooth(b, np.zeros_like(b), 40)
    assert np.linalg.norm(x - xd) <= 1e-2 * np.linalg.norm(xd)
    assert np.linalg.norm(V.smooth(b, xd, 1) - xd) <= 1e-12 * np.linalg.norm(xd)


@pytest.mark.parametrize("carreau", [False, True])
def test_mg_preconditioned_fgmres_reaches_direct_solution(carreau):
    """FGMRES preconditioned by V(2,2)-cycles with the GDSW-FGMRES coarse solve to 1e-1
    converges to the direct solution (8^3 fine grid, 4^3 coarse grid with 2x2x2 parts)."""
    ps = I.mg_hierarchy(8, 2, parts=(2, 2, 2), groups=(), levels=2, carreau=carreau)
    M = mg.Multigrid(ps, pre=2, post=2)
    A = M.A[0]
    b = I.random_rhs(A.shape[0], 4)
    x, info = fgmres.fgmres(lambda v: A @ v, b, M.vcycle, tol=1e-10, max_it=60)
    xd = spla.spsolve(A.tocsc(), b)
    assert info["converged"] and info["iterations"] <= 40, info["iterations"]
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)
    assert all(1 <= k <= 20 for k in M.coarse_its)
