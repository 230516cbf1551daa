"""Geometric multigrid whose coarsest problem the multilevel GDSW method solves, FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passage followed (Section 3): besides preconditioning FGMRES directly, the multilevel
Schwarz method serves as the coarse-grid solver of a geometric multigrid method, where
FGMRES preconditioned by it solves the coarsest problem to a relative residual of 1e-1.
The paper names neither the smoother nor the transfer operators, so this module uses the
textbook components on nested voxel grids (readings, also listed in the design notes):
  * grids: the same domain with m, m/2, ... elements per edge; each grid's operator is
    assembled on that grid (rediscretisation) with the frozen Picard velocity sampled at its
    nodes;
  * prolongation P: nodal interpolation of the coarse Q2 velocity and Q1 pressure at the
    fine nodes (the coarse spaces are contained in the fine ones); coarse Dirichlet nodes
    carry a zero correction; restriction R = P^T;
  * smoother: multiplicative element-Vanka over eight colours -- for every fluid element
    the principal submatrix A_e of the assembled operator on the free dofs of its 27 Q2 and
    8 Q1 nodes is solved exactly; elements are coloured by the parity of their voxel indices
    (two elements of one colour share no node), and a smoothing step sweeps the colours in
    order, each colour's corrections computed from the current residual:
    x <- x + omega sum_{e of colour c} R_e^T A_e^{-1} R_e (b - A x), c = 0..7.  (An
    additive, partition-of-unity-weighted Vanka diverged or converged slowly on these Q2/Q1
    problems: the continuous pressure couples every patch to its neighbours.)
  * cycle: V-cycle with nu1 pre- and nu2 post-smoothing steps (optionally the post-smoothing
    sweeps the colours in reverse order: a symmetric cycle), zero initial guess on every
    coarser grid; on the coarsest grid GDSW-preconditioned FGMRES from zero to the relative
    residual coarse_tol (1e-1 in the paper);
  * outer iteration: x <- x + V(b - A x) with the residual in FP64, until
    ||b - A x|| <= tol ||b||.

Parity status: pinned (Galerkin identity P^T A_f P = A_c for the Newtonian operator on
nested grids, polynomial reproduction of P, the vanishing restricted residual after an
exact coarse-grid correction, the colour classes sharing no dof, the Vanka sweep converging
on its own, convergence to the direct solution).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from oracle import fem, fgmres, gdsw


def _lagrange2(t):
    """Quadratic Lagrange weights of the nodes 0, 1, 2 at t in [0, 2]."""
    return np.array([(t - 1.0) * (t - 2.0) / 2.0, t * (2.0 - t), t * (t - 1.0) / 2.0])


def _axis_weights_q2(i, mc):
    """Coarse Q2 node indices and weights along one axis for the fine Q2 node index i:
    the fine node sits at coarse node coordinate t = i / 2, inside coarse element
    E = min(floor(t / 2), mc - 1)."""
    t = i / 2.0
    E = min(int(t // 2), mc - 1)
    w = _lagrange2(t - 2 * E)
    return [(2 * E + a, w[a]) for a in range(3) if w[a] != 0.0]


def _axis_weights_q1(p, mc):
    """Coarse Q1 node indices (in Q1 numbering) and weights for the fine Q1 index p: the
    fine vertex sits at coarse vertex coordinate p / 2."""
    P0 = min(p // 2, mc - 1)
    f = p / 2.0 - P0
    return [(P0 + a, w) for a, w in ((0, 1.0 - f), (1, f)) if w != 0.0]


def prolongation(Sf, Sc):
    """P: coarse free dofs -> fine free dofs (nodal interpolation, see module header)."""
    mf, mc = Sf["mesh"], Sc["mesh"]
    pf, pc = mf.p, mc.p
    nfx, ncx = pf.nx, pc.nx
    assert (pf.nx, pf.ny, pf.nz) == (2 * pc.nx, 2 * pc.ny, 2 * pc.nz), "grids must be nested"
    rows, cols, vals = [], [], []
    # velocity
    for vf, node in enumerate(mf.vnodes):
        i, j, k = node % mf.nxn, (node // mf.nxn) % mf.nyn, node // (mf.nxn * mf.nyn)
        for (I, wi) in _axis_weights_q2(i, pc.nx):
            for (J, wj) in _axis_weights_q2(j, pc.ny):
                for (K, wk) in _axis_weights_q2(k, pc.nz):
                    vc = mc.vindex[I + mc.nxn * (J + mc.nyn * K)]
                    if vc < 0:
                        continue          # coarse Dirichlet node: zero correction
                    w = wi * wj * wk
                    for c in range(3):
                        rows.append(3 * vf + c); cols.append(3 * vc + c); vals.append(w)
    # pressure (Q1 vertices: Q2 indices that are even on every axis)
    for pfi, node in enumerate(mf.pnodes):
        i, j, k = node % mf.nxn, (node // mf.nxn) % mf.nyn, node // (mf.nxn * mf.nyn)
        for (I, wi) in _axis_weights_q1(i // 2, pc.nx):
            for (J, wj) in _axis_weights_q1(j // 2, pc.ny):
                for (K, wk) in _axis_weights_q1(k // 2, pc.nz):
                    cnode = 2 * I + mc.nxn * (2 * J + mc.nyn * 2 * K)
                    pci = mc.pindex[cnode]
                    rows.append(mf.nu + pfi); cols.append(mc.nu + pci); vals.append(wi * wj * wk)
    return sp.csr_matrix((vals, (rows, cols)), shape=(mf.n, mc.n))


class Vanka:
    """Multiplicative element-Vanka smoother over eight colours on the assembled operator.

    Elements are coloured by the parity of their three voxel indices; two elements of one
    colour share no node, so the patch solves of a colour are independent, and a smoothing
    step is a Gauss-Seidel sweep over the colours:
    for c = 0..7: x <- x + omega sum_{e of colour c} R_e^T A_e^{-1} R_e (b - A x)."""

    def __init__(self, S, omega=1.0):
        mesh = S["mesh"]
        A = S["A"]
        p = mesh.p
        self.A = A
        self.omega = omega
        vdof = np.where(mesh.vindex >= 0, 3 * mesh.vindex, -1)
        self.dofs = []
        for e in range(mesh.elems.size):
            v = vdof[mesh.enodes[e]]
            v = v[v >= 0]
            pp = mesh.nu + mesh.pindex[mesh.epnodes[e]]
            self.dofs.append(np.sort(np.concatenate([(v[:, None] + np.arange(3)).ravel(), pp])))
        el = mesh.elems
        self.colour = (el % p.nx) % 2 + 2 * (((el // p.nx) % p.ny) % 2) + 4 * ((el // (p.nx * p.ny)) % 2)
        self.inv = [np.linalg.inv(A[d][:, d].toarray()) for d in self.dofs]

    def smooth(self, b, x, steps, reverse=False):
        for _ in range(steps):
            for c in (range(7, -1, -1) if reverse else range(8)):
                r = b - self.A @ x
                dx = np.zeros_like(x)
                for e in np.nonzero(self.colour == c)[0]:
                    d = self.dofs[e]
                    dx[d] = self.inv[e] @ r[d]
                x = x + self.omega * dx
        return x


class Multigrid:
    """V-cycle on nested grids (finest first) with the multilevel GDSW-FGMRES coarse solver."""

    def __init__(self, probs, omega=1.0, pre=2, post=2, coarse_tol=1e-1, coarse_restart=100, pool=None,
                 symmetric=False):
        self.S = [fem.assemble(p, pool=pool) for p in probs]
        self.A = [S["A"] for S in self.S]
        self.P = [prolongation(self.S[l], self.S[l + 1]) for l in range(len(probs) - 1)]
        self.R = [P.T.tocsr() for P in self.P]
        self.smoothers = [Vanka(self.S[l], omega) for l in range(len(probs) - 1)]
        self.pre, self.post, self.symmetric = pre, post, symmetric
        self.coarse = gdsw.GDSW(self.S[-1], probs[-1], pool=pool)
        self.coarse_tol = coarse_tol
        self.coarse_restart = coarse_restart
        self.coarse_its = []

    def coarse_solve(self, b):
        """Section 3: FGMRES preconditioned by the multilevel GDSW method, from zero, to a
        relative residual of coarse_tol."""
        A = self.A[-1]
        x, info = fgmres.fgmres(lambda v: A @ v, b, self.coarse.apply, tol=self.coarse_tol,
                                restart=self.coarse_restart)
        self.coarse_its.append(info["iterations"])
        return x

    def vcycle(self, b, level=0):
        """z ~ A_level^{-1} b from a zero initial guess."""
        if level == len(self.A) - 1:
            return self.coarse_solve(b)
        A, sm = self.A[level], self.smoothers[level]
        z = sm.smooth(b, np.zeros_like(b), self.pre)
        rc = self.R[level] @ (b - A @ z)
        z = z + self.P[level] @ self.vcycle(rc, level + 1)
        return sm.smooth(b, z, self.post, reverse=self.symmetric)

    def solve(self, b, tol=1e-8, max_cycles=200):
        """Outer iteration x <- x + V(b - A x) with the FP64 residual; returns x and the
        history of relative residuals (one entry per cycle, the initial one first)."""
        A = self.A[0]
        x = np.zeros_like(b)
        bn = np.linalg.norm(b)
        hist = [1.0]
        r = b.copy()
        while hist[-1] > tol and len(hist) <= max_cycles:
            x = x + self.vcycle(r)
            r = b - A @ x
            hist.append(np.linalg.norm(r) / bn)
        return x, hist
