"""Pins of the oracle's Newton linearisation (Section 3: the nonlinear Carreau problem is solved
by alternating Picard and Newton steps) against what the mathematics fixes: the Jacobian equals
central finite differences of the nonlinear residual, it is symmetric (the Carreau problem
minimises a convex energy), it reduces to the Picard operator for a Newtonian fluid (n = 1),
and Newton steps converge quadratically where Picard steps converge linearly."""
import copy

import numpy as np
import pytest

from paper_2606_01433_gb300 import inputs as I
from oracle import fem


def _prob(n=0.5, uk_seed=3):
    return I.box_problem(3, 3, 3, (1, 1, 1), form="symmetric", uk_seed=uk_seed, lam=1.0, n=n, nu_inf=1e-2)


def _residual(p, x):
    """F(x) = A(nu(u(x))) x - b(nu(u(x))) with u(x) the velocity of x plus the Dirichlet data."""
    q = copy.copy(p)
    S0 = fem.assemble(q)
    q.uk, _ = fem.full_solution(S0, x)
    S = fem.assemble(q)
    return S["A"] @ x - fem.lifted_rhs(S)


def test_jacobian_equals_finite_differences_and_is_symmetric():
    p = _prob()
    xs, _ = fem.picard_newton(p, "P")
    x = xs[0]
    q = copy.copy(p)
    S = fem.assemble(q)
    q.uk, _ = fem.full_solution(S, x)
    J = fem.assemble(q, newton=True)["A"]
    A = fem.assemble(q)["A"]
    assert abs(J - J.T).max() <= 1e-13 * abs(J).max()
    assert abs(J - A).max() > 1e-3 * abs(A).max()          # the Newton term is really there
    rng = np.random.default_rng(0)
    for _ in range(3):
        w = rng.standard_normal(x.size)
        w[S["mesh"].nu:] = 0.0 if _ == 0 else w[S["mesh"].nu:]
        eps = 1e-6 * np.linalg.norm(x) / np.linalg.norm(w)
        fd = (_residual(p, x + eps * w) - _residual(p, x - eps * w)) / (2 * eps)
        assert np.linalg.norm(J @ w - fd) <= 1e-6 * np.linalg.norm(fd)


def test_newtonian_limit_has_no_newton_term():
    p = _prob(n=1.0)
    A = fem.assemble(p)["A"]
    J = fem.assemble(p, newton=True)["A"]
    assert abs(J - A).max() <= 1e-15 * abs(A).max()


def test_newton_converges_quadratically():
    """After two Picard steps, Newton steps square the residual (r_{k+1} <= 10 r_k^2) and pass
    1e-10 within four steps; Picard steps alone shrink it only by a roughly constant factor."""
    p = _prob(n=0.4)
    _, rn = fem.picard_newton(p, "PPNNNNP")
    newton = rn[1:]                      # residuals before each Newton step, then after the last
    _, rp = fem.picard_newton(p, "PPPPPPP")
    assert min(newton) <= 1e-10, newton
    k = next(i for i, r in enumerate(newton) if r <= 1e-10)
    assert k <= 4
    for a, b in zip(newton[:k], newton[1:k + 1]):
        assert b <= 10.0 * a * a + 1e-14, newton
    assert rp[-1] > 1e-7, rp                      # Picard is still far from that
