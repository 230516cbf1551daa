"""Q2/Q1 Taylor-Hood discretisation of the stationary (Carreau) Stokes problem, FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages followed:
  * Section 2, weak form: mu * int grad u : grad v  -  int div v p  = int f v,
    -int div u q = 0, u = g on the Dirichlet part, du/dn - p n = 0 on the Neumann part
    ("gradient" form).
  * Section 2, saddle-point equation: A_cal = [[A, B^T], [B, 0]], F_cal = [F; 0].
  * Section 3, constitutive law: sigma = -p I + 2 nu(u) D(u), D(u) = (grad u + grad u^T)/2,
    Carreau viscosity nu = nu0 (1 + (lambda gamma_dot)^2)^((n-1)/2),
    gamma_dot = sqrt(2 D:D); with the "symmetric" bilinear form 2 nu D(u):D(v) and
    traction-free outflow sigma n = 0.  We use nu = nu_inf + (nu0 - nu_inf)(...) which is
    the paper's law for nu_inf = 0.
The paper uses Q2 / P1-discontinuous elements; the workloads here use Q2 / Q1
(Taylor-Hood) with 3x3x3 Gauss quadrature on axis-aligned cubes of edge h; prob.pressure =
"p1disc" selects the paper's pair (pressure 1, xi, eta, zeta per element in reference
coordinates; four dofs per fluid element after the velocity dofs, element order).

Dof order (identical to the library's): free velocity nodes in increasing node index,
three interleaved components each, then the Q1 (even-index) nodes of the fluid region in
increasing node index.

Parity status: pinned (Poiseuille closed form, Carreau closed form; see tests).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

GAUSS_X = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
GAUSS_W = np.array([5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0])


def lagrange_q2_1d(x):
    """Values and derivatives of the quadratic Lagrange basis on the nodes -1, 0, 1."""
    v = np.array([0.5 * x * (x - 1.0), 1.0 - x * x, 0.5 * x * (x + 1.0)])
    d = np.array([x - 0.5, -2.0 * x, x + 0.5])
    return v, d


def lagrange_q1_1d(x):
    return np.array([0.5 * (1.0 - x), 0.5 * (1.0 + x)])


def reference_tables():
    """Q2 values/gradients and Q1 values at the 27 Gauss points of [-1,1]^3.

    Local Q2 node a = a0 + 3 a1 + 9 a2 sits at offsets (a0, a1, a2) in {0,1,2}^3 (in units
    of h/2 from the element's low corner); local Q1 node P = p0 + 2 p1 + 4 p2 sits at
    offsets (2 p0, 2 p1, 2 p2).  Quadrature point q = q0 + 3 q1 + 9 q2.
    Returns phi (27q, 27a), dphi (27q, 27a, 3) in reference coordinates, psi (27q, 8),
    weights (27q,).
    """
    phi = np.zeros((27, 27))
    dphi = np.zeros((27, 27, 3))
    psi = np.zeros((27, 8))
    w = np.zeros(27)
    for q2 in range(3):
        for q1 in range(3):
            for q0 in range(3):
                q = q0 + 3 * q1 + 9 * q2
                xs = (GAUSS_X[q0], GAUSS_X[q1], GAUSS_X[q2])
                w[q] = GAUSS_W[q0] * GAUSS_W[q1] * GAUSS_W[q2]
                v = [lagrange_q2_1d(x) for x in xs]
                l1 = [lagrange_q1_1d(x) for x in xs]
                for a2 in range(3):
                    for a1 in range(3):
                        for a0 in range(3):
                            a = a0 + 3 * a1 + 9 * a2
                            phi[q, a] = v[0][0][a0] * v[1][0][a1] * v[2][0][a2]
                            dphi[q, a, 0] = v[0][1][a0] * v[1][0][a1] * v[2][0][a2]
                            dphi[q, a, 1] = v[0][0][a0] * v[1][1][a1] * v[2][0][a2]
                            dphi[q, a, 2] = v[0][0][a0] * v[1][0][a1] * v[2][1][a2]
                for p2 in range(2):
                    for p1 in range(2):
                        for p0 in range(2):
                            psi[q, p0 + 2 * p1 + 4 * p2] = l1[0][p0] * l1[1][p1] * l1[2][p2]
    return phi, dphi, psi, w


class Mesh:
    """Voxel mesh topology: fluid elements, their 27 Q2 nodes and 8 Q1 nodes."""

    def __init__(self, prob):
        self.p = prob
        nx, ny, nz = prob.nx, prob.ny, prob.nz
        self.nxn, self.nyn, self.nzn = 2 * nx + 1, 2 * ny + 1, 2 * nz + 1
        self.elems = np.nonzero(prob.mask)[0]                 # fluid element ids
        ex = self.elems % nx
        ey = (self.elems // nx) % ny
        ez = self.elems // (nx * ny)
        off = np.array([(a % 3, (a // 3) % 3, a // 9) for a in range(27)])
        i = 2 * ex[:, None] + off[None, :, 0]
        j = 2 * ey[:, None] + off[None, :, 1]
        k = 2 * ez[:, None] + off[None, :, 2]
        self.enodes = i + self.nxn * (j + self.nyn * k)       # (ne, 27) Q2 node ids
        q1 = [0 + 0, 2, 6, 8, 18, 20, 24, 26]                  # local Q2 index of Q1 node P
        self.q1_local = np.array(q1)
        self.epnodes = self.enodes[:, self.q1_local]           # (ne, 8)
        self.active = np.zeros(prob.n_nodes, dtype=bool)
        self.active[self.enodes.ravel()] = True
        dirichlet = (prob.tags == 1) | (prob.tags == 2)
        self.vnodes = np.nonzero(self.active & ~dirichlet)[0]  # free velocity nodes
        self.dnodes = np.nonzero(self.active & dirichlet)[0]   # Dirichlet velocity nodes
        self.pnodes = np.unique(self.epnodes.ravel())          # pressure (Q1) nodes
        self.vindex = -np.ones(prob.n_nodes, dtype=np.int64)
        self.vindex[self.vnodes] = np.arange(self.vnodes.size)
        self.dindex = -np.ones(prob.n_nodes, dtype=np.int64)
        self.dindex[self.dnodes] = np.arange(self.dnodes.size)
        self.pindex = -np.ones(prob.n_nodes, dtype=np.int64)
        self.pdisc = getattr(prob, "pressure", "q1") == "p1disc"
        if self.pdisc:      # no nodal pressure: four dofs per fluid element, element order
            self.pnodes = np.zeros(0, dtype=np.int64)
        else:
            self.pindex[self.pnodes] = np.arange(self.pnodes.size)
        self.nu = 3 * self.vnodes.size
        self.np_ = 4 * self.elems.size if self.pdisc else self.pnodes.size
        self.n = self.nu + self.np_


def carreau(gamma_dot, nu0, nu_inf, lam, n):
    """Carreau law (Section 3) with the infinite-shear offset nu_inf."""
    return nu_inf + (nu0 - nu_inf) * (1.0 + (lam * gamma_dot) ** 2) ** ((n - 1.0) / 2.0)


def quadrature_viscosity(mesh: Mesh, tabs):
    """nu at the 27 Gauss points of every fluid element (Section 3 Carreau law).

    grad u_k at a point = sum over the element's 27 Q2 nodes of u_k[node] (outer) grad phi,
    with grad = (2/h) * reference gradient; D = sym(grad u), gamma_dot = sqrt(2 D:D).
    """
    p = mesh.p
    ne = mesh.elems.size
    if p.uk is None or p.form == "gradient":
        return np.full((ne, 27), p.nu0)
    phi, dphi, psi, w = tabs
    u = p.uk[mesh.enodes]                                # (ne, 27, 3)
    grad = np.einsum("eac,qal->eqcl", u, dphi) * (2.0 / p.h)   # d u_c / d x_l
    D = 0.5 * (grad + np.swapaxes(grad, 2, 3))
    gd = np.sqrt(2.0 * np.einsum("eqcl,eqcl->eq", D, D))
    return carreau(gd, p.nu0, p.nu_inf, p.lam, p.n_carreau)


def carreau_dnu_over_gd(gamma_dot, nu0, nu_inf, lam, n):
    """nu'(gamma_dot) / gamma_dot of the Carreau law (finite at gamma_dot = 0):
    (nu0 - nu_inf) (n - 1) lambda^2 (1 + (lambda gamma_dot)^2)^((n - 3)/2)."""
    return (nu0 - nu_inf) * (n - 1.0) * lam ** 2 * (1.0 + (lam * gamma_dot) ** 2) ** ((n - 3.0) / 2.0)


def quadrature_strain(mesh: Mesh, tabs):
    """D(u_k) (ne, 27, 3, 3) and the Newton weight N = 4 nu'(gamma_dot) / gamma_dot (ne, 27)
    at the Gauss points, for the Newton linearisation of Section 3's alternating
    Picard-Newton iteration (see newton_matrices)."""
    p = mesh.p
    phi, dphi, psi, w = tabs
    u = p.uk[mesh.enodes]
    grad = np.einsum("eac,qal->eqcl", u, dphi) * (2.0 / p.h)
    D = 0.5 * (grad + np.swapaxes(grad, 2, 3))
    gd = np.sqrt(2.0 * np.einsum("eqcl,eqcl->eq", D, D))
    return D, 4.0 * carreau_dnu_over_gd(gd, p.nu0, p.nu_inf, p.lam, p.n_carreau)


def newton_matrices(h, D, N, tabs):
    """Element matrices (ne, 81, 81) of the Newton term of the Carreau operator.

    With a(u; v) = int 2 nu(gamma_dot(u)) D(u):D(v) and gamma_dot = sqrt(2 D:D), the derivative
    in the direction w adds int 4 nu'(gamma_dot)/gamma_dot (D(u):D(w)) (D(u):D(v)); for
    v = phi_a e_c, w = phi_b e_d it is int N (D grad phi_a)_c (D grad phi_b)_d (symmetric: the
    Carreau problem is the minimisation of a convex energy)."""
    phi, dphi, psi, w = tabs
    g = np.einsum("eqcl,qal->eqac", D, dphi) * (2.0 / h)        # (D grad phi_a)_c
    wq = w * (h / 2.0) ** 3
    K = np.einsum("q,eq,eqac,eqbd->eacbd", wq, N, g, g)
    return K.reshape(-1, 81, 81)


def element_matrices(form, h, nu_q, tabs):
    """Element velocity matrices K_e (ne, 81, 81) with row/col index 3*a + c.

    gradient form:  nu * delta_cd grad phi_a . grad phi_b
    symmetric form: 2 nu D(phi_b e_d) : D(phi_a e_c)
                  = nu (delta_cd grad phi_a . grad phi_b + d_d phi_a d_c phi_b)
    integrated with Gauss weights and det J = (h/2)^3, gradients scaled by 2/h.
    """
    phi, dphi, psi, w = tabs
    scale = (h / 2.0) ** 3 * (2.0 / h) ** 2
    G = np.einsum("qak,qbk->qab", dphi, dphi)            # (27q, 27, 27)
    eye = np.eye(3)
    M = np.einsum("qab,cd->qacbd", G, eye)               # delta_cd term
    if form == "symmetric":
        M = M + np.einsum("qad,qbc->qacbd", dphi, dphi)  # d_d phi_a d_c phi_b
    M = (M * (w * scale)[:, None, None, None, None]).reshape(27, 81, 81)
    return np.einsum("eq,qij->eij", nu_q, M)


def p1disc_values(tabs):
    """The discontinuous P1 pressure basis at the 27 Gauss points: 1, xi, eta, zeta (reference
    coordinates of the element, [-1, 1]^3): (27q, 4)."""
    q = np.arange(27)
    xi = np.stack([GAUSS_X[q % 3], GAUSS_X[(q // 3) % 3], GAUSS_X[q // 9]], axis=1)
    return np.concatenate([np.ones((27, 1)), xi], axis=1)


def element_divergence_p1disc(h, tabs):
    """B_e (4, 81): -int psi_k d_d phi_b for the P1-disc pressure basis (p1disc_values)."""
    phi, dphi, psi, w = tabs
    scale = (h / 2.0) ** 3 * (2.0 / h)
    Be = -np.einsum("q,qk,qbd->kbd", w * scale, p1disc_values(tabs), dphi)
    return Be.reshape(4, 81)


def element_divergence(h, tabs):
    """B_e (8, 81): -int psi_P d_d phi_b, det J (h/2)^3 and gradient scale 2/h."""
    phi, dphi, psi, w = tabs
    scale = (h / 2.0) ** 3 * (2.0 / h)
    Be = -np.einsum("q,qP,qbd->Pbd", w * scale, psi, dphi)
    return Be.reshape(8, 81)


def assemble(prob, chunk=2048, pool=None, newton=False):
    """Assemble the full saddle-point operator on free dofs plus the coupling to the
    Dirichlet velocity dofs (for lifting).

    Returns dict with
      mesh, A_cal (n x n CSR, free dofs), A_fd (n x 3 n_dirichlet_nodes, free rows x
      Dirichlet velocity columns), g_d (3 n_dirichlet_nodes,) Dirichlet values, nu_q.
    With a host pool (oracle/parallel.py) the element chunks and each round of their
    pairwise sums run on its threads; the chunks and the summation tree are the serial ones.
    newton=True adds the Newton term of the Carreau law at u_k (newton_matrices): the operator
    is then the Jacobian of the nonlinear residual (symmetric form with a Picard velocity only).
    """
    mesh = Mesh(prob)
    tabs = reference_tables()
    nu_q = quadrature_viscosity(mesh, tabs)
    Be = element_divergence(prob.h, tabs)
    ne = mesh.elems.size
    nu_tot, nd = mesh.nu, 3 * mesh.dnodes.size
    run = map if pool is None else pool.map

    # global velocity column index: free -> [0, nu), Dirichlet -> nu + [0, nd)
    vcol = np.where(mesh.vindex >= 0, 3 * mesh.vindex, -1)
    dcol = np.where(mesh.dindex >= 0, nu_tot + 3 * mesh.dindex, -1)
    node_col = np.where(vcol >= 0, vcol, dcol)            # (n_nodes,)
    nvel = nu_tot + nd

    use_newton = newton and prob.form == "symmetric" and prob.uk is not None
    if use_newton:
        Dq, Nq = quadrature_strain(mesh, tabs)

    def velocity_chunk(s):
        e = slice(s, min(ne, s + chunk))
        Ke = element_matrices(prob.form, prob.h, nu_q[e], tabs)       # (c, 81, 81)
        if use_newton:
            Ke = Ke + newton_matrices(prob.h, Dq[e], Nq[e], tabs)
        nodes = mesh.enodes[e]                                        # (c, 27)
        dof = (node_col[nodes][:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 81)
        r = np.repeat(dof[:, :, None], 81, axis=2).ravel()
        c = np.repeat(dof[:, None, :], 81, axis=1).ravel()
        return sp.csr_matrix((Ke.ravel(), (r, c)), shape=(nvel, nvel))

    parts = list(run(velocity_chunk, range(0, ne, chunk)))
    while len(parts) > 1:     # pairwise sums keep the peak memory low
        pairs = [parts[i:i + 2] for i in range(0, len(parts), 2)]
        parts = list(run(lambda ab: ab[0] + ab[1] if len(ab) == 2 else ab[0], pairs))
    K = parts[0]
    # divergence rows (pressure) x velocity columns
    vdof = (node_col[mesh.enodes][:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 81)
    if mesh.pdisc:    # Section 2's Q2 / P1-disc pair: four element-local pressure rows
        Be = element_divergence_p1disc(prob.h, tabs)
        prow = 4 * np.arange(ne)[:, None] + np.arange(4)[None, :]      # (ne, 4)
    else:
        prow = mesh.pindex[mesh.epnodes]                               # (ne, 8)
    npe = prow.shape[1]
    r = np.repeat(prow[:, :, None], 81, axis=2).ravel()
    c = np.repeat(vdof[:, None, :], npe, axis=1).ravel()
    v = np.broadcast_to(Be[None], (ne, npe, 81)).ravel()
    B = sp.csr_matrix((v, (r, c)), shape=(mesh.np_, nvel))
    A_ff = K[:nu_tot, :nu_tot]
    A_fd = K[:nu_tot, nu_tot:]
    B_f = B[:, :nu_tot]
    B_d = B[:, nu_tot:]
    A_cal = sp.bmat([[A_ff, B_f.T], [B_f, None]], format="csr")
    A_cal.sum_duplicates()
    lift = sp.vstack([A_fd, B_d], format="csr")
    g_d = prob.g[mesh.dnodes].ravel()
    return dict(mesh=mesh, A=A_cal, A_fd=lift, g_d=g_d, nu_q=nu_q)


def lifted_rhs(sys_):
    """Right-hand side of the homogeneous-Dirichlet system: F_cal = -A_(free, D) g_D
    (Section 2: u = g on the Dirichlet part, body force zero)."""
    return -(sys_["A_fd"] @ sys_["g_d"])


def full_solution(sys_, x):
    """Scatter a free-dof solution into nodal velocity (n_nodes, 3) and pressure
    (n_nodes,) arrays, inserting the Dirichlet values."""
    mesh = sys_["mesh"]
    p = mesh.p
    u = np.zeros((p.n_nodes, 3))
    u[mesh.vnodes] = x[:mesh.nu].reshape(-1, 3)
    u[mesh.dnodes] = p.g[mesh.dnodes]
    if mesh.pdisc:   # P1-disc: per fluid element (constant, d/dxi, d/deta, d/dzeta) coefficients
        return u, x[mesh.nu:].reshape(-1, 4).copy()
    pr = np.zeros(p.n_nodes)
    pr[mesh.pnodes] = x[mesh.nu:]
    return u, pr


def picard(prob, steps):
    """The Picard linearisation of Section 3 iterated: starting from the frozen velocity u_0 =
    prob.uk, step k assembles the Stokes operator with nu(u_k) at the Gauss points, solves the
    lifted system exactly (SciPy sparse LU) and takes the new velocity (free values plus the
    Dirichlet data) as u_{k+1}.  Returns the free-dof solutions x_1 .. x_steps."""
    import copy
    import scipy.sparse.linalg as spla
    p = copy.copy(prob)
    xs = []
    for _ in range(steps):
        S = assemble(p)
        x = spla.spsolve(S["A"].tocsc(), lifted_rhs(S))
        u, _ = full_solution(S, x)
        xs.append(x)
        p.uk = u
    return xs


def newton_step(prob, x):
    """One Newton step of Section 3's alternating Picard-Newton iteration from the state x
    (free dofs; prob.uk must hold its velocity with the Dirichlet data): with the nonlinear
    residual R(x) = b(nu(u)) - A(nu(u)) x, solve J(x) delta = R(x) exactly (SciPy sparse LU),
    J the Jacobian (assemble(..., newton=True)); returns x + delta and ||R(x)|| / ||b||."""
    import scipy.sparse.linalg as spla
    S = assemble(prob)
    b = lifted_rhs(S)
    R = b - S["A"] @ x
    J = assemble(prob, newton=True)["A"]
    return x + spla.spsolve(J.tocsc(), R), np.linalg.norm(R) / np.linalg.norm(b)


def picard_newton(prob, kinds):
    """Section 3's alternating Picard-Newton iteration: kinds is a string of 'P' (Picard step:
    solve A(nu(u_k)) x = b(nu(u_k))) and 'N' (Newton step from the previous iterate, which a
    'P' step must precede); u_{k+1} is each new iterate's velocity with the Dirichlet data.
    Returns the iterates x_1 .. and the nonlinear residuals ||R(x_k)|| / ||b|| before each step."""
    import copy
    import scipy.sparse.linalg as spla
    p = copy.copy(prob)
    xs, res = [], []
    x = None
    for kind in kinds:
        S = assemble(p)
        b = lifted_rhs(S)
        if kind == "P":
            if x is not None:
                res.append(np.linalg.norm(b - S["A"] @ x) / np.linalg.norm(b))
            x = spla.spsolve(S["A"].tocsc(), b)
        else:
            if x is None:
                raise ValueError("a Newton step needs a previous iterate")
            x, r = newton_step(p, x)
            res.append(r)
        u, _ = full_solution(S, x)
        p.uk = u
        xs.append(x)
    return xs, res
