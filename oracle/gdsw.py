"""Monolithic multilevel GDSW overlapping Schwarz preconditioner, FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages followed (Section 2.1 and 2.2):
  * first level: N nonoverlapping subdomains Omega_i, each enlarged by k layers of
    elements to Omega_i'; block restriction R_i = diag(R_iu, R_ip) and local saddle-point
    matrices A_i = R_i A R_i^T with homogeneous Dirichlet data on the artificial boundary;
  * interface Gamma = union of subdomain boundaries minus the Dirichlet boundary, split
    into entities (vertices, edges, faces); one coarse column per entity and null-space
    mode (velocity translations, pressure constant); interface part block-diagonal;
  * coarse basis by discrete saddle-point extension Phi_I = -A_II^{-1} A_IGamma Phi_Gamma;
  * coarse operator A_0 = Phi^T A Phi; two-level B = Phi A_0^{-1} Phi^T + sum R_i^T A_i^{-1} R_i;
  * multilevel: A_0^(l) = Phi^(l)T A_0^(l-1) Phi^(l); the inverse of A_0^(l) is replaced by
    the two-level method on a coarser decomposition, recursively; only the coarsest
    A_0^(L) is solved directly (four-level equation of Section 2.2).

Readings where the paper is silent (the same list is in the design notes):
  * overlap: Omega_i' = Omega_i plus every fluid element sharing a node with it (k = 1);
    R_i keeps the free dofs of the nodes whose every fluid element lies in Omega_i'
    (dropping the artificial rim gives the homogeneous Dirichlet condition);
  * sharing set of a node = subdomains owning a fluid element that contains it; interface
    nodes have >= 2; entity = connected component (nodes sharing an element) of interface
    nodes with free dofs and equal sharing sets, ordered by (sorted sharing set, smallest
    node id); columns (ux, uy, uz) if it has a free velocity node, p if it has a Q1 node;
  * coarse levels: a coarse node is an entity of the finer level; its part set is the set
    of coarser groups of its sharing set; two coarse nodes couple iff their sharing sets
    intersect; Omega_J' = nodes whose part set contains J plus every node coupled to one of
    them; entities and interiors as on level 1, with coarse null space = indicator of each
    mode's dofs on the entity;
  * weighting: "plain" (the paper's additive sum) or "pou" (prolongation weighted by the
    inverse multiplicity of each dof among the overlapping subdomains).

Optional variant (two levels only): rotation modes per entity (rigid rotations about the
entity's centroid), the null-space enrichment the paper leaves out.

Optional variant: the paper's Q2 / P1-disc pair (prob.pressure = "p1disc"; four pressure
dofs per element; two to four levels).  Readings: R_i keeps the pressure dofs of the
elements of Omega_i' none of whose 27 nodes lies on the artificial rim (with Dirichlet
velocity there, the constant pressure on all of Omega_i' would be a kernel of A_i); the
interface carries no pressure dof, so the coarse space gets one pressure column per
subdomain -- the constant on the subdomain's own elements, prescribed through the element
constants, which join Gamma -- while the linear pressure dofs of a subdomain's elements are
interior and extended; with one subdomain the coarse space is empty.  On a coarse level a
part's pressure column is a coarse node of that part alone: a local set keeps it only for its
own part, and the level's coarse space adds one pressure column per part (the sum of its
members' columns, prescribed through them), which is a one-part node of the next level.

Optional mixed-precision emulation (`local_precision`): the inputs and outputs of every
local solve of a level are rounded to FP32 or BF16 while the solve itself stays exact, so
that iteration counts of the GPU's mixed path (FP32/BF16 local solves recovered by the FP64
FGMRES) have an oracle counterpart.

Parity status: pinned (partition of unity, constant reproduction, extension property,
brute-force dense preconditioner, one-subdomain reduction, level collapse, symmetry; the
rotation variant by rigid rotations lying in the range of Phi; the P1-disc variant by the
Poiseuille closed form, the box-geometric count of its local pressure sets, its pressure
columns on the cavity, the extension property, brute-force dense two-, three- and four-level
operators and the coarse pressure columns counted by hand).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.sparse.csgraph import connected_components

MODES = 4   # ux, uy, uz, p


class LocalSolver:
    """Exact local solve with a sparse LU (SciPy SuperLU) or a dense LU (NumPy)."""

    def __init__(self, M):
        if sp.issparse(M):
            self.lu = spla.splu(sp.csc_matrix(M))
            self.dense = None
        else:
            self.lu = None
            self.dense = np.asarray(M)
        self.n = M.shape[0]

    def solve(self, b):
        if self.n == 0:
            return np.zeros_like(b)
        if self.lu is not None:
            return self.lu.solve(b)
        return np.linalg.solve(self.dense, b)


def _components(nodes_adj, members):
    """Connected components of the subgraph induced by `members` (sorted ids)."""
    if members.size == 1:
        return [members]
    sub = nodes_adj[members][:, members]
    ncomp, lab = connected_components(sub, directed=False)
    return [members[lab == c] for c in range(ncomp)]


class SchwarzLevel:
    """One Schwarz level: overlapping restrictions, local factors, weights, and the GDSW
    coarse basis Phi towards the next level."""

    # filled by the builders
    n: int
    dofs: list            # per overlapping subdomain: sorted global dofs
    solvers: list
    weights: list
    Phi: object           # (n, n0) sparse or dense
    n0: int
    coarse_nodes: list    # per coarse node: (sharing-set tuple, dof list, mode list)

    pool = None           # host pool holding this level's factors (oracle/parallel.py)
    pool_key = None
    rounding = None       # mixed-precision emulation: round local-solve inputs and outputs

    def local_solves(self, r):
        """[A_i^{-1} R_i r for every subdomain i], in subdomain order.  With a rounding
        function the restricted inputs and the local solutions are rounded to that precision
        (the local solve itself stays exact FP64)."""
        if self.rounding is not None:
            r = self.rounding(r)
        if self.pool is not None:
            z = self.pool.solve(self.pool_key, r)
        else:
            z = [s.solve(r[d]) for d, s in zip(self.dofs, self.solvers)]
        return z if self.rounding is None else [self.rounding(zi) for zi in z]

    def apply_local(self, r, weighting):
        z = np.zeros_like(r)
        for d, zi, w in zip(self.dofs, self.local_solves(r), self.weights):
            z[d] += (w * zi) if weighting == "pou" else zi
        return z


def round_fp32(x):
    """Round to IEEE binary32, nearest-even (NumPy's conversion), back in FP64."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_bf16(x):
    """Round to bfloat16, back in FP64: the nearest number with an 8-bit significand
    (binary32's exponent range), ties to the even significand.  With x = m 2^e and
    1/2 <= |m| < 1, m is rounded to a multiple of 2^-8 (exact scalings by powers of two and
    NumPy's round-half-even rint); normal range only, which covers every value here."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


ROUNDING = {"fp64": None, "fp32": round_fp32, "bf16": round_bf16}


def _multiplicity_weights(dofs, n):
    mult = np.zeros(n)
    for d in dofs:
        mult[d] += 1.0
    return [1.0 / mult[d] for d in dofs], mult


def _coarse_columns(entity_modes):
    """Number the coarse dofs: entities in order, modes in (ux, uy, uz, p[, rx, ry, rz])
    order."""
    col = {}
    nodes = []
    c = 0
    for e, modes in enumerate(entity_modes):
        dl, ml = [], []
        for m in range(len(modes)):
            if modes[m]:
                col[(e, m)] = c
                dl.append(c); ml.append(m)
                c += 1
        nodes.append((dl, ml))
    return col, c, nodes


def _p1disc_kept(mesh, NE, nodes):
    """P1-disc pressure dofs of the overlapping subdomain whose kept nodes are `nodes`: the four
    dofs of every fluid element all of whose 27 nodes are kept (so no element touching the
    artificial boundary carries pressure; with Dirichlet velocity there the subdomain's constant
    pressure would otherwise be a kernel of A_i)."""
    mark = np.zeros(NE.shape[0])
    mark[nodes] = 1.0
    els = np.nonzero(np.asarray(NE.T @ mark).ravel() == 27)[0]
    return (mesh.nu + 4 * els[:, None] + np.arange(4)[None, :]).ravel()


def overlapping_dofs(sys_, prob, overlap=1):
    """Free dofs of every overlapping subdomain Omega_i' (Section 2.1; overlap reading in the
    module header): index sets only, no factorisation."""
    mesh = sys_["mesh"]
    ne = mesh.elems.size
    sub = prob.part[mesh.elems].astype(np.int64)
    N = int(sub.max()) + 1
    nn = prob.n_nodes
    NE = sp.csr_matrix((np.ones(27 * ne), (mesh.enodes.ravel(), np.repeat(np.arange(ne), 27))), shape=(nn, ne))
    NE.data[:] = 1.0
    ES = sp.csr_matrix((np.ones(ne), (np.arange(ne), sub)), shape=(ne, N))
    deg = np.asarray(NE.sum(axis=1)).ravel()
    EO = ES.copy()
    for _ in range(overlap):
        EO = (NE.T @ (NE @ EO)).tocsr()
        EO.data[:] = 1.0
    cntc = (NE @ EO).tocsc()
    vnode_dof = np.where(mesh.vindex >= 0, 3 * mesh.vindex, -1)
    pnode_dof = np.where(mesh.pindex >= 0, mesh.nu + mesh.pindex, -1)
    out = []
    for i in range(N):
        col = cntc[:, i]
        nodes = col.indices[col.data == deg[col.indices]]
        v = vnode_dof[nodes]
        v = v[v >= 0]
        pp = pnode_dof[nodes]
        if mesh.pdisc:
            pp = _p1disc_kept(mesh, NE, nodes)
        out.append(np.sort(np.concatenate([(v[:, None] + np.arange(3)[None, :]).ravel(), pp[pp >= 0]])))
    return out


def build_level1(sys_, prob, overlap=1, dense_local=False, rotations=False, pool=None):
    """First level from the mesh and the element partition (Section 2.1).

    With a host pool (oracle/parallel.py) the local factorisations and the interior solves
    of the coarse basis run in its worker processes; the factors stay there and the level's
    local solves go through the pool.

    rotations=True adds, per entity with at least two free velocity nodes, the three rigid
    rotations about the entity's centroid, e_a x (x - x_c), restricted to its velocity dofs
    (modes rx, ry, rz after ux, uy, uz, p) -- the null-space enrichment that Section 2.1
    leaves out of the monolithic space.  A rotation that vanishes on the entity (the one
    about the line of a straight edge) is dropped."""
    mesh = sys_["mesh"]
    A = sys_["A"]
    n = A.shape[0]
    ne = mesh.elems.size
    sub = prob.part[mesh.elems].astype(np.int64)
    if (sub < 0).any():
        raise ValueError("every fluid element needs a subdomain")
    N = int(sub.max()) + 1
    nn = prob.n_nodes
    # node-element and node-subdomain incidence
    NE = sp.csr_matrix((np.ones(27 * ne), (mesh.enodes.ravel(), np.repeat(np.arange(ne), 27))),
                       shape=(nn, ne))
    NE.data[:] = 1.0
    ES = sp.csr_matrix((np.ones(ne), (np.arange(ne), sub)), shape=(ne, N))
    NS = (NE @ ES).tocsr()
    NS.data[:] = 1.0
    deg = np.asarray(NE.sum(axis=1)).ravel()
    # overlap: add `overlap` layers of elements sharing a node
    EO = ES.copy()
    for _ in range(overlap):
        EO = (NE.T @ (NE @ EO)).tocsr()
        EO.data[:] = 1.0
    cnt = (NE @ EO).tocsr()          # (node, subdomain): fluid elements of the node inside Omega_i'
    # dofs of a node
    vnode_dof = np.where(mesh.vindex >= 0, 3 * mesh.vindex, -1)
    pnode_dof = np.where(mesh.pindex >= 0, mesh.nu + mesh.pindex, -1)

    def node_dofs(nodes):
        nodes = np.asarray(nodes)
        out = []
        v = vnode_dof[nodes]
        vv = v[v >= 0]
        out.append((vv[:, None] + np.arange(3)[None, :]).ravel())
        pp = pnode_dof[nodes]
        out.append(pp[pp >= 0])
        return np.sort(np.concatenate(out))

    cntc = cnt.tocsc()
    lev = SchwarzLevel()
    lev.n = n
    lev.dofs = []
    for i in range(N):
        col = cntc[:, i]
        nodes = col.indices[col.data == deg[col.indices]]
        d = node_dofs(nodes)
        if mesh.pdisc:
            d = np.sort(np.concatenate([d, _p1disc_kept(mesh, NE, nodes)]))
        lev.dofs.append(d)
    lev.solvers = []
    if pool is not None and not dense_local:
        pool.share_csr("A", A)
        lev.pool, lev.pool_key = pool, "level1"
        pool.factor(lev.pool_key, "A", lev.dofs)
    else:
        for d in lev.dofs:
            Ai = A[d][:, d]
            lev.solvers.append(LocalSolver(Ai.toarray() if dense_local else Ai))
    lev.weights, lev.mult = _multiplicity_weights(lev.dofs, n)
    lev.N = N

    # --- interface and entities (Section 2.1) ---
    has_free = (mesh.vindex >= 0) | (mesh.pindex >= 0)
    nsh = np.diff(NS.indptr)
    iface = np.nonzero((nsh >= 2) & has_free)[0]
    key = {}
    for v in iface:
        s = tuple(sorted(NS.indices[NS.indptr[v]:NS.indptr[v + 1]].tolist()))
        key.setdefault(s, []).append(v)
    node_adj = (NE @ NE.T).tocsr()
    entities = []
    for s in key:
        members = np.array(sorted(key[s]))
        for comp in _components(node_adj, members):
            entities.append((s, np.sort(comp)))
    entities.sort(key=lambda t: (t[0], int(t[1][0])))
    # node coordinates: Q2 node (i, j, k) at origin + (h/2)(i, j, k)
    nid = np.arange(nn)
    xyz = np.asarray(prob.origin, dtype=np.float64)[None, :] + 0.5 * prob.h * np.stack(
        [nid % mesh.nxn, (nid // mesh.nxn) % mesh.nyn, nid // (mesh.nxn * mesh.nyn)], axis=1)
    ent_modes, ent_rot = [], []
    for s, nodes in entities:
        hv = (mesh.vindex[nodes] >= 0).any()
        hp = (mesh.pindex[nodes] >= 0).any()
        modes = [hv, hv, hv, hp]
        rot = None
        if rotations:
            vn = nodes[mesh.vindex[nodes] >= 0]
            rot = np.zeros((vn.size, 3, 3))      # rot[node, mode a, component c]
            if vn.size >= 2:
                d = xyz[vn] - xyz[vn].mean(axis=0)
                for a in range(3):
                    rot[:, a, :] = np.cross(np.eye(3)[a][None, :], d)
            keep = [np.linalg.norm(rot[:, a, :]) > 1e-8 * prob.h for a in range(3)]
            modes += keep
        ent_modes.append(modes)
        ent_rot.append(rot)
    col, n0, cnodes = _coarse_columns(ent_modes)
    # Phi_Gamma: Gamma dof -> coarse column (translations and the pressure constant are
    # indicators; rotations carry the coordinates relative to the entity's centroid)
    g_rows, g_cols, g_vals = [], [], []
    for e, (s, nodes) in enumerate(entities):
        v = vnode_dof[nodes]
        v = v[v >= 0]
        for c in range(3):
            g_rows.append(v + c); g_cols.append(np.full(v.size, col[(e, c)]) if v.size else np.zeros(0, int))
            g_vals.append(np.ones(v.size))
        pdofs = pnode_dof[nodes]
        pdofs = pdofs[pdofs >= 0]
        if pdofs.size:
            g_rows.append(pdofs); g_cols.append(np.full(pdofs.size, col[(e, 3)])); g_vals.append(np.ones(pdofs.size))
        if rotations:
            for a in range(3):
                if (e, 4 + a) not in col:
                    continue
                for c in range(3):
                    g_rows.append(v + c); g_cols.append(np.full(v.size, col[(e, 4 + a)]))
                    g_vals.append(ent_rot[e][:, a, c])
    n_ent_cols = n0
    if mesh.pdisc and N >= 2:
        # P1-disc: no pressure dof lies on the interface, so the pressure null space enters as
        # one column per subdomain -- the constant pressure on the subdomain's own elements --
        # prescribed like an interface trace (the element constants join Gamma; the linear
        # pressure dofs stay interior and are extended).  With one subdomain there is no
        # interface and the coarse space stays empty.
        el_const = mesh.nu + 4 * np.arange(ne)
        g_rows.append(el_const); g_cols.append(n0 + sub); g_vals.append(np.ones(ne))
        n0 += N
    g_rows = np.concatenate(g_rows) if g_rows else np.zeros(0, int)
    g_cols = np.concatenate(g_cols) if g_cols else np.zeros(0, int)
    g_vals = np.concatenate(g_vals) if g_vals else np.zeros(0)
    PhiG = sp.csr_matrix((g_vals, (g_rows, g_cols)), shape=(n, n0))
    gamma = np.zeros(n, dtype=bool)
    gamma[g_rows] = True
    # interior dofs of each subdomain: free dofs of nodes with sharing set {i}
    inter_nodes = np.nonzero((nsh == 1) & has_free)[0]
    owner = NS.indices[NS.indptr[inter_nodes]]
    lev.interior = []
    Phi_rows, Phi_cols, Phi_vals = [g_rows], [g_cols], [g_vals]
    AG = A[:, gamma.nonzero()[0]] @ PhiG[gamma.nonzero()[0]]       # A_{:,Gamma} Phi_Gamma
    AG = AG.tocsr()
    blocks = []                      # (interior dofs, coupled columns, -A_IGamma Phi_Gamma)
    for i in range(N):
        I = node_dofs(inter_nodes[owner == i])
        if mesh.pdisc:   # the pressure dofs of the subdomain's own elements that are not in Gamma
            els = np.nonzero(sub == i)[0]
            k = np.arange(1, 4) if N >= 2 else np.arange(4)
            I = np.sort(np.concatenate([I, (mesh.nu + 4 * els[:, None] + k[None, :]).ravel()]))
        lev.interior.append(I)
        if I.size == 0 or n0 == 0:
            continue
        rhs = -AG[I]
        cols = np.unique(rhs.indices)
        if cols.size == 0:
            continue
        blocks.append((I, cols, rhs[:, cols].toarray()))
    if pool is not None:
        pool.share_csr("A", A)
        Xs = pool.extend("A", [(I, R) for I, cols, R in blocks])
    else:
        Xs = [LocalSolver(A[I][:, I]).solve(R) for I, cols, R in blocks]
    for (I, cols, R), X in zip(blocks, Xs):
        rr, cc = np.meshgrid(I, cols, indexing="ij")
        Phi_rows.append(rr.ravel()); Phi_cols.append(cc.ravel()); Phi_vals.append(X.ravel())
    lev.Phi = sp.csr_matrix((np.concatenate(Phi_vals), (np.concatenate(Phi_rows), np.concatenate(Phi_cols))),
                            shape=(n, n0))
    lev.PhiGamma = PhiG
    lev.gamma = gamma
    lev.n0 = n0
    lev.coarse_nodes = [(entities[e][0], cnodes[e][0], cnodes[e][1]) for e in range(len(entities))]
    if mesh.pdisc and N >= 2:   # the subdomain pressure columns as coarse nodes of one part each
        lev.coarse_nodes += [((i,), [n_ent_cols + i], [3]) for i in range(N)]
    lev.entities = entities
    if n0 == 0:
        A0 = np.zeros((0, 0))
    elif pool is None:
        A0 = (lev.Phi.T @ (A @ lev.Phi)).toarray()
    else:   # the same products, by row blocks on the pool's threads
        AP = pool.row_product(A, lev.Phi)
        A0 = pool.row_product(lev.Phi.T.tocsr(), AP).toarray()
    return lev, A0


def build_coarse_level(A, cnodes, group, dense_local=True):
    """A Schwarz level on a coarse operator (Section 2.2 recursion).

    A: dense coarse operator of the finer level; cnodes: list of (sharing set, dofs, modes)
    per coarse node; group: maps each finer-level part to its part on this level.

    A coarse node whose sharing set has one part is a part's own pressure column (the P1-disc
    variant): it carries no interface, so, as on the first level, (a) a local set keeps it only
    if its part belongs to the set's own part (the pressure of neighbouring parts is dropped
    with the overlap's rim), (b) this level's coarse space gets one pressure column per part,
    the sum of its members' columns, prescribed through them (they join Gamma), and (c) those
    columns become the next level's one-part coarse nodes."""
    n = A.shape[0]
    nn = len(cnodes)
    parts = [tuple(sorted({int(group[i]) for i in s})) for (s, d, m) in cnodes]
    own = np.array([len(s) == 1 for (s, d, m) in cnodes], dtype=bool)   # part pressure nodes
    N = int(np.max(group)) + 1 if len(group) else 1
    # structural coupling: sharing sets intersect
    inc_r, inc_c = [], []
    for v, (s, d, m) in enumerate(cnodes):
        inc_r += [v] * len(s); inc_c += list(s)
    NS = sp.csr_matrix((np.ones(len(inc_r)), (inc_r, inc_c)), shape=(nn, max(inc_c) + 1 if inc_c else 1))
    adj = (NS @ NS.T).tocsr()
    adj.data[:] = 1.0
    lev = SchwarzLevel()
    lev.n = n
    lev.N = N
    lev.dofs = []
    for J in range(N):
        closure = np.array([v for v in range(nn) if J in parts[v]], dtype=int)
        if closure.size:
            ext = np.unique(adj[closure].indices)
            ext = ext[~own[ext] | np.isin(ext, closure)]
        else:
            ext = closure
        d = np.sort(np.concatenate([np.array(cnodes[v][1], dtype=int) for v in ext])) if ext.size else np.zeros(0, int)
        lev.dofs.append(d)
    lev.solvers = [LocalSolver(A[np.ix_(d, d)]) for d in lev.dofs]
    lev.weights, lev.mult = _multiplicity_weights(lev.dofs, n)
    # entities of this level
    key = {}
    for v in range(nn):
        if len(parts[v]) >= 2:
            key.setdefault(parts[v], []).append(v)
    entities = []
    for s in key:
        members = np.array(sorted(key[s]))
        for comp in _components(adj, members):
            entities.append((s, np.sort(comp)))
    entities.sort(key=lambda t: (t[0], int(t[1][0])))
    ent_modes = []
    for s, nodes in entities:
        present = [False] * MODES
        for v in nodes:
            for mm in cnodes[v][2]:
                present[mm] = True
        ent_modes.append(present)
    col, n0, cn = _coarse_columns(ent_modes)
    n_ent_cols = n0
    pcols = bool(own.any()) and N >= 2
    if pcols:
        n0 += N
    PhiG = np.zeros((n, n0))
    gamma = np.zeros(n, dtype=bool)
    for e, (s, nodes) in enumerate(entities):
        for v in nodes:
            for dof, mm in zip(cnodes[v][1], cnodes[v][2]):
                PhiG[dof, col[(e, mm)]] = 1.0
                gamma[dof] = True
    if pcols:
        for v in np.nonzero(own)[0]:
            for dof in cnodes[v][1]:
                PhiG[dof, n_ent_cols + parts[v][0]] = 1.0
                gamma[dof] = True
    Phi = PhiG.copy()
    lev.interior = []
    for J in range(N):
        inodes = [v for v in range(nn) if parts[v] == (J,) and not (pcols and own[v])]
        I = np.sort(np.array([dd for v in inodes for dd in cnodes[v][1]], dtype=int))
        lev.interior.append(I)
        if I.size == 0 or n0 == 0:
            continue
        G = gamma.nonzero()[0]
        rhs = -A[np.ix_(I, G)] @ PhiG[G]
        Phi[I] = LocalSolver(A[np.ix_(I, I)]).solve(rhs)
    lev.Phi = Phi
    lev.PhiGamma = PhiG
    lev.gamma = gamma
    lev.n0 = n0
    lev.coarse_nodes = [(entities[e][0], cn[e][0], cn[e][1]) for e in range(len(entities))]
    if pcols:
        lev.coarse_nodes += [((J,), [n_ent_cols + J], [3]) for J in range(N)]
    lev.entities = entities
    A0 = Phi.T @ A @ Phi
    return lev, A0


class GDSW:
    """Multilevel monolithic GDSW preconditioner (Section 2.2 four-level equation, for
    L = 2, 3, 4 levels)."""

    def __init__(self, sys_, prob, levels=None, weighting="pou", overlap=1, dense_local=False, rotations=False,
                 pool=None, local_precision=None):
        """local_precision: None (all FP64) or one of "fp64", "fp32", "bf16" per Schwarz level
        (levels 1 .. L-1): the mixed-precision emulation rounds that level's local-solve inputs
        and outputs to the given precision; the coarsest direct solve stays FP64."""
        L = prob.levels if levels is None else levels
        if rotations and L > 2:
            raise ValueError("rotation modes are defined for two-level GDSW only")
        self.L = L
        self.weighting = weighting
        self.levels = []
        self.pool = pool
        lev, A0 = build_level1(sys_, prob, overlap=overlap, dense_local=dense_local, rotations=rotations,
                               pool=pool)
        if pool is not None:      # the first level's transfers as row-block products
            lev.PhiT = lev.Phi.T.tocsr()
        self.levels.append(lev)
        self.A0 = [sys_["A"], A0]
        for l in range(2, L):
            cn = self.levels[-1].coarse_nodes
            lev, A0 = build_coarse_level(A0, cn, prob.groups[l - 2])
            self.levels.append(lev)
            self.A0.append(A0)
        self.coarsest = LocalSolver(A0)
        for lev, prec in zip(self.levels, local_precision or ()):
            lev.rounding = ROUNDING[prec]

    def apply(self, r, level=0):
        """z = B r, recursively: local sum on this level plus Phi (next level) Phi^T."""
        lev = self.levels[level]
        z = lev.apply_local(r, self.weighting)
        if lev.n0 == 0:
            return z
        pooled = self.pool is not None and level == 0
        r0 = self.pool.matvec(lev.PhiT, r) if pooled else lev.Phi.T @ r
        if level + 1 == len(self.levels):
            x0 = self.coarsest.solve(r0)
        else:
            x0 = self.apply(r0, level + 1)
        return z + (self.pool.matvec(lev.Phi, x0) if pooled else lev.Phi @ x0)

    def dense(self):
        """The preconditioner as a dense matrix (for small tests)."""
        n = self.levels[0].n
        return np.column_stack([self.apply(e) for e in np.eye(n)])
