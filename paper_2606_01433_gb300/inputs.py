"""Seeded synthetic inputs for the GDSW Stokes solver (shared by the library's tests,
the benchmark and the FP64 CPU oracle).

This module holds NO arithmetic of the method: no finite-element basis, no assembly,
no Schwarz or Krylov step.  It only describes problems: a voxel box of hexahedral
elements, an element mask (fluid elements), a per-node boundary tag and Dirichlet
datum, a frozen Picard velocity sampled from an analytic field, a right-hand side of
random numbers, an element partition and the grouping of subdomains into coarser
levels.  Everything is a plain numpy array so that both the CUDA library (through its
C ABI) and the CPU oracle receive bit-identical inputs.

Conventions (the C ABI documents the same ones):
  * element (ex, ey, ez) has linear index ex + nx*(ey + ny*ez); the mask is uint8 of
    shape (nz, ny, nx) flattened in that order;
  * Q2 node (i, j, k), i in [0, 2nx], sits at origin + (h/2)*(i, j, k) and has linear
    index i + (2nx+1)*(j + (2ny+1)*k);
  * node tags: 0 interior, 1 no-slip wall (Dirichlet 0), 2 inflow (Dirichlet g),
    3 outflow / natural boundary.  Only tags 1 and 2 are Dirichlet.

The workloads follow the model problem of the paper (Section 3: stationary Carreau
Stokes flow with inflow, outflow and no-slip walls) on synthetic geometries, because the
extrusion-die mesh of the paper's Figure 1 is not available.
"""
from __future__ import annotations

import dataclasses
import numpy as np

TAG_INTERIOR, TAG_WALL, TAG_INFLOW, TAG_OUTFLOW = 0, 1, 2, 3


@dataclasses.dataclass
class Problem:
    """One Stokes problem instance: mesh, boundary data, viscosity, partition."""
    name: str
    nx: int
    ny: int
    nz: int
    h: float
    origin: tuple
    mask: np.ndarray            # uint8 (nx*ny*nz,) 1 = fluid element
    tags: np.ndarray            # uint8 (n_nodes,)
    g: np.ndarray               # float64 (n_nodes, 3) Dirichlet datum (used where tag in {1,2})
    form: str                   # "gradient" (mu grad u : grad v) or "symmetric" (2 nu D(u):D(v))
    nu0: float = 1.0
    nu_inf: float = 0.0
    lam: float = 0.0
    n_carreau: float = 1.0
    uk: np.ndarray | None = None   # float64 (n_nodes, 3) frozen Picard velocity, None = Newtonian
    part: np.ndarray | None = None  # int32 (n_elems,) subdomain of each element, -1 for void
    groups: list = dataclasses.field(default_factory=list)  # level l>=2 grouping arrays (int32)
    levels: int = 2
    rhs_seed: int | None = None     # random right-hand side on free dofs (seeded), else lifted inflow
    pressure: str = "q1"            # "q1": continuous Q1 (Taylor-Hood); "p1disc": discontinuous P1
                                    # per element (constant and three linear dofs, element order)

    @property
    def n_nodes(self) -> int:
        return (2 * self.nx + 1) * (2 * self.ny + 1) * (2 * self.nz + 1)

    @property
    def n_elems(self) -> int:
        return self.nx * self.ny * self.nz

    def node_coords(self) -> np.ndarray:
        """(n_nodes, 3) coordinates of every Q2 node of the box."""
        nxn, nyn, nzn = 2 * self.nx + 1, 2 * self.ny + 1, 2 * self.nz + 1
        k, j, i = np.meshgrid(np.arange(nzn), np.arange(nyn), np.arange(nxn), indexing="ij")
        c = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
        return np.asarray(self.origin, dtype=np.float64)[None, :] + 0.5 * self.h * c


# ----------------------------------------------------------------------------------
# geometry helpers (no method arithmetic: only which voxel is fluid and where walls are)
# ----------------------------------------------------------------------------------

def element_centers(nx, ny, nz, h, origin):
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    c = np.stack([ex.ravel(), ey.ravel(), ez.ravel()], axis=1).astype(np.float64) + 0.5
    return np.asarray(origin, dtype=np.float64)[None, :] + h * c


def _node_touch_void(nx, ny, nz, mask, open_face=None):
    """For every Q2 node: (touches a void element position, touches a fluid element).
    Element positions outside the box count as void, except across open_face
    ((axis, side)), where the fluid is continued one layer beyond the box."""
    m = mask.reshape(nz, ny, nx).astype(bool)
    pad = np.zeros((nz + 2, ny + 2, nx + 2), dtype=bool)
    pad[1:-1, 1:-1, 1:-1] = m
    if open_face is not None:
        ax, side = open_face
        npax = 2 - ax
        src = [slice(1, -1)] * 3
        dst = [slice(1, -1)] * 3
        src[npax] = slice(-2, -1) if side == 1 else slice(1, 2)
        dst[npax] = slice(-1, None) if side == 1 else slice(0, 1)
        pad[tuple(dst)] = pad[tuple(src)]
    nxn, nyn, nzn = 2 * nx + 1, 2 * ny + 1, 2 * nz + 1
    ii, jj, kk = np.arange(nxn), np.arange(nyn), np.arange(nzn)

    def cand(idx):
        # element positions (shifted by +1 for the padding) containing node coordinate idx
        lo = np.where(idx % 2 == 0, idx // 2 - 1, idx // 2) + 1
        hi = idx // 2 + 1
        return lo, hi

    li, hi_ = cand(ii)
    lj, hj = cand(jj)
    lk, hk = cand(kk)
    any_void = np.zeros((nzn, nyn, nxn), dtype=bool)
    any_fluid = np.zeros((nzn, nyn, nxn), dtype=bool)
    for ck in (lk, hk):
        for cj in (lj, hj):
            for ci in (li, hi_):
                v = pad[ck[:, None, None], cj[None, :, None], ci[None, None, :]]
                any_void |= ~v
                any_fluid |= v
    return any_void.ravel(), any_fluid.ravel()


def boundary_tags(nx, ny, nz, h, origin, mask, inflow, outflow, extent=None):
    """Tag boundary nodes of the fluid region.

    inflow / outflow: (axis, side) with side 0 = low face, 1 = high face of the box.
    A boundary node on the inflow face is inflow; a boundary node on the outflow face that
    touches void only through that face is outflow; every other boundary node is a
    no-slip wall.
    """
    any_void, any_fluid = _node_touch_void(nx, ny, nz, mask)
    nxn, nyn, nzn = 2 * nx + 1, 2 * ny + 1, 2 * nz + 1
    k, j, i = np.meshgrid(np.arange(nzn), np.arange(nyn), np.arange(nxn), indexing="ij")
    ijk = [i.ravel(), j.ravel(), k.ravel()]
    nmax = [2 * nx, 2 * ny, 2 * nz]
    tags = np.zeros(nxn * nyn * nzn, dtype=np.uint8)
    bnd = any_void & any_fluid
    tags[bnd] = TAG_WALL

    def on_face(ax, side):
        return ijk[ax] == (0 if side == 0 else nmax[ax])

    if outflow is not None:
        void_open, _ = _node_touch_void(nx, ny, nz, mask, open_face=outflow)
        tags[bnd & on_face(*outflow) & ~void_open] = TAG_OUTFLOW
    if inflow is not None:
        tags[bnd & on_face(*inflow)] = TAG_INFLOW
    return tags


def box_partition(nx, ny, nz, parts, mask=None):
    """Element -> subdomain for a px*py*pz box partition (void elements get -1).
    Subdomains are renumbered densely (empty boxes dropped)."""
    px, py, pz = parts
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    bx, by, bz = ex.ravel() * px // nx, ey.ravel() * py // ny, ez.ravel() * pz // nz
    sub = (bx + px * (by + py * bz)).astype(np.int64)
    if mask is not None:
        sub = np.where(mask.astype(bool), sub, -1)
    used = np.unique(sub[sub >= 0])
    remap = -np.ones(px * py * pz, dtype=np.int64)
    remap[used] = np.arange(used.size)
    out = np.where(sub >= 0, remap[np.maximum(sub, 0)], -1).astype(np.int32)
    return out, used


def box_groups(parts, group, used):
    """Group box subdomains (bx,by,bz) into boxes of size group; returns the dense group
    index of every used subdomain and the number of groups."""
    px, py, pz = parts
    gx, gy, gz = group
    b = np.asarray(used)
    bx, by, bz = b % px, (b // px) % py, b // (px * py)
    qx, qy = (px + gx - 1) // gx, (py + gy - 1) // gy
    gid = (bx // gx) + qx * ((by // gy) + qy * (bz // gz))
    u = np.unique(gid)
    remap = {int(v): i for i, v in enumerate(u)}
    return np.array([remap[int(v)] for v in gid], dtype=np.int32), gid


def rcb_partition(centers, active, nparts):
    """Recursive coordinate bisection of the active elements into nparts (a power of two):
    split along the longest extent at the median count, ties by element index.  Part ids
    are numbered in tree order, so parts 8q..8q+7 are the leaves of one subtree."""
    idx = np.nonzero(active)[0]
    out = -np.ones(active.size, dtype=np.int32)

    def rec(ids, p0, np_):
        if np_ == 1:
            out[ids] = p0
            return
        c = centers[ids]
        ax = int(np.argmax(c.max(axis=0) - c.min(axis=0))) if ids.size else 0
        order = np.lexsort((ids, c[:, ax]))
        half = ids.size // 2
        rec(ids[order[:half]], p0, np_ // 2)
        rec(ids[order[half:]], p0 + np_ // 2, np_ // 2)

    rec(idx, 0, nparts)
    return out


# ----------------------------------------------------------------------------------
# analytic fields (input definitions)
# ----------------------------------------------------------------------------------

def sine_field(rng, n_modes=8, kmax=4):
    """Random analytic velocity field u(x) = sum_m a_m sin(pi k_m . x + phi_m)."""
    a = rng.standard_normal((n_modes, 3))
    k = rng.integers(1, kmax + 1, size=(n_modes, 3)).astype(np.float64)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    return a, k, phi


def sine_eval(field, x, amp):
    a, k, phi = field
    arg = np.pi * x @ k.T + phi[None, :]
    return amp * np.sin(arg) @ a


def sine_grad_fro(field, x, amp):
    """Frobenius norm of the analytic gradient of the sine field at points x."""
    a, k, phi = field
    arg = np.pi * x @ k.T + phi[None, :]
    cos = np.cos(arg)                       # (P, M)
    # grad u_{c,l} = sum_m a_{m,c} pi k_{m,l} cos_m
    g = np.einsum("pm,mc,ml->pcl", cos, a, np.pi * k) * amp
    return np.sqrt((g ** 2).sum(axis=(1, 2)))


def picard_velocity(p: Problem, seed: int):
    """Frozen Picard velocity: a random sine field scaled so that the median Frobenius norm
    of its analytic gradient over fluid-element centres equals 1/lambda; zero on walls
    and equal to g on the inflow."""
    rng = np.random.default_rng(seed)
    field = sine_field(rng)
    cen = element_centers(p.nx, p.ny, p.nz, p.h, p.origin)[p.mask.astype(bool)]
    med = float(np.median(sine_grad_fro(field, cen, 1.0)))
    amp = 1.0 / (max(p.lam, 1e-30) * med)
    x = p.node_coords()
    u = sine_eval(field, x, amp)
    u[p.tags == TAG_WALL] = 0.0
    u[p.tags == TAG_INFLOW] = p.g[p.tags == TAG_INFLOW]
    return np.ascontiguousarray(u)


def mg_hierarchy(m=64, grids=3, parts=(8, 8, 8), groups=((2, 2, 2), (2, 2, 2)), levels=4, seed=4,
                 nu0=1.0, nu_inf=1e-3, lam=1.0, n=0.5, carreau=True):
    """Nested voxel grids for the geometric-multigrid role of the paper (Section 3: the
    multigrid solver whose coarsest problem the multilevel Schwarz method solves): the
    unit-cube channel (inflow x=0 with g = 16 y(1-y) z(1-z) e_x, outflow x=1, no-slip walls)
    with m, m/2, ..., m/2^(grids-1) elements per edge, finest first.  Every grid samples the
    same inflow profile and, for a Carreau fluid, the same frozen Picard velocity (the sine
    field and amplitude of the finest grid, zero on walls and g on the inflow), so a coarse
    node's values equal the fine values at the same point.  The coarsest grid carries the box
    partition and grouping of the multilevel GDSW coarse solver; the finest carries a random
    right-hand side on its free dofs (seed).  Newtonian (nu0, gradient form) when not
    carreau."""
    if m % (1 << (grids - 1)):
        raise ValueError("m must be divisible by 2^(grids-1)")
    out = []
    fa = None
    for gl in range(grids):
        mm = m >> gl
        h = 1.0 / mm
        mask = np.ones(mm ** 3, dtype=np.uint8)
        tags = boundary_tags(mm, mm, mm, h, (0, 0, 0), mask, inflow=(0, 0), outflow=(0, 1), extent=None)
        last = gl == grids - 1
        p = Problem("mg_cube_%d" % mm, mm, mm, mm, h, (0.0, 0.0, 0.0), mask, tags,
                    np.zeros(((2 * mm + 1) ** 3, 3)), "symmetric" if carreau else "gradient", nu0=nu0,
                    nu_inf=nu_inf if carreau else 0.0, lam=lam if carreau else 0.0, n_carreau=n if carreau else 1.0,
                    levels=levels if last else 2, rhs_seed=seed if gl == 0 else None)
        x = p.node_coords()
        inl = tags == TAG_INFLOW
        p.g[inl, 0] = 16.0 * x[inl, 1] * (1 - x[inl, 1]) * x[inl, 2] * (1 - x[inl, 2])
        if carreau:
            if fa is None:
                rng = np.random.default_rng(seed)
                field = sine_field(rng)
                cen = element_centers(mm, mm, mm, h, p.origin)
                fa = (field, 1.0 / (max(lam, 1e-30) * float(np.median(sine_grad_fro(field, cen, 1.0)))))
            u = sine_eval(fa[0], x, fa[1])
            u[tags == TAG_WALL] = 0.0
            u[inl] = p.g[inl]
            p.uk = np.ascontiguousarray(u)
        if last:
            p.part, used = box_partition(mm, mm, mm, parts)
            p.groups = _groups_from_boxes(parts, groups, used, levels)
        else:
            p.part, _ = box_partition(mm, mm, mm, (1, 1, 1))
            p.groups = []
        out.append(p)
    return out


def random_rhs(n_free: int, seed: int):
    """b ~ N(0, 1) on the free dofs."""
    return np.random.default_rng(seed).standard_normal(n_free)


# ----------------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------------

def unit_cube(m=8, parts=(2, 2, 2), seed=1, groups=None, levels=2):
    """Newtonian Stokes (nu = 1, gradient form) on the unit cube with m^3 Q2/Q1 hexahedra:
    Dirichlet inflow at x=0, no-slip walls on y and z faces, do-nothing outflow at x=1,
    box partition, random right-hand side on the free dofs."""
    h = 1.0 / m
    mask = np.ones(m ** 3, dtype=np.uint8)
    tags = boundary_tags(m, m, m, h, (0, 0, 0), mask, inflow=(0, 0), outflow=(0, 1), extent=None)
    p = Problem("unit_cube_%d" % m, m, m, m, h, (0.0, 0.0, 0.0), mask, tags,
                np.zeros(((2 * m + 1) ** 3, 3)), "gradient", nu0=1.0, rhs_seed=seed, levels=levels)
    x = p.node_coords()
    inl = tags == TAG_INFLOW
    p.g[inl, 0] = 16.0 * x[inl, 1] * (1 - x[inl, 1]) * x[inl, 2] * (1 - x[inl, 2])
    p.part, used = box_partition(m, m, m, parts)
    p.groups = _groups_from_boxes(parts, groups, used, levels)
    return p


def _groups_from_boxes(parts, groups, used, levels):
    """Grouping arrays for levels 2.. of a box partition: entry l maps each level-(l+1)
    part to its level-(l+2) group (dense indices)."""
    out = []
    if levels >= 3 and groups is not None:
        g1, gid = box_groups(parts, groups[0], used)
        out.append(g1)
        if levels >= 4:
            q = tuple((parts[a] + groups[0][a] - 1) // groups[0][a] for a in range(3))
            g2, _ = box_groups(q, groups[1], np.unique(gid))
            out.append(g2)
    return out


def poiseuille(m=4, G=1.0, parts=(1, 1, 1), groups=None, levels=2, pressure="q1"):
    """Analytic Poiseuille pin: nu = 1, gradient form on the unit cube,
    u = (G/2) y (1-y) e_x and p = G (1-x); Dirichlet u = exact on x=0 and the y, z faces,
    do-nothing outflow at x=1."""
    h = 1.0 / m
    mask = np.ones(m ** 3, dtype=np.uint8)
    tags = boundary_tags(m, m, m, h, (0, 0, 0), mask, inflow=(0, 0), outflow=(0, 1), extent=None)
    tags = np.where(tags == TAG_WALL, TAG_INFLOW, tags).astype(np.uint8)
    p = Problem("poiseuille_%d" % m, m, m, m, h, (0.0, 0.0, 0.0), mask, tags,
                np.zeros(((2 * m + 1) ** 3, 3)), "gradient", nu0=1.0, levels=levels, pressure=pressure)
    x = p.node_coords()
    p.g[:, 0] = 0.5 * G * x[:, 1] * (1 - x[:, 1])
    p.g[tags == TAG_OUTFLOW] = 0.0
    p.g[tags == TAG_INTERIOR] = 0.0
    p.part, used = box_partition(m, m, m, parts)
    p.groups = _groups_from_boxes(parts, groups, used, levels)
    return p


def poiseuille_exact(p: Problem, G=1.0):
    x = p.node_coords()
    u = np.zeros_like(x)
    u[:, 0] = 0.5 * G * x[:, 1] * (1 - x[:, 1])
    pr = G * (1.0 - x[:, 0])
    return u, pr


def channel(m=32, parts=(4, 4, 4), groups=((2, 2, 2),), levels=3, seed=2,
            nu0=1.0, nu_inf=1e-3, lam=1.0, n=0.5, U=1.0):
    """Carreau Stokes in the unit-cube channel with four z-axis cylinders of radius 0.06
    at (x, y) = (0.25, 0.3), (0.25, 0.7), (0.55, 0.5), (0.8, 0.35) (elements whose centre
    lies inside are void); inflow x=0 with g = 16 U y(1-y) z(1-z) e_x, traction-free
    outflow x=1, no-slip elsewhere; symmetric form; frozen Picard velocity from seed."""
    h = 1.0 / m
    cen = element_centers(m, m, m, h, (0, 0, 0))
    mask = np.ones(m ** 3, dtype=np.uint8)
    for cx, cy in ((0.25, 0.3), (0.25, 0.7), (0.55, 0.5), (0.8, 0.35)):
        mask[(cen[:, 0] - cx) ** 2 + (cen[:, 1] - cy) ** 2 < 0.06 ** 2] = 0
    tags = boundary_tags(m, m, m, h, (0, 0, 0), mask, inflow=(0, 0), outflow=(0, 1), extent=None)
    p = Problem("channel_%d" % m, m, m, m, h, (0.0, 0.0, 0.0), mask, tags,
                np.zeros(((2 * m + 1) ** 3, 3)), "symmetric", nu0=nu0, nu_inf=nu_inf, lam=lam,
                n_carreau=n, levels=levels)
    x = p.node_coords()
    inl = tags == TAG_INFLOW
    p.g[inl, 0] = 16.0 * U * x[inl, 1] * (1 - x[inl, 1]) * x[inl, 2] * (1 - x[inl, 2])
    p.uk = picard_velocity(p, seed)
    p.part, used = box_partition(m, m, m, parts, mask)
    p.groups = _groups_from_boxes(parts, groups, used, levels)
    return p


def die(nx=64, ny=64, nz=128, nparts=512, per_group=8, levels=4, seed=3,
        nu0=1.0, nu_inf=1e-3, lam=1.0, n=0.4):
    """Die-like channel in the box [0,1]x[0,1]x[0,2]: two circular inlet ports at z=0
    (centres x = 0.3, 0.7, y = 0.5, radius 0.12) blend over z in [0, 0.8] into a slot
    whose half-width tapers 0.35 -> 0.45 and half-height 0.2 -> 0.05 at z = 2.  Inflow
    through the ports at z=0 (parabolic in each port), outflow at z=2, RCB partition into
    nparts with groups of per_group consecutive parts per coarser level."""
    h = 1.0 / nx
    cen = element_centers(nx, ny, nz, h, (0, 0, 0))
    xx, yy, zz = cen[:, 0], cen[:, 1], cen[:, 2]
    d_ports = np.minimum(np.hypot(xx - 0.3, yy - 0.5), np.hypot(xx - 0.7, yy - 0.5)) - 0.12
    a = 0.35 + 0.05 * zz
    b = 0.2 - 0.075 * zz
    d_slot = np.maximum(np.abs(xx - 0.5) - a, np.abs(yy - 0.5) - b)
    t = np.clip(zz / 0.8, 0.0, 1.0)
    s = t * t * (3 - 2 * t)
    d = np.where(zz < 0.8, (1 - s) * d_ports + s * d_slot, d_slot)
    mask = (d < 0).astype(np.uint8)
    tags = boundary_tags(nx, ny, nz, h, (0, 0, 0), mask, inflow=(2, 0), outflow=(2, 1), extent=None)
    p = Problem("die_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, h, (0.0, 0.0, 0.0), mask, tags,
                np.zeros(((2 * nx + 1) * (2 * ny + 1) * (2 * nz + 1), 3)), "symmetric", nu0=nu0,
                nu_inf=nu_inf, lam=lam, n_carreau=n, levels=levels)
    x = p.node_coords()
    inl = tags == TAG_INFLOW
    r2 = np.minimum((x[inl, 0] - 0.3) ** 2, (x[inl, 0] - 0.7) ** 2) + (x[inl, 1] - 0.5) ** 2
    p.g[inl, 2] = np.maximum(0.0, 1.0 - r2 / 0.12 ** 2)
    p.uk = picard_velocity(p, seed)
    p.part = rcb_partition(cen, mask.astype(bool), nparts)
    gr = []
    nsub = nparts
    for _ in range(levels - 2):
        gr.append((np.arange(nsub) // per_group).astype(np.int32))
        nsub = (nsub + per_group - 1) // per_group
    p.groups = gr
    return p


def serving_requests(n_req=256, seed=5, sizes=(8, 12, 16, 20, 24, 28, 32)):
    """Request mix for the serving loop: unit-cube Carreau channels of m^3 elements with
    m ~ U{sizes}, n ~ U[0.3, 1], nu0 = 1 and nu0/nu_inf log-uniform in [10, 1e4]; meshes
    up to 16^3 use a 2x2x2 two-level partition, larger ones 4x4x4 grouped 2x2x2 (three
    levels).  Returns a list of (arrival_seed, parameters) dictionaries."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_req):
        m = int(rng.choice(sizes))
        out.append(dict(m=m, n=float(rng.uniform(0.3, 1.0)),
                        nu_inf=float(1.0 / 10 ** rng.uniform(1.0, 4.0)),
                        seed=int(rng.integers(0, 2 ** 31 - 1))))
    return out


def carreau_cube(m, n, nu_inf, seed, lam=1.0):
    """Unit-cube Carreau channel used by the serving workload (no obstacles)."""
    parts, groups, levels = ((2, 2, 2), None, 2) if m <= 16 else ((4, 4, 4), ((2, 2, 2),), 3)
    h = 1.0 / m
    mask = np.ones(m ** 3, dtype=np.uint8)
    tags = boundary_tags(m, m, m, h, (0, 0, 0), mask, inflow=(0, 0), outflow=(0, 1), extent=None)
    p = Problem("carreau_cube_%d" % m, m, m, m, h, (0.0, 0.0, 0.0), mask, tags,
                np.zeros(((2 * m + 1) ** 3, 3)), "symmetric", nu0=1.0, nu_inf=nu_inf, lam=lam,
                n_carreau=n, levels=levels)
    x = p.node_coords()
    inl = tags == TAG_INFLOW
    p.g[inl, 0] = 16.0 * x[inl, 1] * (1 - x[inl, 1]) * x[inl, 2] * (1 - x[inl, 2])
    p.uk = picard_velocity(p, seed)
    p.part, used = box_partition(m, m, m, parts)
    p.groups = _groups_from_boxes(parts, groups, used, levels)
    return p


def box_problem(nx, ny, nz, parts, groups=None, levels=2, form="gradient", bc="channel",
                seed=1, uk_seed=None, nu0=1.0, nu_inf=0.0, lam=0.0, n=1.0, pressure="q1"):
    """Small box problems for tests.  bc: "channel" (inflow x=0 with a parabolic profile,
    outflow x=1, walls elsewhere), "neumann" (every boundary node natural) or "cavity"
    (every boundary node a no-slip wall)."""
    h = 1.0 / max(nx, ny, nz)
    mask = np.ones(nx * ny * nz, dtype=np.uint8)
    if bc == "channel":
        tags = boundary_tags(nx, ny, nz, h, (0, 0, 0), mask, inflow=(0, 0), outflow=(0, 1))
    else:
        tags = boundary_tags(nx, ny, nz, h, (0, 0, 0), mask, inflow=None, outflow=None)
        if bc == "neumann":
            tags = np.where(tags == TAG_WALL, TAG_OUTFLOW, tags).astype(np.uint8)
    nn = (2 * nx + 1) * (2 * ny + 1) * (2 * nz + 1)
    p = Problem("box_%dx%dx%d_%s" % (nx, ny, nz, bc), nx, ny, nz, h, (0.0, 0.0, 0.0), mask, tags,
                np.zeros((nn, 3)), form, nu0=nu0, nu_inf=nu_inf, lam=lam, n_carreau=n,
                rhs_seed=seed, levels=levels, pressure=pressure)
    x = p.node_coords()
    inl = tags == TAG_INFLOW
    ly, lz = ny * h, nz * h
    p.g[inl, 0] = 16.0 * (x[inl, 1] / ly) * (1 - x[inl, 1] / ly) * (x[inl, 2] / lz) * (1 - x[inl, 2] / lz)
    if uk_seed is not None:
        p.uk = picard_velocity(p, uk_seed)
    p.part, used = box_partition(nx, ny, nz, parts)
    p.groups = _groups_from_boxes(parts, groups, used, levels)
    return p
