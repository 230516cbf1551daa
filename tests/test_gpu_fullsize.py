"""Parity at the benchmark's full size (Carreau channel 32^3, four cylinders, 4x4x4 parts
grouped 2x2x2, three levels; FP32 local factors as bench.py times it), on what the FP64
oracle can compute one by one:
  * the assembled operator (Section 2 / 3) and the SpMV against the oracle's assembly;
  * the overlapping dof sets of all 64 parts (Section 2.1), bit-exact;
  * the local solves A_i^{-1} R_i r of three sampled parts (smallest, median, largest) by
    sparse LU, on the dofs that only that part covers (there the local branch equals the
    part's own solve); FP32 factors, so the tolerance is the FP32 one (1e-4 relative);
  * the FGMRES solution's true FP64 relative residual with the oracle's matrix <= 1e-8.
"""
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


def test_channel32_full_size(lib):
    from oracle import fem, gdsw as og
    p = I.channel(32)
    S = fem.assemble(p)
    A = S["A"]
    ctx = lib.Context(p, precision=("fp32",) * 3, phi_precision="fp32", tol=1e-8)
    n = ctx.n
    assert n == A.shape[0]
    Ag = ctx.gdsw_matrix_csr()
    assert abs(Ag - A).max() <= 1e-14 * abs(A).max()
    rng = np.random.default_rng(0)
    x = rng.standard_normal(n)
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    ctx.gdsw_spmv(torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    assert np.linalg.norm(y.cpu().numpy() - A @ x) <= 1e-14 * np.linalg.norm(A @ x)
    # overlapping index sets, all parts
    od = og.overlapping_dofs(S, p)
    gd = ctx.gdsw_level_dofs(0)
    assert len(od) == len(gd) and all(np.array_equal(a, b) for a, b in zip(od, gd))
    # sampled local solves on exclusively covered dofs
    mult = np.zeros(n, dtype=int)
    for d in od:
        mult[d] += 1
    r = rng.standard_normal(n)
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    ctx.gdsw_apply_local(0, torch.from_numpy(r).cuda(), z)
    torch.cuda.synchronize()
    z = z.cpu().numpy()
    sizes = np.array([d.size for d in od])
    for i in (int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2]), int(np.argmax(sizes))):
        d = od[i]
        zi = spla.splu(A[d][:, d].tocsc()).solve(r[d])
        own = mult[d] == 1
        assert own.sum() > 0
        err = np.linalg.norm(z[d][own] - zi[own]) / np.linalg.norm(zi[own])
        assert err <= 1e-4, (i, err)
    # full solve: true residual with the oracle's operator and right-hand side
    b = fem.lifted_rhs(S)
    xs = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = ctx.gdsw_solve(torch.from_numpy(b).cuda(), xs)
    torch.cuda.synchronize()
    xs = xs.cpu().numpy()
    assert info.status == 0
    assert np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1e-8
    ctx.close()
