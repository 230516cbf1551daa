"""gdsw_apply_local_noalloc: the local branch of a level computed without allocating memory
(for callers that cannot call cudaMalloc while they run, e.g. a process whose device memory is
all pre-reserved by its own pool, or a latency-critical loop that cannot take the device-wide
synchronisation of a cudaFree).  Its result must equal
gdsw_apply_local's, call after call, since the two run the same kernels in the same order;
only the scratch differs (a fixed device array instead of the context's workspace), so the two
results are compared for exact equality.

This file is named so that pytest collects it last; it must pass in a fresh process as well
as after the other tests.
"""
import numpy as np
import pytest

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_noalloc_matches_apply_local(lib, prec):
    """Every Schwarz level of a three-level context, in each local precision: the no-alloc
    call returns exactly gdsw_apply_local's result, on two calls in a row."""
    p = I.box_problem(4, 4, 4, (2, 2, 2), groups=((2, 2, 1),), levels=3, form="symmetric", uk_seed=3, lam=1.0,
                      n=0.5, nu_inf=1e-3)
    ctx = lib.Context(p, precision=(prec, prec, prec), phi_precision="fp64" if prec == "fp64" else "fp32")
    rng = np.random.default_rng(7)
    sizes = [ctx.n] + [int(v) for v in list(ctx.sizes.n_coarse)[:ctx.sizes.levels - 2]]
    assert len(sizes) == 2
    for level, n in enumerate(sizes):
        for call in range(2):  # two calls in a row: the shared scratch keeps the previous contents
            r = torch.from_numpy(rng.standard_normal(n)).cuda()
            z_ref = torch.zeros_like(r)
            z_new = torch.full_like(r, float("nan"))
            ctx.gdsw_apply_local(level, r, z_ref)
            ctx.gdsw_apply_local_noalloc(level, r, z_new)
            torch.cuda.synchronize()
            a, b = z_new.cpu().numpy(), z_ref.cpu().numpy()
            assert np.all(np.isfinite(a)) and np.any(a != 0.0)
            assert np.array_equal(a, b), (level, call, rel(a, b))
    ctx.close()


def test_noalloc_rejects_oversized_level(lib):
    p = I.channel(24)
    ctx = lib.Context(p, precision=("fp64", "fp64", "fp64"))
    r = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    with pytest.raises(lib.GdswError) as e:
        ctx.gdsw_apply_local_noalloc(0, r, z)
    assert e.value.code == lib.GDSW_ERR_INVALID_ARG
    assert "scratch" in str(e.value)
    ctx.close()
