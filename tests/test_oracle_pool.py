"""The host pool of the oracle (oracle/parallel.py) runs the oracle's own units on several
cores and combines them in the serial order: a pooled assembly, preconditioner apply, SpMV
and FGMRES solve equal the serial oracle's (checked bit for bit on a three-level box)."""
import numpy as np

from paper_2606_01433_gb300 import inputs as I
from oracle import fem, fgmres, gdsw
from oracle.parallel import HostPool


def test_pool_equals_serial():
    p = I.box_problem(6, 6, 6, (3, 3, 2), groups=((3, 3, 1),), levels=3, form="symmetric", uk_seed=3, lam=1.0,
                      n=0.5, nu_inf=1e-3)
    with HostPool(3) as pool:
        S1, S2 = fem.assemble(p), fem.assemble(p, pool=pool)
        assert (S1["A"] != S2["A"]).nnz == 0
        P1, P2 = gdsw.GDSW(S1, p), gdsw.GDSW(S2, p, pool=pool)
        r = np.random.default_rng(0).standard_normal(S1["A"].shape[0])
        assert np.array_equal(P1.apply(r), P2.apply(r))
        assert np.array_equal(pool.matvec(S1["A"], r), S1["A"] @ r)
        x1, i1 = fgmres.fgmres(lambda v: S1["A"] @ v, r, P1.apply, tol=1e-10)
        x2, i2 = fgmres.fgmres(lambda v: pool.matvec(S2["A"], v), r, P2.apply, tol=1e-10)
        assert i1["iterations"] == i2["iterations"] and np.array_equal(x1, x2)
