"""Writes channel32_oracle.json: the FP64 oracle's GDSW-FGMRES iteration count and final
true relative residual on the benchmark workload (32^3 Carreau channel with four cylinders,
4x4x4 parts grouped 2x2x2, three levels, PoU weighting, restart 100, tolerance 1e-8,
right-hand side = the lifted inflow).  It calls oracle/ only (on a pool of all host cores,
whose results equal the serial oracle's), never the library.

  python tests/golden/make_channel32_oracle.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


def main():
    from oracle import fem, fgmres, gdsw as og
    from oracle.parallel import HostPool
    from paper_2606_01433_gb300 import inputs as I
    p = I.channel(32)
    t0 = time.perf_counter()
    with HostPool() as pool:
        S = fem.assemble(p, pool=pool)
        P = og.GDSW(S, p, pool=pool)
        b = fem.lifted_rhs(S)
        x, info = fgmres.fgmres(lambda v: pool.matvec(S["A"], v), b, P.apply, tol=1e-8, restart=100, max_it=1000)
    out = {"workload": p.name, "n": int(S["A"].shape[0]), "levels": 3, "weighting": "pou", "restart": 100,
           "tol": 1e-8, "iterations": int(info["iterations"]), "relres": float(info["relres"]),
           "coarse_dims": [int(lev.n0) for lev in P.levels],
           "written_by": "tests/golden/make_channel32_oracle.py (oracle only)",
           "wall_s": round(time.perf_counter() - t0, 1)}
    with open(os.path.join(HERE, "channel32_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
