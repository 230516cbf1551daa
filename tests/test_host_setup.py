"""CPU tests of the library's host logic (no GPU): the C ABI library loads and exports
every declared entry point, and its symbolic set-up (gdsw_analyze: dof numbering,
overlapping subdomains, interface entities, coarse sizes on every level) produces exactly
the index sets of the FP64 oracle (Section 2.1 / 2.2)."""
import numpy as np
import pytest

from paper_2606_01433_gb300 import inputs as I


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_01433_gb300 import gdsw
    return gdsw


def test_exports_every_declared_symbol(lib):
    L = lib.load()
    names = lib.declared_symbols()
    assert len(names) >= 20
    missing = [s for s in names if not hasattr(L, s)]
    assert not missing, missing


def _p1disc(p):
    p.pressure = "p1disc"
    return p


def test_launch_overlap_switch(lib):
    """gdsw_set_launch_overlap takes 0 or 1 (a process-wide flag; no device work) and rejects
    anything else."""
    L = lib.load()
    assert L.gdsw_set_launch_overlap(5) == 1        # GDSW_ERR_INVALID_ARG
    assert L.gdsw_set_launch_overlap(0) == 0
    assert L.gdsw_set_launch_overlap(1) == 0


CASES = [
    ("cube8_2x2x2", lambda: I.unit_cube(8)),
    ("box_3lvl", lambda: I.box_problem(4, 4, 4, (2, 2, 2), groups=((2, 2, 1),), levels=3)),
    ("box_4lvl", lambda: I.box_problem(4, 4, 2, (4, 4, 2), groups=((2, 2, 1), (2, 1, 1)), levels=4)),
    ("channel16_obstacles", lambda: I.channel(16, parts=(4, 4, 4), groups=((2, 2, 2),), levels=3)),
    ("die_rcb", lambda: I.die(16, 16, 32, nparts=16, per_group=4, levels=3)),
    # Q2 / P1-disc (two levels): element pressure sets and per-subdomain pressure columns
    ("cube6_p1disc", lambda: _p1disc(I.unit_cube(6, parts=(2, 2, 2)))),
    ("channel12_p1disc", lambda: _p1disc(I.channel(12, parts=(3, 3, 3), groups=(), levels=2))),
    ("die_rcb_p1disc", lambda: _p1disc(I.die(16, 16, 32, nparts=16, per_group=4, levels=2))),
    ("box_4lvl_p1disc", lambda: _p1disc(I.box_problem(4, 4, 2, (4, 4, 2), groups=((2, 2, 1), (2, 1, 1)), levels=4))),
    ("channel12_p1disc_3lvl", lambda: _p1disc(I.channel(12, parts=(4, 4, 4), groups=((2, 2, 2),), levels=3))),
    ("die_rcb_p1disc_4lvl", lambda: _p1disc(I.die(16, 16, 32, nparts=32, per_group=4, levels=4))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_symbolic_setup_matches_oracle(lib, name, make):
    from oracle import fem, gdsw as og
    p = make()
    ctx = lib.Context(p, analyze_only=True)
    S = fem.assemble(p)
    mesh = S["mesh"]
    assert ctx.sizes.n == S["A"].shape[0]
    assert ctx.sizes.n_u == mesh.nu and ctx.sizes.n_p == mesh.np_
    P = og.GDSW(S, p)
    assert all(np.array_equal(a, b) for a, b in zip(og.overlapping_dofs(S, p), P.levels[0].dofs))
    for l, lev in enumerate(P.levels):
        mine = ctx.gdsw_level_dofs(l)
        assert len(mine) == len(lev.dofs)
        for a, b in zip(mine, lev.dofs):
            assert np.array_equal(a, b)
        assert ctx.gdsw_level_entities(l) == len(lev.entities)
        assert ctx.sizes.n_coarse[l] == lev.n0
    assert ctx.sizes.device_bytes > 0
    ctx.close()
