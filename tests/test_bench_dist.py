"""The N > 1 path of bench.py on CPU: two ranks over gloo (127.0.0.1), as torchrun would start
them.  The job time is the maximum over ranks (replicas: the slowest defines it), the barrier
brackets the timed region, and the reference arm is run and printed by rank 0 alone while the
other ranks exit without work."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), GDSW_BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    r, w, _ = bench.dist_init()
    slowest = bench.allreduce_max(10.0 * (rank + 1), w)
    bench.barrier(w)
    stub = {"ms": 123.0, "cores": 1, "iterations": 3, "relres": 1e-9, "assembly_s": 0.1, "setup_s": 0.1,
            "full_solve_s": 0.1, "krylov_rest_s": 0.0, "apply_s_mean": 0.01, "spmv_s_mean": 0.01,
            "sample_wall_s": 0.1}
    bench.oracle_reference = lambda p, steps, warmup: stub  # the oracle itself is not timed here

    class Args:
        m, warmup, steps, gpus = 8, 0, 2, world
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(Args, r, w)
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((rank, r, w, slowest, buf.getvalue()))


def test_two_rank_replicas_over_gloo():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, r, w, slowest, text = q.get(timeout=180)
        out[rank] = (r, w, slowest, text)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][:3] == (0, 2, 20.0) and out[1][:3] == (1, 2, 20.0)
    assert out[1][3] == ""  # rank 1 runs no reference work and prints nothing
    lines = [json.loads(x) for x in out[0][3].splitlines() if x.startswith("{")]
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["value"] == 123.0
    assert lines[0]["e2e"] == {"value": 123.0, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
