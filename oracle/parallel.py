"""Host-core execution of the oracle's independent work units.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The oracle's arithmetic is unchanged by this module.  The units are the ones the serial
code runs one after another -- element chunks of the assembly and their pairwise sums, the
factorisation and the solve of each overlapping subdomain (Section 2.1), the interior
solves of the coarse basis (Section 2.1, discrete saddle-point extension), row blocks of
sparse products -- and the caller combines their results in the serial order, so a pooled
oracle returns the serial oracle's numbers.

Threads run the units whose library routines release the interpreter lock (NumPy, SciPy
sparse products and SuperLU solves).  SuperLU factorisations hold it, so every subdomain's
factor lives in one of a set of worker processes (started with 'spawn', never forked), which
also runs the solves with it; the operator reaches the workers through shared memory.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ThreadPoolExecutor
from multiprocessing import shared_memory

import numpy as np
import scipy.sparse as sp


def host_cores() -> int:
    return len(os.sched_getaffinity(0))


# ----------------------------------------------------------------------------- worker side
def _attach(spec, keep):
    # spawned workers share the creating process's resource tracker, which unlinks the
    # segment once, when the pool releases it
    shm = shared_memory.SharedMemory(name=spec[0])
    keep.append(shm)
    return np.ndarray((spec[2],), dtype=np.dtype(spec[1]), buffer=shm.buf)


def _worker(conn):
    from oracle.gdsw import LocalSolver      # the oracle's own local solver
    keep, mats, vecs, solvers = [], {}, {}, {}
    while True:
        msg = conn.recv()
        op = msg[0]
        try:
            if op == "stop":
                conn.send(("ok", None))
                break
            if op == "csr":
                _, name, specs, shape = msg
                data, indices, indptr = (_attach(s, keep) for s in specs)
                mats[name] = sp.csr_matrix((data, indices, indptr), shape=shape, copy=False)
                conn.send(("ok", None))
            elif op == "vec":
                _, name, spec = msg
                vecs[name] = _attach(spec, keep)
                conn.send(("ok", None))
            elif op == "factor":
                _, key, name, items = msg
                A = mats[name]
                for i, d in items:
                    solvers[(key, i)] = (d, LocalSolver(A[d][:, d]))
                conn.send(("ok", None))
            elif op == "solve":
                _, key, vname, ids = msg
                r = vecs[vname]
                conn.send(("ok", [(i, solvers[(key, i)][1].solve(r[solvers[(key, i)][0]])) for i in ids]))
            elif op == "extend":
                _, name, items = msg
                A = mats[name]
                out = []
                for i, I, rhs in items:
                    out.append((i, LocalSolver(A[I][:, I]).solve(rhs)))
                conn.send(("ok", out))
            elif op == "drop":
                _, key = msg
                for k in [k for k in solvers if k[0] == key]:
                    del solvers[k]
                conn.send(("ok", None))
            else:
                conn.send(("err", "unknown op %r" % (op,)))
        except Exception as e:          # report, keep serving
            conn.send(("err", "%s: %s" % (type(e).__name__, e)))


# ----------------------------------------------------------------------------- main side
class HostPool:
    """A pool of `workers` processes (subdomain factors and solves) and as many threads
    (products, assembly chunks).  `cores` is the number of host threads it uses."""

    def __init__(self, workers: int | None = None):
        self.cores = int(workers or host_cores())
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for _ in range(self.cores):
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_worker, args=(b,), daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        self.threads = ThreadPoolExecutor(self.cores)
        self.shm = {}          # name -> list of SharedMemory
        self.views = {}        # name -> (arrays...)
        self.owner = {}        # (key, i) -> worker index
        self.shapes = {}       # name -> (shape, nnz)
        self.vec_for = {}      # factor key -> shared right-hand-side vector
        self.count = {}        # factor key -> number of subdomains
        self.blocks = {}       # id(matrix) -> (matrix, its row blocks)

    # ---- plumbing
    def _ask(self, w, msg):
        self.conns[w].send(msg)

    def _get(self, w):
        st, val = self.conns[w].recv()
        if st != "ok":
            raise RuntimeError("oracle worker %d: %s" % (w, val))
        return val

    def _all(self, msg):
        for w in range(self.cores):
            self._ask(w, msg)
        return [self._get(w) for w in range(self.cores)]

    def _new(self, arr):
        arr = np.ascontiguousarray(arr)
        shm = shared_memory.SharedMemory(create=True, size=max(arr.nbytes, 1))
        view = np.ndarray(arr.shape, dtype=arr.dtype, buffer=shm.buf)
        view[...] = arr
        return shm, view, (shm.name, arr.dtype.str, arr.size)

    def share_csr(self, name, M):
        """Place a CSR matrix in shared memory (or overwrite its values when the same
        sparsity pattern is shared again under the same name)."""
        M = sp.csr_matrix(M)
        if name in self.views and self.shapes[name] == (M.shape, M.nnz) and \
                np.array_equal(self.views[name][1], M.indices) and np.array_equal(self.views[name][2], M.indptr):
            self.views[name][0][...] = M.data
            return
        self.release(name)
        parts = [self._new(a) for a in (M.data, M.indices, M.indptr)]
        self.shm[name] = [p[0] for p in parts]
        self.views[name] = [p[1] for p in parts]
        self.shapes[name] = (M.shape, M.nnz)
        self._all(("csr", name, [p[2] for p in parts], M.shape))

    def share_vec(self, name, n):
        """A shared FP64 vector of length n; returns the writable main-side view."""
        if name in self.views and self.views[name][0].size == n:
            return self.views[name][0]
        self.release(name)
        shm, view, spec = self._new(np.zeros(n))
        self.shm[name] = [shm]
        self.views[name] = [view]
        self._all(("vec", name, spec))
        return view

    def release(self, name):
        for s in self.shm.pop(name, []):
            s.close()
            s.unlink()
        self.views.pop(name, None)

    # ---- subdomain factors (Section 2.1 local solvers A_i^{-1})
    def factor(self, key, name, dofs):
        """Factor A[d][:, d] of every dof list with the oracle's LocalSolver, each in one
        worker (largest first onto the least loaded worker)."""
        load = np.zeros(self.cores)
        items = [[] for _ in range(self.cores)]
        for i in np.argsort([-len(d) for d in dofs], kind="stable"):
            w = int(np.argmin(load))
            load[w] += float(len(dofs[i])) ** 2
            items[w].append((int(i), dofs[i]))
            self.owner[(key, int(i))] = w
        for w in range(self.cores):
            self._ask(w, ("factor", key, name, items[w]))
        for w in range(self.cores):
            self._get(w)
        self.vec_for[key] = self.share_vec("r:" + key, self.shapes[name][0][0])
        self.count[key] = len(dofs)

    def solve(self, key, r):
        """[A_i^{-1} r[d_i] for every factored subdomain i], in subdomain order."""
        self.vec_for[key][...] = r
        ids = [[] for _ in range(self.cores)]
        for i in range(self.count[key]):
            ids[self.owner[(key, i)]].append(i)
        busy = [w for w in range(self.cores) if ids[w]]
        for w in busy:
            self._ask(w, ("solve", key, "r:" + key, ids[w]))
        out = [None] * self.count[key]
        for w in busy:
            for i, z in self._get(w):
                out[i] = z
        return out

    def drop(self, key):
        self._all(("drop", key))

    def extend(self, name, blocks):
        """For blocks [(I, rhs)], LocalSolver(A[I][:, I]).solve(rhs) of each (Section 2.1
        interior solves of the coarse basis), spread over the workers; results in order."""
        load = np.zeros(self.cores)
        items = [[] for _ in range(self.cores)]
        for i in np.argsort([-len(b[0]) for b in blocks], kind="stable"):
            w = int(np.argmin(load))
            load[w] += float(len(blocks[i][0])) ** 2
            items[w].append((int(i), blocks[i][0], blocks[i][1]))
        busy = [w for w in range(self.cores) if items[w]]
        for w in busy:
            self._ask(w, ("extend", name, items[w]))
        out = [None] * len(blocks)
        for w in busy:
            for i, X in self._get(w):
                out[i] = X
        return out

    # ---- threads
    def map(self, fn, items):
        return list(self.threads.map(fn, items))

    def matvec(self, M, x):
        """M @ x by row blocks on the threads; every row is summed exactly as in the serial
        product, so the result is the serial one.  The row blocks of a matrix are cut once
        and kept while the matrix object is alive in the pool's cache."""
        n = M.shape[0]
        y = np.empty(n, dtype=np.result_type(M.dtype, x.dtype))

        def run(blk):
            a, b, Mb = blk
            y[a:b] = Mb @ x
        self.map(run, self._row_blocks(M))
        return y

    def row_product(self, M, B):
        """The sparse product M @ B by row blocks of M on the threads (each row of the result
        is formed as in the serial product), stacked back in row order."""
        blocks = self._row_blocks(M)
        parts = self.map(lambda blk: blk[2] @ B, blocks)
        return sp.vstack(parts, format="csr")

    def _row_blocks(self, M):
        cache = self.blocks
        hit = cache.get(id(M))
        if hit is not None and hit[0] is M:
            return hit[1]
        n = M.shape[0]
        nb = min(self.cores * 4, max(n // 4096, 1))
        cuts = np.searchsorted(M.indptr, np.linspace(0, M.nnz, nb + 1)).clip(0, n)
        cuts[0], cuts[-1] = 0, n
        blocks = [(int(a), int(b), M[int(a):int(b)]) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
        if len(cache) >= 8:
            cache.clear()
        cache[id(M)] = (M, blocks)
        return blocks

    def close(self):
        try:
            self._all(("stop",))
        except Exception:
            pass
        for pr in self.procs:
            pr.join(timeout=10)
        for name in list(self.shm):
            self.release(name)
        self.threads.shutdown()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
