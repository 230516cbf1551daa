"""Thin ctypes binding of libgdsw.so (C ABI declared in include/gdsw.h).

Argument marshalling only: every numeric step runs inside the CUDA library.  Device
vectors are passed as torch CUDA tensors (float64, contiguous); their data pointers go
straight to the library, which works on the current torch stream.  If the library has not
been built, load() raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgdsw.so")

GDSW_OK, GDSW_ERR_INVALID_ARG, GDSW_ERR_OOM, GDSW_ERR_SINGULAR = 0, 1, 2, 3
GDSW_ERR_NOT_CONVERGED, GDSW_ERR_NAN, GDSW_ERR_TIMEOUT, GDSW_ERR_CUDA = 4, 5, 6, 7
FP64, FP32, BF16 = 0, 1, 2
WEIGHT_POU, WEIGHT_PLAIN = 0, 1
FORM = {"gradient": 0, "symmetric": 1}
PREC = {"fp64": FP64, "fp32": FP32, "bf16": BF16}
KERNEL_GROUPS = ["spmv", "gather", "local", "scatter", "restrict", "coarse", "prolong", "arnoldi",
                 "apply", "assembly", "viscosity", "other"]


class GdswError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("gdsw error %d: %s" % (code, msg))
        self.code = code


class gdsw_mesh(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("h", C.c_double),
                ("origin", C.c_double * 3), ("mask", C.c_void_p), ("tags", C.c_void_p), ("g", C.c_void_p),
                ("pressure", C.c_int32)]


PRESSURE = {"q1": 0, "p1disc": 1}


class gdsw_viscosity(C.Structure):
    _fields_ = [("form", C.c_int32), ("nu0", C.c_double), ("nu_inf", C.c_double), ("lambda_", C.c_double),
                ("n", C.c_double), ("uk", C.c_void_p)]


class gdsw_partition(C.Structure):
    _fields_ = [("elem_part", C.c_void_p), ("n_groups", C.c_int32), ("groups", C.c_void_p * 2),
                ("group_len", C.c_int32 * 2)]


class gdsw_levels(C.Structure):
    _fields_ = [("levels", C.c_int32), ("overlap", C.c_int32), ("rotations", C.c_int32)]


class gdsw_options(C.Structure):
    _fields_ = [("weighting", C.c_int32), ("precision", C.c_int32 * 3), ("phi_precision", C.c_int32),
                ("restart", C.c_int32), ("max_it", C.c_int32), ("tol", C.c_double), ("slab_elems", C.c_int32),
                ("use_graph", C.c_int32), ("stream", C.c_void_p)]


class gdsw_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("status", C.c_int32), ("relres", C.c_double),
                ("est_relres", C.c_double), ("time_ms", C.c_double), ("apply_ms", C.c_double),
                ("spmv_ms", C.c_double), ("arnoldi_ms", C.c_double)]


class gdsw_sizes_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_u", C.c_int64), ("n_p", C.c_int64), ("n_elems", C.c_int64),
                ("n_nodes", C.c_int64), ("levels", C.c_int32), ("n_coarse", C.c_int64 * 4),
                ("n_parts", C.c_int32 * 3), ("local_dofs", C.c_int64 * 3), ("factor_entries", C.c_int64 * 3),
                ("max_local", C.c_int64 * 3), ("max_slabs", C.c_int32), ("nnzb_A", C.c_int64),
                ("nnz_B", C.c_int64), ("phi_entries", C.c_int64), ("device_bytes", C.c_int64),
                ("setup_ms", C.c_double * 6), ("tile_rows", C.c_int32 * 3), ("persistent", C.c_int32 * 3),
                ("tuned_ms", C.c_double * 3)]


class gdsw_gemm_task(C.Structure):
    _fields_ = [("a", C.c_void_p), ("b", C.c_void_p), ("c", C.c_void_p), ("M", C.c_int32), ("N", C.c_int32),
                ("K", C.c_int32), ("lda", C.c_int32), ("ldb", C.c_int32), ("ldc", C.c_int32),
                ("trans_a", C.c_int32), ("trans_b", C.c_int32), ("alpha", C.c_double), ("beta", C.c_double)]


GEMM_ENGINE = {"auto": 0, "simt": 1, "tensor": 2}


class gdsw_mg_options(C.Structure):
    _fields_ = [("omega", C.c_double), ("pre", C.c_int32), ("post", C.c_int32), ("smoother_precision", C.c_int32),
                ("symmetric", C.c_int32)]


class gdsw_profile(C.Structure):
    _fields_ = [("enabled", C.c_int32), ("calls", C.c_int64 * 12), ("ms", C.c_double * 12),
                ("bytes", C.c_double * 12)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libgdsw.so; raises if it is missing (build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libgdsw.so is not built (%s); run __graft_entry__.build()" % path)
    lib = C.CDLL(path)
    vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.c_void_p
    sig = {
        "gdsw_setup": ([C.POINTER(gdsw_mesh), C.POINTER(gdsw_viscosity), C.POINTER(gdsw_partition),
                        C.POINTER(gdsw_levels), C.POINTER(gdsw_options), C.POINTER(vp)], C.c_int),
        "gdsw_analyze": ([C.POINTER(gdsw_mesh), C.POINTER(gdsw_viscosity), C.POINTER(gdsw_partition),
                          C.POINTER(gdsw_levels), C.POINTER(gdsw_options), C.POINTER(vp)], C.c_int),
        "gdsw_destroy": ([vp], None),
        "gdsw_last_error": ([vp], C.c_char_p),
        "gdsw_sizes": ([vp, C.POINTER(gdsw_sizes_info)], C.c_int),
        "gdsw_rhs_lift": ([vp, dp], C.c_int),
        "gdsw_spmv": ([vp, dp, dp], C.c_int),
        "gdsw_apply": ([vp, dp, dp], C.c_int),
        "gdsw_solve": ([vp, dp, dp, C.POINTER(gdsw_solve_info)], C.c_int),
        "gdsw_solve_host": ([vp, dp, dp, C.POINTER(gdsw_solve_info)], C.c_int),
        "gdsw_reassemble": ([vp, dp], C.c_int),
        "gdsw_apply_local": ([vp, i32, dp, dp], C.c_int),
        "gdsw_apply_local_noalloc": ([vp, i32, dp, dp], C.c_int),
        "gdsw_restrict": ([vp, i32, dp, dp], C.c_int),
        "gdsw_prolong": ([vp, i32, dp, dp], C.c_int),
        "gdsw_coarse_matrix": ([vp, i32, dp], C.c_int),
        "gdsw_matrix_csr": ([vp, dp, dp, dp, C.POINTER(i64)], C.c_int),
        "gdsw_viscosity_values": ([vp, dp], C.c_int),
        "gdsw_level_dofs": ([vp, i32, dp, dp], C.c_int),
        "gdsw_level_entities": ([vp, i32, C.POINTER(i32)], C.c_int),
        "gdsw_kernel_launches": ([], i64),
        "gdsw_probe_fma": ([i32, C.POINTER(C.c_double)], C.c_int),
        "gdsw_gemm_f32": ([C.POINTER(gdsw_gemm_task), i32, i32], C.c_int),
        "gdsw_mg_create": ([C.POINTER(vp), i32, C.POINTER(gdsw_mg_options), C.POINTER(vp)], C.c_int),
        "gdsw_mg_destroy": ([vp], None),
        "gdsw_mg_last_error": ([vp], C.c_char_p),
        "gdsw_mg_vcycle": ([vp, dp, dp], C.c_int),
        "gdsw_mg_smooth": ([vp, i32, dp, dp, i32], C.c_int),
        "gdsw_mg_prolong": ([vp, i32, dp, dp], C.c_int),
        "gdsw_mg_restrict": ([vp, i32, dp, dp], C.c_int),
        "gdsw_mg_stats": ([vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)], C.c_int),
        "gdsw_set_gemm_engine": ([i32], C.c_int),
        "gdsw_set_launch_overlap": ([i32], C.c_int),
        "gdsw_plan_bytes": ([vp, i32, i32, i32, C.POINTER(C.c_double)], C.c_int),
        "gdsw_set_local_sweep": ([vp, i32, i32, i32], C.c_int),
        "gdsw_picard_update": ([vp, vp], C.c_int),
        "gdsw_residual": ([vp, dp, dp, dp], C.c_int),
        "gdsw_newton_step": ([vp, dp, C.POINTER(gdsw_solve_info)], C.c_int),
        "gdsw_sweep_wait_selftest": ([vp], C.c_int),
        "gdsw_profile_enable": ([vp, i32], C.c_int),
        "gdsw_profile_read": ([vp, C.POINTER(gdsw_profile)], C.c_int),
        "gdsw_profile_reset": ([vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def probe_fma(precision="fp64"):
    """FMA throughput of the current device in TFLOP/s (gdsw_probe_fma)."""
    lib = load()
    t = C.c_double()
    rc = lib.gdsw_probe_fma(PREC[precision], C.byref(t))
    if rc != GDSW_OK:
        raise GdswError(rc, "gdsw_probe_fma failed")
    return t.value


def gemm_f32(tasks, engine="tensor"):
    """Batched FP32 GEMM (gdsw_gemm_f32): tasks = [(A, B, C, trans_a, trans_b, alpha, beta)]
    with contiguous float32 CUDA tensors; C = alpha op(A) op(B) + beta C in place."""
    import torch
    lib = load()
    arr = (gdsw_gemm_task * max(len(tasks), 1))()
    for i, (A, B, Cm, ta, tb, alpha, beta) in enumerate(tasks):
        for t in (A, B, Cm):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise TypeError("expected contiguous float32 CUDA tensors")
        M, K = (A.shape[1], A.shape[0]) if ta else (A.shape[0], A.shape[1])
        N = B.shape[0] if tb else B.shape[1]
        arr[i] = gdsw_gemm_task(A.data_ptr(), B.data_ptr(), Cm.data_ptr(), M, N, K, A.shape[1], B.shape[1],
                                Cm.shape[1], int(ta), int(tb), float(alpha), float(beta))
    rc = lib.gdsw_gemm_f32(arr, len(tasks), GEMM_ENGINE[engine])
    if rc != GDSW_OK:
        raise GdswError(rc, "gdsw_gemm_f32 failed")


def set_launch_overlap(on=True):
    """Overlapped (programmatic dependent) launch chain of the local sweeps, process-wide."""
    rc = load().gdsw_set_launch_overlap(1 if on else 0)
    if rc != GDSW_OK:
        raise GdswError(rc, "gdsw_set_launch_overlap failed")


def set_gemm_engine(engine):
    rc = load().gdsw_set_gemm_engine(GEMM_ENGINE[engine])
    if rc != GDSW_OK:
        raise GdswError(rc, "gdsw_set_gemm_engine failed")


def declared_symbols():
    """Function names declared in include/gdsw.h (for the export check)."""
    import re
    hdr = open(os.path.join(os.path.dirname(HERE), "include", "gdsw.h")).read()
    return sorted(set(re.findall(r"\b(gdsw_[a-z0-9_]+)\s*\(", hdr)))


def _ptr(t):
    """Device pointer of a contiguous float64 CUDA tensor."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Context:
    """One preconditioner/solver context (gdsw_ctx*)."""

    def __init__(self, prob, levels=None, weighting="pou", precision=("fp64", "fp64", "fp64"),
                 phi_precision="fp64", restart=100, max_it=1000, tol=1e-8, slab_elems=1, use_graph=False,
                 overlap=1, stream=None, analyze_only=False, rotations=False):
        lib = load()
        self.lib = lib
        self.prob = prob
        L = prob.levels if levels is None else levels
        self._keep = []
        mask = _np(prob.mask, np.uint8)
        tags = _np(prob.tags, np.uint8)
        g = _np(prob.g, np.float64)
        part = _np(prob.part, np.int32)
        self._keep += [mask, tags, g, part]
        m = gdsw_mesh(prob.nx, prob.ny, prob.nz, prob.h, (C.c_double * 3)(*prob.origin),
                      mask.ctypes.data, tags.ctypes.data, g.ctypes.data, PRESSURE[prob.pressure])
        uk = None
        if prob.uk is not None:
            uk = _np(prob.uk, np.float64)
            self._keep.append(uk)
        v = gdsw_viscosity(FORM[prob.form], prob.nu0, prob.nu_inf, prob.lam, prob.n_carreau,
                           uk.ctypes.data if uk is not None else None)
        pa = gdsw_partition()
        pa.elem_part = part.ctypes.data
        pa.n_groups = max(L - 2, 0)     # levels = 1: operator only (no Schwarz levels)
        for l in range(L - 2):
            gr = _np(prob.groups[l], np.int32)
            self._keep.append(gr)
            pa.groups[l] = gr.ctypes.data
            pa.group_len[l] = gr.size
        lv = gdsw_levels(L, overlap, 1 if rotations else 0)
        if stream is None and not analyze_only:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
            except Exception:
                stream = None
        prec = [PREC[p] if isinstance(p, str) else int(p) for p in precision]
        prec = (prec + [prec[-1]] * 3)[:3]
        o = gdsw_options(WEIGHT_POU if weighting == "pou" else WEIGHT_PLAIN, (C.c_int32 * 3)(*prec),
                         PREC[phi_precision], restart, max_it, tol, slab_elems, 1 if use_graph else 0, stream)
        self.stream = stream
        h = C.c_void_p()
        entry = lib.gdsw_analyze if analyze_only else lib.gdsw_setup
        rc = entry(C.byref(m), C.byref(v), C.byref(pa), C.byref(lv), C.byref(o), C.byref(h))
        if rc != GDSW_OK:
            raise GdswError(rc, lib.gdsw_last_error(None).decode())
        self.h = h
        self._keep = None
        si = gdsw_sizes_info()
        lib.gdsw_sizes(h, C.byref(si))
        self.sizes = si
        self.n = si.n

    def _check(self, rc):
        if rc not in (GDSW_OK, GDSW_ERR_NOT_CONVERGED):
            raise GdswError(rc, self.lib.gdsw_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.gdsw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- the C ABI, one method per entry point
    def gdsw_spmv(self, x, y):
        return self._check(self.lib.gdsw_spmv(self.h, _ptr(x), _ptr(y)))

    def gdsw_apply(self, r, z):
        return self._check(self.lib.gdsw_apply(self.h, _ptr(r), _ptr(z)))

    def gdsw_rhs_lift(self, b):
        return self._check(self.lib.gdsw_rhs_lift(self.h, _ptr(b)))

    def gdsw_solve(self, b, x):
        info = gdsw_solve_info()
        rc = self._check(self.lib.gdsw_solve(self.h, _ptr(b), _ptr(x), C.byref(info)))
        return info

    def gdsw_solve_host(self, b, x):
        """b, x: numpy float64 arrays (x holds the initial guess and receives the result)."""
        assert b.dtype == np.float64 and x.dtype == np.float64 and b.flags.c_contiguous and x.flags.c_contiguous
        info = gdsw_solve_info()
        self._check(self.lib.gdsw_solve_host(self.h, b.ctypes.data, x.ctypes.data, C.byref(info)))
        return info

    def gdsw_reassemble(self, uk=None):
        if uk is None:
            return self._check(self.lib.gdsw_reassemble(self.h, None))
        u = _np(uk, np.float64)
        return self._check(self.lib.gdsw_reassemble(self.h, u.ctypes.data))

    def gdsw_sweep_wait_selftest(self):
        """Run the level-1 persistent sweep with one unreachable dependency (expects GDSW_ERR_TIMEOUT)."""
        return self._check(self.lib.gdsw_sweep_wait_selftest(self.h))

    def gdsw_picard_update(self, x):
        """u_k <- velocity of the device solution x (free nodes) and the Dirichlet data."""
        return self._check(self.lib.gdsw_picard_update(self.h, _ptr(x)))

    def picard_step(self, x, b):
        """One Section 3 Picard step with the frozen preconditioner of this context: re-evaluate
        nu(u_k) and re-assemble, lift the right-hand side into b, solve into x (warm start from
        the previous iterate), then take u_{k+1} from x.  x, b: device FP64 vectors of length n.
        Returns the solve's gdsw_solve_info."""
        self.gdsw_reassemble()
        self.gdsw_rhs_lift(b)
        info = self.gdsw_solve(b, x)
        self.gdsw_picard_update(x)
        return info

    def gdsw_residual(self, b, x, r):
        return self._check(self.lib.gdsw_residual(self.h, _ptr(b), _ptr(x), _ptr(r)))

    def newton_step(self, x):
        """One Section 3 Newton step from the state x (device FP64; u_k must be its velocity):
        gdsw_newton_step.  Returns the linear solve's gdsw_solve_info."""
        info = gdsw_solve_info()
        rc = self.lib.gdsw_newton_step(self.h, _ptr(x), C.byref(info))
        if rc not in (GDSW_OK, GDSW_ERR_NOT_CONVERGED):
            raise GdswError(rc, self.lib.gdsw_last_error(self.h).decode())
        return info

    def gdsw_apply_local(self, level, r, z):
        return self._check(self.lib.gdsw_apply_local(self.h, level, _ptr(r), _ptr(z)))

    def gdsw_apply_local_noalloc(self, level, r, z):
        """gdsw_apply_local without any allocation (fixed 4 MiB device scratch; see gdsw.h)."""
        return self._check(self.lib.gdsw_apply_local_noalloc(self.h, level, _ptr(r), _ptr(z)))

    def gdsw_restrict(self, level, r, r0):
        return self._check(self.lib.gdsw_restrict(self.h, level, _ptr(r), _ptr(r0)))

    def gdsw_prolong(self, level, x0, z):
        return self._check(self.lib.gdsw_prolong(self.h, level, _ptr(x0), _ptr(z)))

    def gdsw_coarse_matrix(self, l):
        """A_0^(l+2) as a dense host array (l = 0 .. L-2)."""
        n = int(self.sizes.n_coarse[l])
        out = np.zeros((n, n))
        self._check(self.lib.gdsw_coarse_matrix(self.h, l, out.ctypes.data))
        return out

    def gdsw_matrix_csr(self):
        import scipy.sparse as sp
        nnz = C.c_int64()
        self._check(self.lib.gdsw_matrix_csr(self.h, None, None, None, C.byref(nnz)))
        rp = np.zeros(self.n + 1, np.int64)
        col = np.zeros(nnz.value, np.int32)
        val = np.zeros(nnz.value)
        self._check(self.lib.gdsw_matrix_csr(self.h, rp.ctypes.data, col.ctypes.data, val.ctypes.data, C.byref(nnz)))
        return sp.csr_matrix((val, col, rp), shape=(self.n, self.n))

    def gdsw_viscosity_values(self):
        out = np.zeros((int(self.sizes.n_elems), 27))
        self._check(self.lib.gdsw_viscosity_values(self.h, out.ctypes.data))
        return out

    def gdsw_level_dofs(self, level):
        N = self.sizes.n_parts[level]
        off = np.zeros(N + 1, np.int64)
        self._check(self.lib.gdsw_level_dofs(self.h, level, off.ctypes.data, None))
        d = np.zeros(int(off[-1]), np.int32)
        self._check(self.lib.gdsw_level_dofs(self.h, level, off.ctypes.data, d.ctypes.data))
        return [d[off[i]:off[i + 1]] for i in range(N)]

    def gdsw_level_entities(self, level):
        n = C.c_int32()
        self._check(self.lib.gdsw_level_entities(self.h, level, C.byref(n)))
        return n.value

    def gdsw_set_local_sweep(self, persistent=True, ctas_per_sm=0, tile_rows=0):
        """Override the set-up autotuner: local solves as one persistent launch per level or one
        launch per slab step, and rows per forward tile (32/64/128; 0 keeps the current)."""
        return self._check(self.lib.gdsw_set_local_sweep(self.h, 1 if persistent else 0, int(ctas_per_sm),
                                                         int(tile_rows)))

    def gdsw_profile_enable(self, on=True):
        """on: False/0 = off, True/1 = time every apply, k > 1 = every k-th apply."""
        v = (1 if on else 0) if isinstance(on, bool) else int(on)
        return self._check(self.lib.gdsw_profile_enable(self.h, v))

    def gdsw_profile_reset(self):
        return self._check(self.lib.gdsw_profile_reset(self.h))

    def gdsw_profile_read(self):
        p = gdsw_profile()
        self._check(self.lib.gdsw_profile_read(self.h, C.byref(p)))
        return {KERNEL_GROUPS[i]: dict(calls=p.calls[i], ms=p.ms[i], bytes=p.bytes[i]) for i in range(12)}


# ----------------------------------------------------------------------------- serving
class gdsw_request(C.Structure):
    _fields_ = [("mesh", gdsw_mesh), ("visc", gdsw_viscosity), ("part", gdsw_partition), ("levels", gdsw_levels),
                ("opt", gdsw_options), ("rhs", C.c_void_p), ("x", C.c_void_p), ("x_len", C.c_int64)]


class gdsw_request_status(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("iterations", C.c_int32), ("slot", C.c_int32),
                ("n", C.c_int64), ("est_bytes", C.c_int64), ("relres", C.c_double), ("queue_ms", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double), ("latency_ms", C.c_double)]


class gdsw_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("budget_bytes", C.c_int64), ("used_bytes", C.c_int64), ("peak_used_bytes", C.c_int64),
                ("running", C.c_int32), ("peak_running", C.c_int32)]


REQ_DONE, REQ_FAILED = 4, 5


def count_dofs(prob):
    """n of the free-dof vector by the convention of gdsw.h: 3 per fluid node that is not a
    wall/inflow node, plus one per fluid node with all-even indices (Q1 pressure)."""
    nx, ny, nz = prob.nx, prob.ny, prob.nz
    m = np.asarray(prob.mask, bool).reshape(nz, ny, nx)
    act = np.zeros((2 * nz + 1, 2 * ny + 1, 2 * nx + 1), bool)
    for c in range(3):
        for b in range(3):
            for a in range(3):
                act[c:c + 2 * nz:2, b:b + 2 * ny:2, a:a + 2 * nx:2] |= m
    act = act.ravel()
    tags = np.asarray(prob.tags).ravel()
    vel = act & (tags != 1) & (tags != 2)
    pr = act.reshape(2 * nz + 1, 2 * ny + 1, 2 * nx + 1)[::2, ::2, ::2]
    return int(3 * vel.sum() + pr.sum())


def _server_sigs(lib):
    vp = C.c_void_p
    sig = {
        "gdsw_server_create": ([C.c_int32, C.c_int64, C.c_int32, C.POINTER(vp)], C.c_int),
        "gdsw_server_submit": ([vp, C.POINTER(gdsw_request), C.POINTER(C.c_int64)], C.c_int),
        "gdsw_server_poll": ([vp, C.c_int64, C.POINTER(gdsw_request_status)], C.c_int),
        "gdsw_server_wait": ([vp, C.c_int64, C.POINTER(gdsw_request_status)], C.c_int),
        "gdsw_server_stats_read": ([vp, C.POINTER(gdsw_server_stats)], C.c_int),
        "gdsw_server_destroy": ([vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res


class Server:
    """Continuous-batching solve server (gdsw_server_*): submit problems, wait for results."""

    def __init__(self, device=0, mem_budget_bytes=64 << 30, max_slots=4):
        lib = load()
        _server_sigs(lib)
        self.lib = lib
        h = C.c_void_p()
        rc = lib.gdsw_server_create(device, int(mem_budget_bytes), max_slots, C.byref(h))
        if rc != GDSW_OK:
            raise GdswError(rc, "gdsw_server_create failed")
        self.h = h
        self.pending = {}

    def gdsw_server_submit(self, prob, levels=None, weighting="pou", precision=("fp32", "fp32", "fp32"),
                           phi_precision="fp32", tol=1e-8, restart=100, max_it=1000, slab_elems=1, rhs=None):
        """Queue one problem; returns a ticket.  The result buffer is kept until wait()."""
        L = prob.levels if levels is None else levels
        n = count_dofs(prob)
        keep = [np.ascontiguousarray(prob.mask, np.uint8), np.ascontiguousarray(prob.tags, np.uint8),
                np.ascontiguousarray(prob.g, np.float64), np.ascontiguousarray(prob.part, np.int32)]
        r = gdsw_request()
        r.mesh = gdsw_mesh(prob.nx, prob.ny, prob.nz, prob.h, (C.c_double * 3)(*prob.origin),
                           keep[0].ctypes.data, keep[1].ctypes.data, keep[2].ctypes.data, PRESSURE[prob.pressure])
        uk = None
        if prob.uk is not None:
            uk = np.ascontiguousarray(prob.uk, np.float64)
            keep.append(uk)
        r.visc = gdsw_viscosity(FORM[prob.form], prob.nu0, prob.nu_inf, prob.lam, prob.n_carreau,
                                uk.ctypes.data if uk is not None else None)
        r.part.elem_part = keep[3].ctypes.data
        r.part.n_groups = L - 2
        for l in range(L - 2):
            gr = np.ascontiguousarray(prob.groups[l], np.int32)
            keep.append(gr)
            r.part.groups[l] = gr.ctypes.data
            r.part.group_len[l] = gr.size
        r.levels = gdsw_levels(L, 1, 0)
        prec = [PREC[q] for q in precision]
        r.opt = gdsw_options(WEIGHT_POU if weighting == "pou" else WEIGHT_PLAIN, (C.c_int32 * 3)(*prec),
                             PREC[phi_precision], restart, max_it, tol, slab_elems, 0, None)
        x = np.zeros(n)
        if rhs is not None:
            rb = np.ascontiguousarray(rhs, np.float64)
            keep.append(rb)
            r.rhs = rb.ctypes.data
        r.x = x.ctypes.data
        r.x_len = n
        t = C.c_int64()
        rc = self.lib.gdsw_server_submit(self.h, C.byref(r), C.byref(t))
        if rc != GDSW_OK:
            raise GdswError(rc, "gdsw_server_submit failed")
        self.pending[t.value] = x
        return t.value

    def gdsw_server_wait(self, ticket):
        st = gdsw_request_status()
        rc = self.lib.gdsw_server_wait(self.h, ticket, C.byref(st))
        if rc != GDSW_OK:
            raise GdswError(rc, "gdsw_server_wait failed")
        return st, self.pending.pop(ticket)

    def gdsw_server_poll(self, ticket):
        st = gdsw_request_status()
        self.lib.gdsw_server_poll(self.h, ticket, C.byref(st))
        return st

    def gdsw_server_stats_read(self):
        st = gdsw_server_stats()
        self.lib.gdsw_server_stats_read(self.h, C.byref(st))
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.gdsw_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- multigrid
class Multigrid:
    """Geometric multigrid over nested grids (gdsw_mg_*): probs finest first; the fine grids
    become operator-only contexts, the coarsest a multilevel GDSW context whose FGMRES
    tolerance coarse_tol is the coarse-solve tolerance.  solve() runs FP64 FGMRES on the
    finest grid preconditioned by V-cycles (every step in the library's kernels)."""

    def __init__(self, probs, omega=1.0, pre=2, post=2, smoother="fp32", coarse_tol=1e-1,
                 coarse_precision=("fp32", "fp32", "fp32"), coarse_phi="fp32", tol=1e-8, restart=100, max_it=1000,
                 symmetric=False):
        lib = load()
        self.lib = lib
        self.h = None
        self.grids = [Context(p, levels=1, tol=tol, restart=restart, max_it=max_it) for p in probs[:-1]]
        self.grids.append(Context(probs[-1], precision=coarse_precision, phi_precision=coarse_phi, tol=coarse_tol,
                                  restart=100, max_it=1000))
        arr = (C.c_void_p * len(self.grids))(*[g.h.value for g in self.grids])
        o = gdsw_mg_options(float(omega), int(pre), int(post), PREC[smoother], 1 if symmetric else 0)
        h = C.c_void_p()
        rc = lib.gdsw_mg_create(arr, len(self.grids), C.byref(o), C.byref(h))
        if rc != GDSW_OK:
            raise GdswError(rc, lib.gdsw_mg_last_error(None).decode())
        self.h = h
        self.n = self.grids[0].n

    def _check(self, rc):
        if rc != GDSW_OK:
            raise GdswError(rc, self.lib.gdsw_mg_last_error(self.h).decode())
        return rc

    def gdsw_mg_vcycle(self, r, z):
        return self._check(self.lib.gdsw_mg_vcycle(self.h, _ptr(r), _ptr(z)))

    def gdsw_mg_smooth(self, grid, b, x, steps):
        return self._check(self.lib.gdsw_mg_smooth(self.h, grid, _ptr(b), _ptr(x), steps))

    def gdsw_mg_prolong(self, grid, xc, zf):
        return self._check(self.lib.gdsw_mg_prolong(self.h, grid, _ptr(xc), _ptr(zf)))

    def gdsw_mg_restrict(self, grid, rf, rc):
        return self._check(self.lib.gdsw_mg_restrict(self.h, grid, _ptr(rf), _ptr(rc)))

    def gdsw_mg_stats(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self.lib.gdsw_mg_stats(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return dict(cycles=a.value, coarse_solves=b.value, coarse_iterations=c.value)

    def solve(self, b, x):
        """FGMRES on the finest grid, V-cycle preconditioned; x holds the initial guess."""
        return self.grids[0].gdsw_solve(b, x)

    def close(self):
        if self.h:
            self.lib.gdsw_mg_destroy(self.h)
            self.h = None
        for g in getattr(self, "grids", []):
            g.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
