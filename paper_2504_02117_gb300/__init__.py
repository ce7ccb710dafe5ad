"""Thin Python binding of libpint (include/pint.h), GB300 / sm_103a.

Argument marshalling only: every step of the block solve runs in the CUDA
kernels of libpint.so. PyTorch provides device memory and streams. The
functions keep the C names; tensors are passed as their data pointers.
Importing this package loads libpint.so and fails loudly when it has not been
built (run `python -c "import __graft_entry__ as g; g.build()"`).
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# PINT_LIB may name the checked build (libpint_bounds.so) or another build
# of the same library; the default is the in-tree libpint.so
LIB_PATH = os.environ.get("PINT_LIB") or os.path.join(_HERE, "libpint.so")

PINT_OK = 0
PINT_ERR_INVALID = 1
PINT_ERR_NOMEM = 2
PINT_ERR_CUDA = 3
PINT_ERR_NOT_CONVERGED = 4
PINT_ERR_BREAKDOWN = 5
PINT_ERR_TIMEOUT = 6
PINT_MAX_S = 16
PINT_MEM_HOST, PINT_MEM_DEVICE = 0, 1
PINT_PC_NONE, PINT_PC_JACOBI, PINT_PC_ILU0 = 0, 1, 2
PINT_FP64, PINT_FP32, PINT_BF16 = 0, 1, 2
PINT_SOLVER_GMRES, PINT_SOLVER_CG, PINT_SOLVER_BICGSTAB, PINT_SOLVER_GLOBAL = 0, 1, 2, 3
PINT_PROBLEM_DIFFREACT, PINT_PROBLEM_RICHARDS = 1, 2
KERNEL_FAMILIES = ["coupled", "spmm", "gram", "update", "cholqr", "hess", "ilu", "norm", "vec",
                   "nl"]

_STATUS = {0: "PINT_OK", 1: "PINT_ERR_INVALID", 2: "PINT_ERR_NOMEM", 3: "PINT_ERR_CUDA",
           4: "PINT_ERR_NOT_CONVERGED", 5: "PINT_ERR_BREAKDOWN", 6: "PINT_ERR_TIMEOUT"}


class PintError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class pint_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("inner_tol", C.c_double), ("max_step", C.c_double),
                ("lscheme_L", C.c_double), ("restart", C.c_int),
                ("max_outer", C.c_int), ("max_inner", C.c_int), ("precond", C.c_int),
                ("precision", C.c_int), ("solver", C.c_int), ("reserved", C.c_int * 2)]


class pint_batch_job(C.Structure):
    _fields_ = [("op", C.c_void_p), ("B", C.c_void_p), ("B0", C.c_void_p), ("Y", C.c_void_p)]


class pint_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("outer_its", C.c_int), ("inner_its", C.c_int),
                ("restarts", C.c_int), ("deflations", C.c_int), ("kernel_launches", C.c_int),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double),
                ("col_relres", C.c_double * PINT_MAX_S), ("flops", C.c_double)]

    def as_dict(self, s=PINT_MAX_S):
        return {"status": self.status, "outer_its": self.outer_its, "inner_its": self.inner_its,
                "restarts": self.restarts, "deflations": self.deflations,
                "kernel_launches": self.kernel_launches, "setup_ms": self.setup_ms,
                "solve_ms": self.solve_ms, "col_relres": list(self.col_relres)[:s],
                "flops": self.flops}


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2504_02117_gb300.build.build() "
                      "(nvcc, sm_103a); there is no fallback path")
lib = C.CDLL(LIB_PATH)

_vp, _i, _i64, _d, _sz = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_size_t
_SIGS = {
    "pint_opts_default": (None, [C.POINTER(pint_opts)]),
    "pint_create": (_i, [C.POINTER(_vp), _i, _sz]),
    "pint_destroy": (_i, [_vp]),
    "pint_last_error": (C.c_char_p, [_vp]),
    "pint_bytes_in_use": (_sz, [_vp]),
    "pint_operator_assemble": (_i, [_vp, C.POINTER(_vp), _i64, _vp, _vp, _vp, _vp, _i, _vp]),
    "pint_operator_update_values": (_i, [_vp, _vp, _vp, _i, _vp]),
    "pint_operator_destroy": (_i, [_vp]),
    "pint_operator_nnz": (_i64, [_vp]),
    "pint_fv_convdiff": (_i, [_vp, C.POINTER(_vp), _i, _i, _i, _vp, _d, _d, _d, _i, _vp]),
    "pint_set_coupling": (_i, [_vp, _i, _vp, _vp]),
    "pint_coupling_from_dirk": (_i, [_vp, _i, _i, _d, _i, _vp, _vp, _vp, C.POINTER(_i)]),
    "pint_apply_coupled": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "pint_solve_block": (_i, [_vp, _vp, _vp, _vp, C.POINTER(pint_opts), C.POINTER(pint_stats), _vp]),
    "pint_solve_batch": (_i, [_vp, _i, C.POINTER(pint_batch_job), C.POINTER(pint_opts), _i,
                              _i, C.POINTER(pint_stats), _vp]),
    "pint_batch_plan_create": (_i, [_vp, _i, C.POINTER(pint_batch_job), C.POINTER(pint_opts),
                                    _i, _i, C.POINTER(_vp), _vp]),
    "pint_batch_plan_run": (_i, [_vp, C.POINTER(pint_stats), _vp]),
    "pint_batch_plan_shape": (_i, [_vp, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i)]),
    "pint_batch_plan_destroy": (_i, [_vp]),
    "pint_batch_auto_cluster": (_i, [_vp, _i, C.POINTER(pint_batch_job)]),
    "pint_batch_auto_threads": (_i, [_vp, _i, _i]),
    "pint_shift": (_i, [_vp, _i64, _i, _vp]),
    "pint_problem_create": (_i, [_vp, C.POINTER(_vp), _i, _i, _i, _i, _vp, _vp, _vp]),
    "pint_problem_destroy": (_i, [_vp]),
    "pint_vg_lipschitz": (_i, [_vp, C.POINTER(_d)]),
    "pint_problem_operator": (_vp, [_vp]),
    "pint_problem_eval": (_i, [_vp, _d, _vp, _vp, _vp, _vp]),
    "pint_problem_residual": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "pint_newton_step": (_i, [_vp, _vp, _vp, _vp, C.POINTER(pint_opts), C.POINTER(_i),
                              C.POINTER(pint_stats), _vp]),
    "pint_pipeline_run": (_i, [_vp, _vp, _vp, _i, _d, _i, _vp, _i, _vp, C.POINTER(pint_opts),
                               C.POINTER(pint_stats), _vp]),
    "pint_profile_enable": (_i, [_vp, _i]),
    "pint_profile_read": (_i, [_vp, _i, C.POINTER(_d), C.POINTER(_d), C.POINTER(_d),
                               C.POINTER(C.c_longlong)]),
    "pint_profile_reset": (_i, [_vp]),
    "pint_residual_history": (_i, [_vp, _vp, _i, C.POINTER(_i), C.POINTER(_i)]),
    "pint_residual_history_reset": (_i, [_vp]),
    "pint_bounds_report": (_i, [_vp, C.POINTER(C.c_longlong), C.POINTER(_i),
                                C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "pint_test_bounds": (_i, [_vp, C.c_longlong, C.c_longlong]),
    "pint_kernel_launches": (C.c_longlong, [_vp]),
    "pint_inner_apply": (_i, [_vp, _vp, _vp, _vp]),
    "pint_inner_apply_lowp": (_i, [_vp, _i, _vp, _vp, _vp]),
    "pint_precond_apply": (_i, [_vp, _i, _vp, _vp, _vp]),
    "pint_ilu0_apply_f32": (_i, [_vp, _vp, _vp, _vp]),
    "pint_block_gram": (_i, [_vp, _i, _i64, _i, _i, _vp, _vp, _vp, _vp]),
    "pint_block_update": (_i, [_vp, _i, _i64, _i, _i, _vp, _vp, _vp, _vp]),
    "pint_block_gram_noalloc": (_i, [_i, _i64, _i, _i, _vp, _vp, _vp, _vp]),
    "pint_cholqr2": (_i, [_vp, _i, _i64, _i, _vp, _vp, _vp]),
    "pint_colnorms": (_i, [_vp, _i, _i64, _i, _vp, _vp, _vp]),
    "pint_test_wait_timeout": (_i, [_vp, _i, _d, _vp]),
    "pint_fp64_fma_peak": (_i, [_vp, C.POINTER(_d)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


# ------------------------------------------------------------------ helpers
def _ptr(t):
    """Data pointer of a tensor / numpy array / None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return C.c_void_p(t.data_ptr())
    if hasattr(t, "ctypes"):
        return C.c_void_p(t.ctypes.data)
    raise TypeError(type(t))


def _stream(stream=None):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)


def _check(rc, ctx=None, allow=()):
    if rc != PINT_OK and rc not in allow:
        raise PintError(rc, lib.pint_last_error(ctx).decode())
    return rc


def _host_f64(a):
    import numpy as np
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------- same-name API
def pint_opts_default():
    o = pint_opts()
    lib.pint_opts_default(C.byref(o))
    return o


def pint_create(device=0, hbm_budget=0):
    h = C.c_void_p()
    _check(lib.pint_create(C.byref(h), device, hbm_budget))
    return h


def pint_destroy(ctx):
    return lib.pint_destroy(ctx)


def pint_last_error(ctx):
    return lib.pint_last_error(ctx).decode()


def pint_bytes_in_use(ctx):
    return lib.pint_bytes_in_use(ctx)


def pint_operator_assemble(ctx, n, rowptr, colind, K_vals, M_diag=None, stream=None):
    """CSR arrays: torch CUDA tensors (device) or numpy arrays (host)."""
    dev = hasattr(rowptr, "is_cuda") and rowptr.is_cuda
    op = C.c_void_p()
    _check(lib.pint_operator_assemble(ctx, C.byref(op), n, _ptr(rowptr), _ptr(colind),
                                      _ptr(K_vals), _ptr(M_diag),
                                      PINT_MEM_DEVICE if dev else PINT_MEM_HOST,
                                      _stream(stream) if dev else None), ctx)
    return op


def pint_operator_update_values(ctx, op, K_vals=None, M_diag=None, stream=None):
    ref = K_vals if K_vals is not None else M_diag
    dev = hasattr(ref, "is_cuda") and ref.is_cuda
    _check(lib.pint_operator_update_values(op, _ptr(K_vals), _ptr(M_diag),
                                           PINT_MEM_DEVICE if dev else PINT_MEM_HOST,
                                           _stream(stream) if dev else None), ctx)


def pint_operator_destroy(op):
    return lib.pint_operator_destroy(op)


def pint_operator_nnz(op):
    return lib.pint_operator_nnz(op)


def pint_fv_convdiff(ctx, nx, ny, nz, D, velocity, stream=None):
    dev = hasattr(D, "is_cuda") and D.is_cuda
    op = C.c_void_p()
    Dh = D if dev else _host_f64(D)
    _check(lib.pint_fv_convdiff(ctx, C.byref(op), nx, ny, nz, _ptr(Dh), *map(float, velocity),
                                PINT_MEM_DEVICE if dev else PINT_MEM_HOST, _stream(stream)), ctx)
    return op


def pint_set_coupling(ctx, op, A1, A2):
    A1 = _host_f64(A1)
    A2 = _host_f64(A2)
    s = A1.shape[0]
    _check(lib.pint_set_coupling(op, s, _ptr(A1), _ptr(A2)), ctx)


def pint_coupling_from_dirk(A, steps, tau, eliminate_first=False):
    import numpy as np
    A = _host_f64(A)
    m = A.shape[0]
    mp = m - 1 if eliminate_first else m
    S = steps * mp
    A1 = np.zeros((S, S))
    A2 = np.zeros((S, S))
    e = np.zeros(max(m, 1))
    s = C.c_int()
    _check(lib.pint_coupling_from_dirk(_ptr(A), m, steps, tau, int(eliminate_first), _ptr(A1),
                                       _ptr(A2), _ptr(e), C.byref(s)))
    return A1, A2, e[:m - 1] if eliminate_first else None


def pint_apply_coupled(ctx, op, Y, B, B0, R, stream=None):
    _check(lib.pint_apply_coupled(op, _ptr(Y), _ptr(B), _ptr(B0), _ptr(R), _stream(stream)), ctx)


def pint_solve_block(ctx, op, B, B0, Y, opts=None, stream=None, raise_on_nonconvergence=False):
    o = opts if opts is not None else pint_opts_default()
    st = pint_stats()
    rc = lib.pint_solve_block(op, _ptr(B), _ptr(B0), _ptr(Y), C.byref(o), C.byref(st),
                              _stream(stream))
    _check(rc, ctx, allow=() if raise_on_nonconvergence else (PINT_ERR_NOT_CONVERGED,))
    return st


def pint_solve_batch(ctx, jobs, opts=None, cluster_ctas=0, cta_threads=0, stream=None,
                     raise_on_nonconvergence=False):
    """jobs: sequence of (op, B, B0, Y) (B, B0 may be None). Returns the
    per-job pint_stats list."""
    o = opts if opts is not None else pint_opts_default()
    arr = _batch_jobs(jobs)
    sts = (pint_stats * len(jobs))()
    rc = lib.pint_solve_batch(ctx, len(jobs), arr, C.byref(o), int(cluster_ctas),
                              int(cta_threads), sts, _stream(stream))
    _check(rc, ctx, allow=() if raise_on_nonconvergence else (PINT_ERR_NOT_CONVERGED,))
    return list(sts)


def _batch_jobs(jobs):
    arr = (pint_batch_job * len(jobs))()
    for i, (op, B, B0, Y) in enumerate(jobs):
        arr[i].op = op.value if isinstance(op, C.c_void_p) else op
        arr[i].B = None if B is None else B.data_ptr()
        arr[i].B0 = None if B0 is None else B0.data_ptr()
        arr[i].Y = Y.data_ptr()
    return arr


def pint_batch_plan_create(ctx, jobs, opts=None, cluster_ctas=0, cta_threads=0, stream=None):
    """jobs: sequence of (op, B, B0, Y) device tensors (B, B0 may be None);
    the tensors must stay alive until pint_batch_plan_destroy."""
    o = opts if opts is not None else pint_opts_default()
    h = C.c_void_p()
    _check(lib.pint_batch_plan_create(ctx, len(jobs), _batch_jobs(jobs), C.byref(o),
                                      int(cluster_ctas), int(cta_threads), C.byref(h),
                                      _stream(stream)), ctx)
    return h


def pint_batch_plan_run(ctx, plan, njobs, stream=None, raise_on_nonconvergence=False):
    sts = (pint_stats * njobs)()
    rc = lib.pint_batch_plan_run(plan, sts, _stream(stream))
    _check(rc, ctx, allow=() if raise_on_nonconvergence else (PINT_ERR_NOT_CONVERGED,))
    return list(sts)


def pint_batch_plan_shape(ctx, plan):
    c, t, r = C.c_int(), C.c_int(), C.c_int()
    _check(lib.pint_batch_plan_shape(plan, C.byref(c), C.byref(t), C.byref(r)), ctx)
    return {"cluster_ctas": c.value, "cta_threads": t.value, "resident_clusters": r.value}


def pint_batch_plan_destroy(plan):
    return lib.pint_batch_plan_destroy(plan)


class BatchPlan:
    """A resident batched solve over the pint_batch_plan_* calls: the jobs'
    device buffers are borrowed; write new B / initial Y into them between
    run() calls."""

    def __init__(self, ctx, jobs, opts=None, cluster_ctas=0, cta_threads=0, stream=None):
        self.ctx = ctx
        self.njobs = len(jobs)
        self._keep = list(jobs)                    # keep the tensors alive
        self.h = pint_batch_plan_create(ctx, jobs, opts, cluster_ctas, cta_threads, stream)

    def run(self, stream=None, raise_on_nonconvergence=False):
        return pint_batch_plan_run(self.ctx, self.h, self.njobs, stream,
                                   raise_on_nonconvergence)

    def shape(self):
        return pint_batch_plan_shape(self.ctx, self.h)

    def close(self):
        if self.h:
            pint_batch_plan_destroy(self.h)
            self.h = None


def pint_batch_auto_cluster(ctx, jobs):
    """jobs: sequence of (op, B, B0, Y) as for pint_solve_batch."""
    return lib.pint_batch_auto_cluster(ctx, len(jobs), _batch_jobs(jobs))


def pint_batch_auto_threads(ctx, njobs, cluster_ctas):
    return lib.pint_batch_auto_threads(ctx, int(njobs), int(cluster_ctas))


def pint_shift(Y, n, s, stream=None):
    _check(lib.pint_shift(_ptr(Y), n, s, _stream(stream)))


def pint_problem_create(ctx, kind, nx, ny, nz, params=None, field=None, stream=None):
    p = C.c_void_p()
    prm = None if params is None else _host_f64(params)
    _check(lib.pint_problem_create(ctx, C.byref(p), kind, nx, ny, nz, _ptr(prm), _ptr(field),
                                   _stream(stream)), ctx)
    return p


def pint_problem_destroy(prob):
    return lib.pint_problem_destroy(prob)


def pint_vg_lipschitz(params):
    """sup theta'(psi) of the van Genuchten params (alpha, n, theta_r, theta_s)."""
    L = _d()
    _check(lib.pint_vg_lipschitz(_ptr(_host_f64(params[:4])), C.byref(L)))
    return L.value


def pint_problem_operator(prob):
    return C.c_void_p(lib.pint_problem_operator(prob))


def pint_problem_eval(ctx, prob, t, y, mass_out=None, f_out=None, stream=None):
    _check(lib.pint_problem_eval(prob, float(t), _ptr(y), _ptr(mass_out), _ptr(f_out),
                                 _stream(stream)), ctx)


def pint_problem_residual(ctx, prob, times, Y, B0, R, stream=None):
    tt = _host_f64(times)
    _check(lib.pint_problem_residual(prob, _ptr(tt), _ptr(Y), _ptr(B0), _ptr(R),
                                     _stream(stream)), ctx)


def pint_newton_step(ctx, prob, times, Y, B0, opts=None, stream=None):
    o = opts if opts is not None else pint_opts_default()
    tt = _host_f64(times)
    conv = C.c_int()
    st = pint_stats()
    _check(lib.pint_newton_step(prob, _ptr(tt), _ptr(Y), _ptr(B0), C.byref(o), C.byref(conv),
                                C.byref(st), _stream(stream)), ctx)
    return bool(conv.value), st


def pint_pipeline_run(ctx, prob, A, c, tau, s, y0, nstages, stages_out, opts=None, stream=None):
    o = opts if opts is not None else pint_opts_default()
    A = _host_f64(A)
    c = _host_f64(c)
    st = pint_stats()
    _check(lib.pint_pipeline_run(prob, _ptr(A), _ptr(c), A.shape[0], float(tau), s, _ptr(y0),
                                 nstages, _ptr(stages_out), C.byref(o), C.byref(st),
                                 _stream(stream)), ctx)
    return st


def pint_inner_apply(ctx, op, X, Z, stream=None):
    _check(lib.pint_inner_apply(op, _ptr(X), _ptr(Z), _stream(stream)), ctx)


def pint_inner_apply_lowp(ctx, op, precision, X, Z, stream=None):
    _check(lib.pint_inner_apply_lowp(op, precision, _ptr(X), _ptr(Z), _stream(stream)), ctx)


def pint_precond_apply(ctx, op, precond, X, Z, stream=None):
    _check(lib.pint_precond_apply(op, precond, _ptr(X), _ptr(Z), _stream(stream)), ctx)


def pint_ilu0_apply_f32(ctx, op, X, Z, stream=None):
    _check(lib.pint_ilu0_apply_f32(op, _ptr(X), _ptr(Z), _stream(stream)), ctx)


def pint_block_gram(ctx, precision, n, s, nb, V, W, H, stream=None):
    _check(lib.pint_block_gram(ctx, precision, n, s, nb, _ptr(V), _ptr(W), _ptr(H),
                               _stream(stream)), ctx)


def pint_block_gram_noalloc(precision, n, s, nb, V, W, H, stream=None):
    """Gram product without device allocation (no context; fixed scratch)."""
    _check(lib.pint_block_gram_noalloc(precision, n, s, nb, _ptr(V), _ptr(W), _ptr(H),
                                       _stream(stream)))


def pint_block_update(ctx, precision, n, s, nb, V, H, W, stream=None):
    _check(lib.pint_block_update(ctx, precision, n, s, nb, _ptr(V), _ptr(H), _ptr(W),
                                 _stream(stream)), ctx)


def pint_cholqr2(ctx, precision, n, s, W, R, stream=None):
    _check(lib.pint_cholqr2(ctx, precision, n, s, _ptr(W), _ptr(R), _stream(stream)), ctx)


def pint_colnorms(ctx, precision, n, s, X, stream=None):
    import numpy as np
    out = np.zeros(s)
    _check(lib.pint_colnorms(ctx, precision, n, s, _ptr(X), _ptr(out), _stream(stream)), ctx)
    return out


def pint_test_wait_timeout(ctx, which, limit_ms, stream=None):
    """Run one bounded device wait that must run out (0: the ILU(0) flag
    wait, 1: the bulk-copy mbarrier wait); returns the status code."""
    return lib.pint_test_wait_timeout(ctx, which, limit_ms, _stream(stream))


def pint_fp64_fma_peak(ctx):
    """Measured float64 FMA throughput of the device, TFLOP/s."""
    v = C.c_double()
    _check(lib.pint_fp64_fma_peak(ctx, C.byref(v)), ctx)
    return v.value


def pint_profile_enable(ctx, on=True, nvtx=False):
    """on: CUDA-event timing per kernel family; nvtx: an NVTX range per
    family launch."""
    _check(lib.pint_profile_enable(ctx, int(bool(on)) | (2 if nvtx else 0)), ctx)


def pint_profile_read(ctx, k):
    """Totals of kernel family k: dict(ms, bytes, flops, launches)."""
    ms, by, fl, la = C.c_double(), C.c_double(), C.c_double(), C.c_longlong()
    _check(lib.pint_profile_read(ctx, k, C.byref(ms), C.byref(by), C.byref(fl), C.byref(la)), ctx)
    return {"ms": ms.value, "bytes": by.value, "flops": fl.value, "launches": la.value}


def pint_profile_reset(ctx):
    _check(lib.pint_profile_reset(ctx), ctx)


def pint_kernel_launches(ctx):
    return lib.pint_kernel_launches(ctx)


def pint_residual_history(ctx):
    """The last solve's per-column relative residuals: a (rows, s) numpy
    array, one row per outer (or Newton) iteration."""
    import numpy as np
    rows, s = C.c_int(), C.c_int()
    _check(lib.pint_residual_history(ctx, None, 0, C.byref(rows), C.byref(s)), ctx)
    out = np.zeros((rows.value, max(s.value, 0)))
    if rows.value and s.value:
        _check(lib.pint_residual_history(ctx, _ptr(out), rows.value, C.byref(rows),
                                         C.byref(s)), ctx)
    return out


def pint_residual_history_reset(ctx):
    _check(lib.pint_residual_history_reset(ctx), ctx)


def pint_bounds_report(ctx):
    """(count, site, index, bound) of the index checks since the last report;
    count is -1 when the library was built without them."""
    c, st, i, b = C.c_longlong(), C.c_int(), C.c_longlong(), C.c_longlong()
    _check(lib.pint_bounds_report(ctx, C.byref(c), C.byref(st), C.byref(i), C.byref(b)), ctx)
    return c.value, st.value, i.value, b.value


def pint_test_bounds(ctx, index, bound):
    _check(lib.pint_test_bounds(ctx, int(index), int(bound)), ctx)
