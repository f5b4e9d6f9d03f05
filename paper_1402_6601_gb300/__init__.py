"""GB300 (sm_103a) tiled Cholesky factorization and solves behind a C ABI.

This module is a thin ctypes binding over ``include/chol.h``: the functions with the C names
(``chol_factor``, ``chol_solve``, ...) marshal arguments and call the CUDA library; the
Pythonic helpers (``factor``, ``solve``, ``posv``) only allocate workspaces with torch and
check layouts. Every step of the computation runs in the library's kernels; there is no
CPU or PyTorch fallback, and a missing library raises at import time.

Matrices are float64 and column-major: a CUDA tensor ``A`` with ``A.stride(0) == 1`` and
``A.stride(1) >= A.shape[0]`` (``colmajor(x)`` makes one).
"""
import ctypes
import os

import torch

from . import build as _build

__all__ = [
    "lib", "ChOpts", "POLICIES", "opts", "colmajor", "factor", "solve", "trsm_sweep", "posv",
    "posv_host", "workspace_size", "solve_workspace_size", "num_workers", "trace", "factor_f32",
    "solve_refine", "refine_workspace_size", "cholesky_backward", "solve_backward", "lower",
    "cholesky", "cholesky_solve", "solve_spd", "BatchOpts", "Batch", "posv_batched", "factor_batched",
    "solve_batched", "batched_autotune", "lu_factor", "lu_solve", "lu_workspace_size", "lu_solve_workspace_size",
    "LUFactors",
    "dag_describe", "dag_bottom_levels", "lu_dag_describe", "lu_dag_bottom_levels", "dag_bottom_levels_device", "chrome_trace", "sched_activate", "sched_activate_device",
    "CholeskyError", "probe_fp64",
]

POLICIES = {"heft": 0, "dada": 1, "steal": 2, "static": 3}
STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "workspace too small",
          -4: "device wait timed out", -5: "unsupported device or shape", 1: "not positive definite"}
INFO_TIMEOUT = -1
INFO_QUEUE_FULL = -2


class CholeskyError(RuntimeError):
    pass


class ChOpts(ctypes.Structure):
    _fields_ = [
        ("nb", ctypes.c_int),
        ("policy", ctypes.c_int),
        ("alpha", ctypes.c_double),
        ("steal", ctypes.c_int),
        ("workers_per_sm", ctypes.c_int),
        ("num_workers", ctypes.c_int),
        ("queue_order", ctypes.c_int),
        ("dada_max_iter", ctypes.c_int),
        ("dada_eps", ctypes.c_double),
        ("cost_ns", ctypes.c_longlong * 4),
        ("timeout_ns", ctypes.c_longlong),
        ("trace", ctypes.c_int),
        ("hold_task", ctypes.c_longlong),
        ("use_cp", ctypes.c_int),
        ("cp_gbs", ctypes.c_double),
        ("split", ctypes.c_int),
        ("keep_next", ctypes.c_int),
    ]


_c = ctypes
_P = ctypes.c_void_p
_SZ = ctypes.c_size_t
_I = ctypes.c_int
_LL = ctypes.c_longlong
_D = ctypes.c_double
_OPTS = ctypes.POINTER(ChOpts)

_SIGNATURES = {
    "chol_opts_default": (None, [_OPTS]),
    "chol_opts_size": (_SZ, []),
    "chol_factor_workspace_size": (_SZ, [_I, _OPTS]),
    "chol_factor": (_I, [_I, _P, _I, _OPTS, _P, _SZ, _P, _P]),
    "chol_factor_trace_offset": (_LL, [_I, _OPTS]),
    "chol_solve_workspace_size": (_SZ, [_I, _I]),
    "chol_solve": (_I, [_I, _I, _P, _I, _P, _I, _P, _SZ, _P, _P]),
    "chol_trsm_sweep": (_I, [_I, _I, _I, _P, _I, _P, _I, _P, _SZ, _P, _P]),
    "chol_solve_f32": (_I, [_I, _I, _P, _I, _P, _I, _P, _SZ, _P, _P]),
    "chol_solve_noalloc": (_I, [_I, _I, _P, _I, _P, _I, _P, _P]),
    "chol_factor_f32": (_I, [_I, _P, _I, _OPTS, _P, _SZ, _P, _P]),
    "chol_factor_lowp": (_I, [_I, _I, _P, _I, _OPTS, _P, _SZ, _P, _P]),
    "chol_factor_lowp_workspace_size": (_SZ, [_I, _I, _OPTS]),
    "chol_solve_refine_prec_workspace_size": (_SZ, [_I, _I, _I, _OPTS]),
    "chol_solve_refine_workspace_size": (_SZ, [_I, _I, _OPTS]),
    "chol_solve_refine": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _I, _D, _I, _OPTS, _P, _SZ, _P, _P, _P, _P]),
    "chol_backward_workspace_size": (_SZ, [_I]),
    "chol_backward": (_I, [_I, _P, _I, _P, _I, _P, _SZ, _P]),
    "chol_solve_backward_workspace_size": (_SZ, [_I, _I]),
    "chol_solve_backward": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P, _SZ, _P]),
    "chol_lower_copy": (_I, [_I, _P, _I, _P, _I, _P]),
    "chol_batch_opts_default": (None, [_P]),
    "chol_batched_workspace_size": (_SZ, [_I]),
    "chol_posv_batched": (_I, [_I, _I, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "chol_factor_batched": (_I, [_I, _I, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "chol_solve_batched": (_I, [_I, _I, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "chol_batched_autotune": (_I, [_I, _I, _P, _P, _P, _P, _P, _P, _SZ, _P, _P, _P]),
    "chol_posv_host_stage_size": (_SZ, [_I, _I, _OPTS]),
    "chol_posv_host": (_I, [_I, _I, _P, _I, _P, _I, _OPTS, _P, _SZ, _P, _P]),
    "chol_lu_workspace_size": (_SZ, [_I, _OPTS]),
    "chol_lu_aux_size": (_I, [_I, _OPTS, _P, _P]),
    "chol_lu_factor": (_I, [_I, _P, _I, _P, _P, _OPTS, _P, _SZ, _P, _P]),
    "chol_lu_solve_workspace_size": (_SZ, [_I, _I, _OPTS]),
    "chol_lu_solve": (_I, [_I, _I, _P, _I, _P, _P, _OPTS, _P, _I, _P, _SZ, _P, _P]),
    "chol_lu_dag_task_count": (_LL, [_I]),
    "chol_lu_dag_describe": (_I, [_I, _P, _P, _P, _P, _P, _P, _P]),
    "chol_lu_dag_bottom_levels": (_I, [_I, _P, _P]),
    "chol_dag_task_count": (_LL, [_I]),
    "chol_dag_edge_count": (_LL, [_I]),
    "chol_dag_describe": (_I, [_I, _P, _P, _P, _P, _P, _P, _P]),
    "chol_dag_bottom_levels": (_I, [_I, _P, _P]),
    "chol_dag_bottom_levels_device": (_I, [_I, _I, _P, _P, _P]),
    "chol_sched_activate": (_I, [_I, _D, _I, _D, _I, _P, _P, _P, _P, _P, _I, _P, _P, _P, _I, _P, _P, _P, _P]),
    "chol_sched_activate_device": (_I, [_I, _D, _I, _D, _I, _P, _P, _P, _P, _P, _I, _P, _P, _P, _I, _P, _P, _P,
                                        _P, _P]),
    "chol_probe_fp64_flops": (_LL, [_I, _I, _I, _LL]),
    "chol_probe_fp64": (_I, [_I, _I, _I, _LL, _P, _P]),
    "chol_version": (ctypes.c_char_p, []),
    "chol_num_workers": (_I, [_OPTS]),
}


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError("the CUDA library is not built (%s); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()
for _name in _SIGNATURES:
    globals()[_name] = getattr(lib, _name)
    __all__.append(_name)


def opts(nb=0, policy="heft", alpha=0.5, steal=None, workers_per_sm=2, num_workers=0,
         queue_order=None, dada_max_iter=16, dada_eps=0.01, cost_ns=None, timeout_ns=0, trace=False,
         hold_task=-1, use_cp=False, cp_gbs=40.0, split=1, keep_next=1):
    o = ChOpts()
    lib.chol_opts_default(ctypes.byref(o))
    o.nb = nb
    o.policy = POLICIES[policy] if isinstance(policy, str) else int(policy)
    o.alpha = alpha
    o.steal = (0 if o.policy == 3 else 1) if steal is None else int(bool(steal))
    o.workers_per_sm = workers_per_sm
    o.num_workers = num_workers
    o.queue_order = (1 if o.policy == 2 else 0) if queue_order is None else int(queue_order)
    o.dada_max_iter = dada_max_iter
    o.dada_eps = dada_eps
    if cost_ns is not None:
        for k in range(4):
            o.cost_ns[k] = int(cost_ns[k])
    o.timeout_ns = int(timeout_ns)
    o.trace = int(bool(trace))
    o.hold_task = int(hold_task)
    o.use_cp = int(bool(use_cp))
    o.cp_gbs = float(cp_gbs)
    o.split = int(split)
    o.keep_next = int(keep_next)
    return o


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(status, what):
    if status != 0:
        raise CholeskyError("%s: %s (%d)" % (what, STATUS.get(status, "?"), status))


def colmajor(x):
    """Column-major copy of a 2-D tensor (or a 1-D tensor as one column). Always a new
    tensor, never a view of x, so that in-place calls on it leave x untouched."""
    if x.dim() == 1:
        x = x.reshape(-1, 1)
    y = torch.empty_strided(tuple(x.shape), (1, max(1, x.shape[0])), dtype=x.dtype, device=x.device)
    y.copy_(x)
    return y


def _check_matrix(A, name, dtype=torch.float64):
    if not (A.is_cuda and A.dtype == dtype and A.dim() == 2):
        raise ValueError("%s must be a 2-D %s CUDA tensor" % (name, str(dtype).replace("torch.", "")))
    if A.shape[0] > 0 and A.shape[1] > 0 and A.stride(0) != 1:
        raise ValueError("%s must be column-major (stride(0) == 1); use colmajor()" % name)
    return max(1, A.stride(1) if A.shape[1] > 1 else A.shape[0])


def workspace_size(n, o=None):
    o = o or opts()
    return int(lib.chol_factor_workspace_size(n, ctypes.byref(o)))


def solve_workspace_size(n, nrhs):
    return int(lib.chol_solve_workspace_size(n, nrhs))


def num_workers(o=None):
    o = o or opts()
    return int(lib.chol_num_workers(ctypes.byref(o)))


def _workspace(nbytes, device):
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def factor(A, o=None, work=None, info=None, stream=None, check=False):
    """Factor A = L L^T in place (lower triangle of A). Returns (info tensor, workspace).

    With check=True the call synchronises and raises CholeskyError on a non-zero info."""
    o = o or opts()
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("A must be square")
    lda = _check_matrix(A, "A")
    if work is None:
        work = _workspace(workspace_size(n, o), A.device)
    if info is None:
        info = torch.zeros(1, dtype=torch.int32, device=A.device)
    st = lib.chol_factor(n, A.data_ptr(), lda, ctypes.byref(o), work.data_ptr(), work.numel(),
                         info.data_ptr(), _stream(stream))
    _check(st, "chol_factor")
    if check:
        v = int(info.item())
        if v != 0:
            raise CholeskyError("chol_factor: info = %d" % v)
    return info, work


# precisions of the low-precision factor (chol_precision)
F64, F32, BF16, BF16X3 = 0, 1, 2, 3
_PREC = {"f32": F32, "bf16": BF16, "bf16x3": BF16X3, F32: F32, BF16: BF16, BF16X3: BF16X3}


def factor_f32(A, o=None, work=None, info=None, stream=None, check=False, precision="f32"):
    """FP32-storage tile Cholesky in place on a column-major float32 CUDA tensor. precision:
    "f32" (FFMA tile bodies), "bf16" (tensor-core SYRK/GEMM with BF16 operands, FP32
    accumulation) or "bf16x3" (three BF16 operand terms: FP32-accurate tensor-core GEMM updates,
    SYRK updates in FFMA)."""
    o = o or opts()
    prec = _PREC[precision]
    n = A.shape[0]
    if not (A.is_cuda and A.dtype == torch.float32 and A.dim() == 2 and A.shape[1] == n):
        raise ValueError("A must be a square float32 CUDA tensor")
    if n > 0 and A.stride(0) != 1:
        raise ValueError("A must be column-major (stride(0) == 1); use colmajor()")
    lda = max(1, A.stride(1) if n > 1 else n)
    if work is None:
        work = _workspace(int(lib.chol_factor_lowp_workspace_size(prec, n, ctypes.byref(o))), A.device)
    if info is None:
        info = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib.chol_factor_lowp(prec, n, A.data_ptr(), lda, ctypes.byref(o), work.data_ptr(), work.numel(),
                                info.data_ptr(), _stream(stream)), "chol_factor_lowp")
    if check and int(info.item()) != 0:
        raise CholeskyError("chol_factor_f32: info = %d" % int(info.item()))
    return info, work


def refine_workspace_size(n, nrhs, o=None, precision=None):
    """Workspace of solve_refine: for one low-precision form, or (None) for any of them."""
    o = o or opts()
    if precision is None:
        return int(lib.chol_solve_refine_workspace_size(n, nrhs, ctypes.byref(o)))
    return int(lib.chol_solve_refine_prec_workspace_size(_PREC[precision], n, nrhs, ctypes.byref(o)))


def lowp_workspace_size(n, o=None, precision="bf16x3"):
    o = o or opts()
    return int(lib.chol_factor_lowp_workspace_size(_PREC[precision], n, ctypes.byref(o)))


def solve_refine(A, B, X=None, tol=1e-14, max_iter=30, o=None, work=None, stream=None, precision="f32"):
    """Mixed-precision solve (low-precision factor: "f32", "bf16" or "bf16x3"; FP64
    refinement). Returns (X, info, iters, berr) as device tensors (no synchronisation)."""
    o = o or opts()
    prec = _PREC[precision]
    n = A.shape[0]
    lda = _check_matrix(A, "A")
    ldb = _check_matrix(B, "B")
    nrhs = B.shape[1]
    if X is None:
        X = colmajor(torch.empty(n, nrhs, dtype=torch.float64, device=A.device))
    ldx = _check_matrix(X, "X")
    if work is None:
        work = _workspace(refine_workspace_size(n, nrhs, o, precision), A.device)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    iters = torch.zeros(1, dtype=torch.int32, device=A.device)
    berr = torch.zeros(1, dtype=torch.float64, device=A.device)
    _check(lib.chol_solve_refine(n, nrhs, A.data_ptr(), lda, B.data_ptr(), ldb, X.data_ptr(), ldx, prec, tol,
                                 max_iter, ctypes.byref(o), work.data_ptr(), work.numel(), info.data_ptr(),
                                 iters.data_ptr(), berr.data_ptr(), _stream(stream)), "chol_solve_refine")
    return X, info, iters, berr


def solve(L, B, work=None, info=None, stream=None):
    """Overwrite B with A^{-1} B given the factor from factor()."""
    n = L.shape[0]
    lda = _check_matrix(L, "L")
    ldb = _check_matrix(B, "B")
    nrhs = B.shape[1]
    if work is None:
        work = _workspace(solve_workspace_size(n, nrhs), L.device)
    st = lib.chol_solve(n, nrhs, L.data_ptr(), lda, B.data_ptr(), ldb, work.data_ptr(), work.numel(),
                        info.data_ptr() if info is not None else None, _stream(stream))
    _check(st, "chol_solve")
    return B


def solve_f32(L, B, work=None, info=None, stream=None):
    """X = (L L^T)^{-1} B in place on the column-major float32 CUDA matrix B, with an FP32 factor."""
    n = L.shape[0]
    lda = _check_matrix(L, "L", torch.float32)
    ldb = _check_matrix(B, "B", torch.float32)
    nrhs = B.shape[1]
    if work is None:
        work = _workspace(solve_workspace_size(n, nrhs), L.device)
    st = lib.chol_solve_f32(n, nrhs, L.data_ptr(), lda, B.data_ptr(), ldb, work.data_ptr(), work.numel(),
                            info.data_ptr() if info is not None else None, _stream(stream))
    _check(st, "chol_solve_f32")
    return B


def trsm_sweep(L, B, transpose=False, work=None, info=None, stream=None):
    n = L.shape[0]
    lda = _check_matrix(L, "L")
    ldb = _check_matrix(B, "B")
    nrhs = B.shape[1]
    if work is None:
        work = _workspace(solve_workspace_size(n, nrhs), L.device)
    st = lib.chol_trsm_sweep(int(bool(transpose)), n, nrhs, L.data_ptr(), lda, B.data_ptr(), ldb,
                             work.data_ptr(), work.numel(),
                             info.data_ptr() if info is not None else None, _stream(stream))
    _check(st, "chol_trsm_sweep")
    return B


def posv(A, B, o=None, stream=None):
    """Factor A in place and overwrite B with the solution; returns the info tensor."""
    info, _ = factor(A, o, stream=stream)
    solve(A, B, stream=stream)
    return info


def posv_host(A, B, o=None, stage=None, stream=None):
    """Host-buffer call: A, B are float64 Fortran-ordered numpy arrays (A is overwritten by
    L in its lower triangle, B by X). Returns info."""
    import numpy as np
    o = o or opts()
    n = A.shape[0]
    nrhs = B.shape[1] if B.ndim == 2 else 1
    assert A.dtype == np.float64 and A.flags.f_contiguous and B.dtype == np.float64 and B.flags.f_contiguous
    need = int(lib.chol_posv_host_stage_size(n, nrhs, ctypes.byref(o)))
    if stage is None:
        stage = _workspace(need, torch.device("cuda", torch.cuda.current_device()))
    info = ctypes.c_int(0)
    st = lib.chol_posv_host(n, nrhs, A.ctypes.data, max(1, n), B.ctypes.data, max(1, n), ctypes.byref(o),
                            stage.data_ptr(), stage.numel(), ctypes.byref(info), _stream(stream))
    if st not in (0, 1, -4):
        _check(st, "chol_posv_host")
    return int(info.value)


def trace(work, n, o, graph="chol"):
    """The per-task trace (ntasks x 4 int64: worker, queue it was taken from, start ns, end ns)
    recorded when o.trace is set, from the workspace of chol_factor (graph="chol") or of
    chol_lu_factor (graph="lu"). o.nb must be the tile size the call used (not 0)."""
    off = int(lib.chol_factor_trace_offset(n, ctypes.byref(o)))
    if off < 0:
        raise ValueError("tracing is off")
    if o.nb <= 0:
        raise ValueError("pass the options with the tile size the factorization used")
    T = (n + o.nb - 1) // o.nb
    nt = int(lib.chol_lu_dag_task_count(T) if graph == "lu" else lib.chol_dag_task_count(T))
    return work[off:off + nt * 32].view(torch.int64).reshape(nt, 4)


_KIND_NAMES = {"chol": ("POTRF", "TRSM", "SYRK", "GEMM"), "lu": ("GETRF", "GESSM", "TSTRF", "SSSSM")}


def chrome_trace(records, T, graph="chol", path=None):
    """Chrome-trace (about:tracing / Perfetto) events from a per-task trace: one complete
    event per task on the row of the worker that ran it, named by kind and tile indices,
    times in microseconds from the first start. Tasks without a record (start < 0) are left
    out. Returns the JSON object; writes it to `path` when given."""
    import json
    import numpy as np
    rec = np.asarray(records.cpu() if hasattr(records, "cpu") else records, dtype=np.int64)
    kind, ti, tj, tk, *_ = lu_dag_describe(T) if graph == "lu" else dag_describe(T)
    names = _KIND_NAMES[graph]
    ran = rec[:, 2] >= 0
    t0 = int(rec[ran, 2].min()) if ran.any() else 0
    events = []
    for t in np.nonzero(ran)[0]:
        w, q, a, b = (int(x) for x in rec[t])
        k = int(kind[t])
        events.append({"name": "%s(%d,%d,%d)" % (names[k], ti[t], tj[t], tk[t]), "cat": names[k], "ph": "X",
                       "ts": (a - t0) / 1000.0, "dur": (b - a) / 1000.0, "pid": 0, "tid": w,
                       "args": {"task": int(t), "queue": q}})
    out = {"traceEvents": events, "displayTimeUnit": "ms"}
    if path is not None:
        with open(path, "w") as f:
            json.dump(out, f)
    return out


def dag_describe(T):
    """(kind, i, j, k, indeg, succ_ptr, succ) as numpy arrays, from the library (host code)."""
    import numpy as np
    nt = int(lib.chol_dag_task_count(T))
    ne = int(lib.chol_dag_edge_count(T))
    if nt < 0:
        raise ValueError("T out of range")
    arrs = [np.zeros(nt, np.int32) for _ in range(5)]
    ptr = np.zeros(nt + 1, np.int64)
    succ = np.zeros(max(ne, 1), np.int64)
    _check(lib.chol_dag_describe(T, *[a.ctypes.data for a in arrs], ptr.ctypes.data, succ.ctypes.data),
           "chol_dag_describe")
    return (*arrs, ptr, succ[:ne])


def lu_dag_describe(T):
    """The tile LU graph: (kind, i, j, k, indeg, succ_ptr, succ) as numpy arrays (host code)."""
    import numpy as np
    nt = int(lib.chol_lu_dag_task_count(T))
    if nt < 0:
        raise ValueError("T out of range")
    arrs = [np.zeros(nt, np.int32) for _ in range(5)]
    ptr = np.zeros(nt + 1, np.int64)
    _check(lib.chol_lu_dag_describe(T, *[a.ctypes.data for a in arrs], ptr.ctypes.data, None),
           "chol_lu_dag_describe")
    succ = np.zeros(max(int(ptr[-1]), 1), np.int64)
    _check(lib.chol_lu_dag_describe(T, None, None, None, None, None, None, succ.ctypes.data),
           "chol_lu_dag_describe")
    return (*arrs, ptr, succ[:int(ptr[-1])])


def lu_dag_bottom_levels(T, cost_ns):
    import numpy as np
    nt = int(lib.chol_lu_dag_task_count(T))
    c = np.asarray(cost_ns, dtype=np.int64)
    bl = np.zeros(nt, np.int64)
    _check(lib.chol_lu_dag_bottom_levels(T, c.ctypes.data, bl.ctypes.data), "chol_lu_dag_bottom_levels")
    return bl


def dag_bottom_levels(T, cost_ns):
    import numpy as np
    nt = int(lib.chol_dag_task_count(T))
    c = np.asarray(cost_ns, dtype=np.int64)
    bl = np.zeros(nt, np.int64)
    _check(lib.chol_dag_bottom_levels(T, c.ctypes.data, bl.ctypes.data), "chol_dag_bottom_levels")
    return bl


def _sched_arrays(tasks):
    import numpy as np
    m = len(tasks)
    tid = np.array([t["tid"] for t in tasks], np.int32)
    p = np.array([t["p"] for t in tasks], np.int64)
    prio = np.array([t["prio"] for t in tasks], np.int64)
    aff = np.array([t["aff"] for t in tasks], np.int32)
    score = np.array([t["score"] for t in tasks], np.int64)
    comm = np.array([t.get("comm", 0) for t in tasks], np.int64)
    own = np.array([(list(t.get("own", [])) + [-1, -1, -1])[:3] for t in tasks], np.int32).reshape(-1)
    nin = np.array([t.get("nin", 0) for t in tasks], np.int32)
    return m, tid, p, prio, aff, score, comm, own, nin


def sched_activate(policy, tasks, load, alpha=0.5, max_iter=16, eps=0.01, use_cp=False):
    """Host placement (same code as the device). Returns ([(tid, worker)], iterations)."""
    import numpy as np
    m, tid, p, prio, aff, score, comm, own, nin = _sched_arrays(tasks)
    ld = np.asarray(load, np.int64)
    ot = np.zeros(max(m, 1), np.int32)
    ow = np.zeros(max(m, 1), np.int32)
    it = ctypes.c_int(0)
    pol = POLICIES[policy] if isinstance(policy, str) else policy
    _check(lib.chol_sched_activate(pol, alpha, max_iter, eps, m, tid.ctypes.data, p.ctypes.data,
                                   prio.ctypes.data, aff.ctypes.data, score.ctypes.data, int(bool(use_cp)),
                                   comm.ctypes.data, own.ctypes.data, nin.ctypes.data, len(ld),
                                   ld.ctypes.data, ot.ctypes.data, ow.ctypes.data, ctypes.byref(it)),
           "chol_sched_activate")
    return [(int(a), int(b)) for a, b in zip(ot[:m], ow[:m])], int(it.value)


def dag_bottom_levels_device(T, cost_ns, lu=False, device="cuda", stream=None):
    """Bottom levels computed by the device kernel that prepares each factor launch
    (int64 CUDA tensor, one entry per task id)."""
    import numpy as np
    count = lib.chol_lu_dag_task_count(T) if lu else lib.chol_dag_task_count(T)
    if count < 1:
        raise ValueError(f"no task graph for T={T}")
    c = np.ascontiguousarray(cost_ns, dtype=np.int64)
    out = torch.empty(int(count), dtype=torch.int64, device=device)
    _check(lib.chol_dag_bottom_levels_device(int(bool(lu)), T, c.ctypes.data, out.data_ptr(), _stream(stream)),
           "chol_dag_bottom_levels_device")
    return out


def sched_activate_device(policy, tasks, load, alpha=0.5, max_iter=16, eps=0.01, device="cuda", use_cp=False):
    """The same placement computed by one warp on the GPU."""
    m, tid, p, prio, aff, score, comm, own, nin = _sched_arrays(tasks)
    t = lambda a: torch.from_numpy(a).to(device)
    dt, dp, dpr, da, ds = t(tid), t(p), t(prio), t(aff), t(score)
    dc, do, dn = t(comm), t(own), t(nin)
    dl = torch.tensor(list(load), dtype=torch.int64, device=device)
    ot = torch.zeros(m, dtype=torch.int32, device=device)
    ow = torch.zeros(m, dtype=torch.int32, device=device)
    it = torch.zeros(1, dtype=torch.int32, device=device)
    pol = POLICIES[policy] if isinstance(policy, str) else policy
    _check(lib.chol_sched_activate_device(pol, alpha, max_iter, eps, m, dt.data_ptr(), dp.data_ptr(),
                                          dpr.data_ptr(), da.data_ptr(), ds.data_ptr(), int(bool(use_cp)),
                                          dc.data_ptr(), do.data_ptr(), dn.data_ptr(), len(load),
                                          dl.data_ptr(), ot.data_ptr(), ow.data_ptr(), it.data_ptr(),
                                          _stream(None)), "chol_sched_activate_device")
    torch.cuda.synchronize()
    return [(int(a), int(b)) for a, b in zip(ot.tolist(), ow.tolist())], int(it.item())


# ----------------------------------------------------------------------------------------
# Derivatives: C ABI wrappers and torch.autograd.Function classes (marshalling only; the
# forward and backward passes run in the library's kernels).

def lower(A, stream=None):
    """Lower triangle of a column-major FP64 CUDA matrix (strict upper part zero)."""
    n = A.shape[0]
    lda = _check_matrix(A, "A")
    out = colmajor(torch.empty(n, n, dtype=torch.float64, device=A.device))
    _check(lib.chol_lower_copy(n, A.data_ptr(), lda, out.data_ptr(), max(1, n), _stream(stream)),
           "chol_lower_copy")
    return out


def cholesky_backward(L, Lbar, stream=None):
    """Abar (symmetric) for the gradient Lbar of the factor L."""
    n = L.shape[0]
    lda = _check_matrix(L, "L")
    out = colmajor(Lbar.detach().to(torch.float64))
    work = _workspace(int(lib.chol_backward_workspace_size(n)), L.device)
    _check(lib.chol_backward(n, L.data_ptr(), lda, out.data_ptr(), max(1, n), work.data_ptr(), work.numel(),
                             _stream(stream)), "chol_backward")
    return out


def solve_backward(L, X, Xbar, stream=None):
    """(Bbar, Lbar) for X = A^-1 B, A = L L^T."""
    n = L.shape[0]
    lda = _check_matrix(L, "L")
    X = colmajor(X.detach()) if X.dim() == 1 or X.stride(0) != 1 else X
    Xbar = colmajor(Xbar.detach().to(torch.float64))
    nrhs = X.shape[1]
    Bbar = colmajor(torch.empty(n, nrhs, dtype=torch.float64, device=L.device))
    Lbar = colmajor(torch.empty(n, n, dtype=torch.float64, device=L.device))
    work = _workspace(int(lib.chol_solve_backward_workspace_size(n, nrhs)), L.device)
    _check(lib.chol_solve_backward(n, nrhs, L.data_ptr(), lda, X.data_ptr(), max(1, n), Xbar.data_ptr(),
                                   max(1, n), Bbar.data_ptr(), max(1, n), Lbar.data_ptr(), max(1, n),
                                   work.data_ptr(), work.numel(), _stream(stream)), "chol_solve_backward")
    return Bbar, Lbar


class _CholeskyFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, nb):
        F = colmajor(A.detach().to(torch.float64))
        factor(F, opts(nb=nb), check=True)
        L = lower(F)
        ctx.save_for_backward(L)
        return L

    @staticmethod
    def backward(ctx, Lbar):
        (L,) = ctx.saved_tensors
        return cholesky_backward(L, Lbar), None


class _CholSolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, B, L):
        vec = B.dim() == 1
        X = colmajor(B.detach().to(torch.float64))
        solve(L, X)
        ctx.save_for_backward(L, X)
        ctx.vec = vec
        return X.reshape(-1) if vec else X

    @staticmethod
    def backward(ctx, Xbar):
        L, X = ctx.saved_tensors
        Bbar, Lbar = solve_backward(L, X, Xbar.reshape(X.shape))
        return (Bbar.reshape(-1) if ctx.vec else Bbar), Lbar


class _SolveSPDFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, nb, recompute):
        vec = B.dim() == 1
        F = colmajor(A.detach().to(torch.float64))
        factor(F, opts(nb=nb), check=True)
        X = colmajor(B.detach().to(torch.float64))
        solve(F, X)
        ctx.vec, ctx.nb, ctx.recompute = vec, nb, recompute
        if recompute:   # keep only A (the caller holds it anyway) and refactor in backward
            ctx.save_for_backward(A, X)
        else:
            ctx.save_for_backward(F, X)
        return X.reshape(-1) if vec else X

    @staticmethod
    def backward(ctx, Xbar):
        M, X = ctx.saved_tensors
        if ctx.recompute:
            F = colmajor(M.detach().to(torch.float64))
            factor(F, opts(nb=ctx.nb), check=True)
        else:
            F = M
        Bbar, Lbar = solve_backward(F, X, Xbar.reshape(X.shape))
        Abar = cholesky_backward(F, Lbar)
        return Abar, (Bbar.reshape(-1) if ctx.vec else Bbar), None, None


def cholesky(A, nb=0):
    """Differentiable lower Cholesky factor of a symmetric positive definite FP64 CUDA matrix."""
    return _CholeskyFn.apply(A, nb)


def cholesky_solve(B, L):
    """Differentiable X = (L L^T)^-1 B."""
    return _CholSolveFn.apply(B, L)


def solve_spd(A, B, nb=0, recompute=False):
    """Differentiable X = A^-1 B for symmetric positive definite A. With recompute=True the
    backward pass refactors A instead of keeping L."""
    return _SolveSPDFn.apply(A, B, nb, recompute)


# ----------------------------------------------------------------------------------------
# Batched factor + solve

class BatchOpts(ctypes.Structure):
    _fields_ = [("workers_per_sm", ctypes.c_int), ("lpt_order", ctypes.c_int), ("wide_panel_min_n", ctypes.c_int)]


class Batch:
    """Device description of a batch: a flat buffer of column-major matrices (lda = n) and
    right-hand sides, with the pointer, order and leading-dimension arrays the C ABI takes."""

    def __init__(self, flat, offsets, orders, rhs_flat=None, rhs_offsets=None):
        self.flat, self.orders = flat, [int(n) for n in orders]
        dev = flat.device
        es = flat.element_size()
        self.batch = len(self.orders)
        self.N = torch.tensor(self.orders, dtype=torch.int32, device=dev)
        self.lda = torch.tensor([max(1, n) for n in self.orders], dtype=torch.int32, device=dev)
        self.A = torch.tensor([flat.data_ptr() + es * o for o in offsets], dtype=torch.int64, device=dev)
        self.offsets = list(offsets)
        self.rhs_flat, self.rhs_offsets = rhs_flat, rhs_offsets
        self.B = None
        if rhs_flat is not None:
            self.B = torch.tensor([rhs_flat.data_ptr() + es * o for o in rhs_offsets], dtype=torch.int64,
                                  device=dev)
        self.info = torch.zeros(self.batch, dtype=torch.int32, device=dev)
        self.work = _workspace(int(lib.chol_batched_workspace_size(self.batch)), dev)

    def matrix(self, m):
        n = self.orders[m]
        return self.flat[self.offsets[m]:self.offsets[m] + n * n].view(n, n).t()

    def rhs(self, m):
        n = self.orders[m]
        return self.rhs_flat[self.rhs_offsets[m]:self.rhs_offsets[m] + n]


def _prec(flat):
    if flat.dtype == torch.float64:
        return 0
    if flat.dtype == torch.float32:
        return 1
    raise ValueError("batched matrices must be float64 or float32")


def posv_batched(batch, bopts=None, stream=None, factor_only=False):
    """Factor every matrix of `batch` in place and (unless factor_only) solve its right-hand
    side in place. Asynchronous; per-matrix info in batch.info."""
    o = bopts if bopts is not None else BatchOpts()
    if bopts is None:
        lib.chol_batch_opts_default(ctypes.byref(o))
    bptr = None if (factor_only or batch.B is None) else batch.B.data_ptr()
    _check(lib.chol_posv_batched(_prec(batch.flat), batch.batch, batch.N.data_ptr(), batch.A.data_ptr(),
                                 batch.lda.data_ptr(), bptr, batch.info.data_ptr(), ctypes.byref(o),
                                 batch.work.data_ptr(), batch.work.numel(), _stream(stream)), "chol_posv_batched")
    return batch.info


def factor_batched(batch, bopts=None, stream=None):
    """Factor every matrix of `batch` in place (no right-hand sides). Asynchronous."""
    o = bopts if bopts is not None else BatchOpts()
    if bopts is None:
        lib.chol_batch_opts_default(ctypes.byref(o))
    _check(lib.chol_factor_batched(_prec(batch.flat), batch.batch, batch.N.data_ptr(), batch.A.data_ptr(),
                                   batch.lda.data_ptr(), batch.info.data_ptr(), ctypes.byref(o),
                                   batch.work.data_ptr(), batch.work.numel(), _stream(stream)), "chol_factor_batched")
    return batch.info


def solve_batched(batch, bopts=None, stream=None):
    """Solve every matrix's right-hand side with the factors already in `batch` (from
    factor_batched). Asynchronous."""
    if batch.B is None:
        raise ValueError("the batch has no right-hand sides")
    o = bopts if bopts is not None else BatchOpts()
    if bopts is None:
        lib.chol_batch_opts_default(ctypes.byref(o))
    _check(lib.chol_solve_batched(_prec(batch.flat), batch.batch, batch.N.data_ptr(), batch.A.data_ptr(),
                                  batch.lda.data_ptr(), batch.B.data_ptr(), batch.info.data_ptr(), ctypes.byref(o),
                                  batch.work.data_ptr(), batch.work.numel(), _stream(stream)), "chol_solve_batched")
    return batch.info


def batched_autotune(batch, scratch, stream=None):
    """Time every launch shape on `batch` (copied into `scratch`, a Batch with the same
    orders) and return (BatchOpts, ms)."""
    best = BatchOpts()
    ms = ctypes.c_float(0.0)
    _check(lib.chol_batched_autotune(_prec(batch.flat), batch.batch, batch.N.data_ptr(), batch.A.data_ptr(),
                                     scratch.A.data_ptr(), batch.lda.data_ptr(), scratch.info.data_ptr(),
                                     scratch.work.data_ptr(), scratch.work.numel(), ctypes.byref(best),
                                     ctypes.byref(ms), _stream(stream)), "chol_batched_autotune")
    return best, float(ms.value)


# ------------------------------------------------------------------------------------------
# tile LU with incremental pivoting (chol_lu_factor / chol_lu_solve)

class LUFactors:
    """What chol_lu_factor leaves: the factored matrix F (in place of A), the pivots and the
    L11 blocks, with the options (tile size) they were made with."""

    def __init__(self, F, piv, lw, o, info):
        self.F, self.piv, self.lw, self.opts, self.info = F, piv, lw, o, info


def lu_workspace_size(n, o=None):
    o = o or opts()
    return int(lib.chol_lu_workspace_size(n, ctypes.byref(o)))


def lu_factor(A, o=None, work=None, stream=None, check=False):
    """Tile LU with incremental pivoting of the column-major float64 CUDA matrix A, in place.
    Returns LUFactors. With check=True the call synchronises and raises on a non-zero info."""
    o = o or opts()
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("A must be square")
    lda = _check_matrix(A, "A")
    npiv, nlw = ctypes.c_longlong(0), ctypes.c_longlong(0)
    _check(lib.chol_lu_aux_size(n, ctypes.byref(o), ctypes.byref(npiv), ctypes.byref(nlw)), "chol_lu_aux_size")
    piv = torch.zeros(max(1, npiv.value), dtype=torch.int32, device=A.device)
    lw = torch.zeros(max(1, nlw.value), dtype=torch.float64, device=A.device)
    if work is None:
        work = _workspace(lu_workspace_size(n, o), A.device)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib.chol_lu_factor(n, A.data_ptr(), lda, piv.data_ptr(), lw.data_ptr(), ctypes.byref(o),
                              work.data_ptr(), work.numel(), info.data_ptr(), _stream(stream)), "chol_lu_factor")
    if check and int(info.item()) != 0:
        raise CholeskyError("chol_lu_factor: info = %d" % int(info.item()))
    return LUFactors(A, piv, lw, o, info)


def lu_solve_workspace_size(n, nrhs, o=None):
    o = o if o is not None else opts()
    return int(lib.chol_lu_solve_workspace_size(n, nrhs, ctypes.byref(o)))


def lu_solve(f, B, work=None, info=None, stream=None, check=False):
    """X = A^{-1} B in place on the column-major float64 CUDA matrix B, from lu_factor's output.
    Returns the device info tensor (0, or CHOL_INFO_TIMEOUT if a bounded wait expired)."""
    n = f.F.shape[0]
    ldb = _check_matrix(B, "B")
    nrhs = B.shape[1]
    need = lu_solve_workspace_size(n, nrhs, f.opts)
    if work is None:
        work = _workspace(need, B.device)
    if info is None:
        info = torch.zeros(1, dtype=torch.int32, device=B.device)
    _check(lib.chol_lu_solve(n, nrhs, f.F.data_ptr(), _check_matrix(f.F, "F"), f.piv.data_ptr(),
                             f.lw.data_ptr(), ctypes.byref(f.opts), B.data_ptr(), ldb, work.data_ptr(),
                             work.numel(), info.data_ptr(), _stream(stream)),
           "chol_lu_solve")
    if check:
        torch.cuda.synchronize()
        if int(info.item()) != 0:
            raise CholeskyError("chol_lu_solve: info %d" % int(info.item()))
    return info

PROBE_KINDS = {"dfma": 0, "mma_m8n8k4": 1, "mma_m16n8k4": 2, "mma_m16n8k8": 3, "mma_m16n8k16": 4,
               "dfma_free_operands": 5, "dfma_smem_tile": 6}


def probe_fp64(kind, blocks, threads=256, iters=1000, out=None, stream=None):
    """Launch one FP64 throughput probe (measurement support: DFMA chains, or one of the
    mma.sync .f64 shapes) on `stream` and return the flops of the launch; time it with CUDA
    events on the same stream."""
    k = PROBE_KINDS[kind] if isinstance(kind, str) else int(kind)
    flops = int(lib.chol_probe_fp64_flops(k, blocks, threads, iters))
    if flops < 0:
        raise CholeskyError("chol_probe_fp64_flops: invalid arguments")
    if out is None:
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
    _check(lib.chol_probe_fp64(k, blocks, threads, iters, out.data_ptr(), _stream(stream)), "chol_probe_fp64")
    return flops
