"""Thin ctypes binding of libeig.so (argument marshalling only).

Names follow include/eig.h.  Tensors are torch tensors (device memory, streams); host
arrays may be numpy arrays.  Every arithmetic step happens inside libeig.so; when the
library is not built, or no CUDA device is present, load() raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libeig.so")
_lib = None

EIG_OK, EIG_EINVAL, EIG_ENOMEM, EIG_ECUDA, EIG_ENOT_CONVERGED, EIG_EBREAKDOWN, EIG_ETIMEOUT, \
    EIG_EDUPLICATE, EIG_EUNSUPPORTED = range(9)
EIG_F64, EIG_F32, EIG_BF16 = 0, 1, 2
EIG_LANCZOS, EIG_BLOCK_LANCZOS, EIG_LOBPCG, EIG_CHEBFILTER, EIG_RMMDIIS, EIG_HYBRID = range(6)
METHODS = {"lanczos": 0, "block_lanczos": 1, "lobpcg": 2, "chebfilter": 3, "rmmdiis": 4, "hybrid": 5}
STORAGE = {"f64": EIG_F64, "f32": EIG_F32, "bf16": EIG_BF16}


class EigError(RuntimeError):
    def __init__(self, status, where):
        lib = _lib
        msg = lib.eig_strerror(status).decode() if lib else str(status)
        extra = lib.eig_last_cuda_error().decode() if (lib and status == EIG_ECUDA) else ""
        super().__init__(f"{where}: {msg} {extra}".strip())
        self.status = status


class CsrUpper(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("val_type", C.c_int), ("on_device", C.c_int)]


class SpmmInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_block", C.c_int), ("col_block", C.c_int),
                ("n_row_blocks", C.c_int64), ("n_col_blocks", C.c_int64), ("n_tiles", C.c_int64),
                ("n_slots", C.c_int64), ("scratch_bytes_per_col", C.c_int64), ("val_type", C.c_int),
                ("layout", C.c_int), ("layout_entries", C.c_int64), ("device_bytes", C.c_int64)]


class Opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxiter", C.c_int), ("front", C.c_int), ("switch_tau", C.c_double),
                ("switch_res", C.c_double), ("switch_after", C.c_int), ("s_max", C.c_int), ("vec_type", C.c_int),
                ("precond", C.c_int), ("rmm_precond", C.c_int), ("precond_floor", C.c_double),
                ("cheb_degree", C.c_int), ("lambda_ub", C.c_double), ("lanczos_maxbasis", C.c_int),
                ("X0", C.c_void_p), ("x0_cols", C.c_int), ("x0_on_device", C.c_int), ("seed", C.c_uint64),
                ("certify", C.c_int), ("timing", C.c_int), ("stream", C.c_void_p), ("trace", C.c_void_p),
                ("trace_cap", C.c_int), ("rmm_maxiter", C.c_int), ("rmm_fallback", C.c_int),
                ("diis_tol", C.c_double), ("lp_params", C.c_void_p), ("switch_gap", C.c_double),
                ("lanczos_keep", C.c_int), ("rmm_decouple", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("converged", C.c_int), ("iterations_front", C.c_int), ("iterations_rmm", C.c_int),
                ("switch_reason", C.c_int), ("spmm_calls", C.c_int64), ("spmv_count", C.c_int64),
                ("last_tau", C.c_double), ("max_relres", C.c_double), ("time_ms_total", C.c_double),
                ("time_ms_spmm", C.c_double), ("time_ms_front", C.c_double), ("time_ms_rmm", C.c_double),
                ("spmm_timed", C.c_int64), ("spmm_bytes", C.c_double), ("trace_rows", C.c_int),
                ("iterations_fallback", C.c_int), ("precond_fallback", C.c_int), ("lp_spmm_calls", C.c_int64),
                ("spmm_calls_by_shape", C.c_int64 * 12), ("spmm_ms_by_shape", C.c_double * 12),
                ("spmm_bytes_by_shape", C.c_double * 12), ("batch_launches", C.c_int64),
                ("batch_products", C.c_int64)]


def stats_dict(stats):
    """eig_stats as a dict (the per-shape arrays as lists)."""
    out = {}
    for k, _ in Stats._fields_:
        v = getattr(stats, k)
        out[k] = list(v) if isinstance(v, C.Array) else v
    return out


_SIGS = {
    "eig_strerror": (C.c_char_p, [C.c_int]),
    "eig_last_cuda_error": (C.c_char_p, []),
    "eig_version": (C.c_char_p, []),
    "eig_launch_count": (C.c_int64, []),
    "eig_spmm_plan_create": (C.c_int, [C.POINTER(CsrUpper), C.c_int, C.c_int, C.c_int, C.c_void_p,
                                       C.POINTER(C.c_void_p)]),
    "eig_spmm_plan_destroy": (None, [C.c_void_p]),
    "eig_spmm_plan_create_ex": (C.c_int, [C.POINTER(CsrUpper), C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                          C.POINTER(C.c_void_p)]),
    "eig_spmm_plan_info": (C.c_int, [C.c_void_p, C.POINTER(SpmmInfo)]),
    "eig_spmm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "eig_spmm_cheb": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                C.c_double, C.c_double, C.c_int, C.c_void_p]),
    "eig_gram": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "eig_gram_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "eig_gram_noalloc_parts": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                         C.c_void_p]),
    "eig_cholqr2": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "eig_small_syev": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "eig_small_rr": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p,
                               C.POINTER(C.c_int), C.c_void_p]),
    "eig_rmm_rr2": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "eig_rmm_diis": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                               C.c_void_p]),
    "eig_default_opts": (None, [C.POINTER(Opts)]),
    "eig_create": (C.c_int, [C.POINTER(CsrUpper), C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "eig_create_ex": (C.c_int, [C.POINTER(CsrUpper), C.c_int, C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "eig_solver_spmm_info": (C.c_int, [C.c_void_p, C.POINTER(SpmmInfo)]),
    "eig_destroy": (None, [C.c_void_p]),
    "eig_solve": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Opts), C.POINTER(Stats)]),
    "eig_ritz": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "eig_lp_param_count": (C.c_int, []),
    "eig_create_ex2": (C.c_int, [C.POINTER(CsrUpper), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                 C.POINTER(C.c_void_p)]),
    "eig_create_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "eig_autotune_cheb": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_int), C.c_void_p,
                                    C.c_void_p]),
    "eig_solve_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                  C.c_void_p]),
    "eig_solve_batch_ex": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                     C.c_void_p, C.c_void_p]),
    "eig_autotune_spmm": (C.c_int, [C.POINTER(CsrUpper), C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                    C.POINTER(C.c_int), C.c_void_p]),
    "eig_lp_sample": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "eig_lp_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_double,
                               C.c_void_p, C.c_void_p]),
    "eig_lp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "eig_lp_grad_workspace_bytes": (C.c_size_t, []),
    "eig_lp_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int,
                              C.c_void_p, C.c_void_p, C.c_void_p]),
    "eig_lp_adam": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double,
                              C.c_double, C.c_double, C.c_void_p]),
}


def library_path():
    return _LIB_PATH


def load_symbols_only(path=None):
    """Load the shared library without touching a GPU (used by the CPU export tests)."""
    lib = C.CDLL(path or _LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def load():
    """The library, for use on a CUDA device.  Raises when it is missing or no GPU is present."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is not built; run __graft_entry__.build() (no CPU fallback)")
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libeig needs a CUDA device (no CPU fallback)")
    torch.cuda.init()
    _lib = load_symbols_only()
    return _lib


def check(status, where):
    if status != EIG_OK:
        raise EigError(status, where)


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    import numpy as np
    return t.ctypes.data_as(C.c_void_p).value if isinstance(t, np.ndarray) else t


def stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def vec_dtype(t):
    import torch
    if t.dtype == torch.float32:
        return EIG_F32
    if t.dtype == torch.float64:
        return EIG_F64
    raise TypeError(f"vector blocks must be float32 or float64, got {t.dtype}")


def csr_struct(rowptr, col, val, storage, n, on_device):
    """eig_csr_upper over numpy (host) or torch (device) arrays; caller keeps the arrays alive."""
    s = CsrUpper()
    s.n = int(n)
    s.nnz = int(col.shape[0])
    s.rowptr = _ptr(rowptr)
    s.col = _ptr(col)
    s.val = _ptr(val)
    s.val_type = STORAGE[storage] if isinstance(storage, str) else int(storage)
    s.on_device = 1 if on_device else 0
    return s


LAYOUTS = {"auto": 0, "mirrored": 1, "half": 2, "csr": 3}


def layout_code(layout):
    """eig_layout value of a layout name (or pass-through of an int)."""
    return LAYOUTS[layout] if isinstance(layout, str) else int(layout)


class SpmmPlan:
    """eig_spmm_plan_create / eig_spmm / eig_spmm_plan_destroy."""

    def __init__(self, H, row_block=0, col_block=0, device_arrays=None, copy=True, layout="auto"):
        lib = load()
        self._keep = None
        if device_arrays is not None:
            rp, cl, vl = device_arrays
            st = csr_struct(rp, cl, vl, H.storage, H.n, True)
            self._keep = device_arrays
        else:
            import numpy as np
            rp, cl, vl = (np.ascontiguousarray(H.rowptr), np.ascontiguousarray(H.col),
                          np.ascontiguousarray(H.val))
            st = csr_struct(rp, cl, vl, H.storage, H.n, False)
        self.n = H.n
        h = C.c_void_p()
        check(lib.eig_spmm_plan_create_ex(C.byref(st), int(row_block), int(col_block), layout_code(layout),
                                          1 if copy else 0, stream_ptr(), C.byref(h)), "eig_spmm_plan_create_ex")
        self._h = h
        self._lib = lib

    def info(self):
        inf = SpmmInfo()
        check(self._lib.eig_spmm_plan_info(self._h, C.byref(inf)), "eig_spmm_plan_info")
        return {k: getattr(inf, k) for k, _ in SpmmInfo._fields_}

    def spmm(self, X, Y=None, stream=None):
        import torch
        assert X.is_cuda and X.is_contiguous() and X.dim() == 2 and X.shape[0] == self.n
        if Y is None:
            Y = torch.empty_like(X)
        check(self._lib.eig_spmm(self._h, _ptr(X), _ptr(Y), int(X.shape[1]), vec_dtype(X), stream_ptr(stream)),
              "eig_spmm")
        return Y

    def spmm_cheb(self, X, alpha, c, Qp=None, active=None, Y=None, stream=None):
        """eig_spmm_cheb: Y = alpha (H X - c X) - Qp (Qp None: first step), Y = X on inactive
        columns (active: torch int32 on the device, default all active)."""
        import torch
        assert X.is_cuda and X.is_contiguous() and X.dim() == 2 and X.shape[0] == self.n
        if Y is None:
            Y = torch.empty_like(X)
        if active is None:
            active = torch.ones(X.shape[1], dtype=torch.int32, device=X.device)
        check(self._lib.eig_spmm_cheb(self._h, _ptr(X), _ptr(Y), int(X.shape[1]), vec_dtype(X),
                                      None if Qp is None else _ptr(Qp), _ptr(active), float(alpha), float(c),
                                      1 if Qp is None else 0, stream_ptr(stream)), "eig_spmm_cheb")
        return Y

    def close(self):
        if getattr(self, "_h", None):
            self._lib.eig_spmm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------------------
# step-level calls (device tensors)
# ---------------------------------------------------------------------------------------
def gram(A, B):
    """G = A^T B (FP64 nb x nb) through eig_gram."""
    import torch
    lib = load()
    assert A.shape == B.shape and A.dtype == B.dtype and A.is_contiguous() and B.is_contiguous()
    G = torch.empty(A.shape[1], A.shape[1], dtype=torch.float64, device=A.device)
    check(lib.eig_gram(_ptr(A), _ptr(B), A.shape[0], A.shape[1], vec_dtype(A), _ptr(G), stream_ptr()), "eig_gram")
    return G


def gram_noalloc(A, B, max_parts=None):
    """G = A^T B through eig_gram_noalloc (no device allocation; scratch in a fixed device array);
    max_parts caps the CTA partials (eig_gram_noalloc_parts)."""
    import torch
    lib = load()
    assert A.shape == B.shape and A.dtype == B.dtype and A.is_contiguous() and B.is_contiguous()
    G = torch.empty(A.shape[1], A.shape[1], dtype=torch.float64, device=A.device)
    if max_parts is None:
        check(lib.eig_gram_noalloc(_ptr(A), _ptr(B), A.shape[0], A.shape[1], vec_dtype(A), _ptr(G), stream_ptr()),
              "eig_gram_noalloc")
    else:
        check(lib.eig_gram_noalloc_parts(_ptr(A), _ptr(B), A.shape[0], A.shape[1], vec_dtype(A), _ptr(G),
                                         int(max_parts), stream_ptr()), "eig_gram_noalloc_parts")
    return G


def cholqr2(X):
    """In-place CholeskyQR2: returns (Q (= X), R)."""
    import torch
    lib = load()
    assert X.is_contiguous()
    R = torch.empty(X.shape[1], X.shape[1], dtype=torch.float64, device=X.device)
    check(lib.eig_cholqr2(_ptr(X), X.shape[0], X.shape[1], vec_dtype(X), _ptr(R), stream_ptr()), "eig_cholqr2")
    return X, R


def small_syev(A, m):
    import torch
    lib = load()
    k = A.shape[0]
    w = torch.empty(m, dtype=torch.float64, device=A.device)
    Z = torch.empty(k, m, dtype=torch.float64, device=A.device)
    check(lib.eig_small_syev(_ptr(A.contiguous()), k, m, _ptr(w), _ptr(Z), stream_ptr()), "eig_small_syev")
    return w, Z


def small_rr(A, G, nb, piv_tol=1e-13):
    import torch
    lib = load()
    k = A.shape[0]
    th = torch.empty(nb, dtype=torch.float64, device=A.device)
    Cm = torch.empty(k, nb, dtype=torch.float64, device=A.device)
    info = C.c_int(0)
    check(lib.eig_small_rr(_ptr(A.contiguous()), _ptr(G.contiguous()), k, nb, float(piv_tol), _ptr(th), _ptr(Cm),
                           C.byref(info), stream_ptr()), "eig_small_rr")
    return th, Cm, info.value


def rmm_rr2(dots, active):
    import torch
    lib = load()
    m = dots.shape[0]
    th = torch.empty(m, dtype=torch.float64, device=dots.device)
    g = torch.empty(m, 2, dtype=torch.float64, device=dots.device)
    check(lib.eig_rmm_rr2(_ptr(dots.contiguous()), _ptr(active), m, _ptr(th), _ptr(g), stream_ptr()), "eig_rmm_rr2")
    return th, g


def rmm_diis(B, slots, active):
    import torch
    lib = load()
    m = B.shape[0]
    alpha = torch.empty(m, 20, dtype=torch.float64, device=B.device)
    arr = (C.c_int * len(slots))(*slots)
    check(lib.eig_rmm_diis(_ptr(B.contiguous()), arr, len(slots), _ptr(active), m, _ptr(alpha), stream_ptr()),
          "eig_rmm_diis")
    return alpha


# ---------------------------------------------------------------------------------------
# solver handle
# ---------------------------------------------------------------------------------------
def _make_opts(lib, X0, opts, n_ev, stream=True):
    """eig_opts from keyword options (vec_type as 'f32'/'f64', front as a method name, lp_params a
    parameter vector, X0 numpy (host) or torch (device) FP64 n x k); returns (opts, arrays to keep
    alive while the call runs, trace buffer or None)."""
    import numpy as np
    o = Opts()
    lib.eig_default_opts(C.byref(o))
    keeps = []
    for k, v in opts.items():
        if k == "lp_params":
            lp = np.ascontiguousarray(v, dtype=np.float32)
            assert lp.shape == (N_LP_PARAMS,), lp.shape
            o.lp_params = lp.ctypes.data_as(C.c_void_p).value
            keeps.append(lp)
            continue
        if k == "vec_type":
            v = STORAGE[v] if isinstance(v, str) else v
        if k == "front":
            v = METHODS[v] if isinstance(v, str) else v
        setattr(o, k, v)
    if X0 is not None:
        if hasattr(X0, "data_ptr"):
            assert X0.dtype.is_floating_point and X0.element_size() == 8 and X0.is_contiguous()
            o.X0 = X0.data_ptr()
            o.x0_on_device = 1
            keep = X0
        else:
            keep = np.ascontiguousarray(X0, dtype=np.float64)
            o.X0 = keep.ctypes.data_as(C.c_void_p).value
            o.x0_on_device = 0
        keeps.append(keep)
        o.x0_cols = int(keep.shape[1])
    if stream and not o.stream:
        o.stream = stream_ptr()
    tr = None
    if opts.get("trace_cap", 0):
        tr = np.zeros((int(opts["trace_cap"]), 2 + 2 * n_ev))
        o.trace = tr.ctypes.data_as(C.c_void_p).value
        keeps.append(tr)
    return o, keeps, tr


class Solver:
    """eig_create / eig_solve / eig_ritz / eig_destroy."""

    def __init__(self, H, n_ev, block, layout="auto", row_block=0, col_block=0):
        import numpy as np
        self._lib = lib = load()
        rp, cl, vl = (np.ascontiguousarray(H.rowptr), np.ascontiguousarray(H.col), np.ascontiguousarray(H.val))
        st = csr_struct(rp, cl, vl, H.storage, H.n, False)
        h = C.c_void_p()
        check(lib.eig_create_ex2(C.byref(st), int(n_ev), int(block), layout_code(layout), int(row_block),
                                 int(col_block), C.byref(h)), "eig_create_ex2")
        self._h = h
        self.n, self.n_ev = H.n, n_ev

    def spmm_info(self):
        """eig_solver_spmm_info as a dict (layout, tiles, device bytes of the SpMM plan)."""
        inf = SpmmInfo()
        check(self._lib.eig_solver_spmm_info(self._h, C.byref(inf)), "eig_solver_spmm_info")
        return {k: getattr(inf, k) for k, _ in SpmmInfo._fields_}

    def solve(self, method="hybrid", X0=None, **opts):
        """Runs a method; returns (status, stats dict).  X0: numpy (host) or torch (device) FP64
        n x k array.  Keyword options map to eig_opts fields (vec_type as 'f32'/'f64',
        front as a method name)."""
        import numpy as np
        o, keeps, tr = _make_opts(self._lib, X0, opts, self.n_ev)
        stats = Stats()
        rc = self._lib.eig_solve(self._h, METHODS[method] if isinstance(method, str) else int(method), C.byref(o),
                                 C.byref(stats))
        del keeps
        if rc not in (EIG_OK, EIG_ENOT_CONVERGED, EIG_EDUPLICATE):
            raise EigError(rc, "eig_solve")
        st = stats_dict(stats)
        if tr is not None:
            st["trace"] = tr[: stats.trace_rows].copy()
        return rc, st

    def ritz(self, X_on_device=False, out=None):
        """(theta[n_ev], X (n x n_ev FP64; numpy or torch), relres[n_ev]).  out: a C-contiguous
        FP64 host array (n x n_ev) to receive X (e.g. in page-locked memory)."""
        import numpy as np
        th = np.zeros(self.n_ev)
        rel = np.zeros(self.n_ev)
        if X_on_device:
            import torch
            X = torch.empty(self.n, self.n_ev, dtype=torch.float64, device="cuda")
            check(self._lib.eig_ritz(self._h, _ptr(th), _ptr(X), _ptr(rel), 1), "eig_ritz")
        else:
            if out is not None:
                assert out.dtype == np.float64 and out.shape == (self.n, self.n_ev) and out.flags.c_contiguous
                X = out
            else:
                X = np.zeros((self.n, self.n_ev))
            check(self._lib.eig_ritz(self._h, _ptr(th), _ptr(X), _ptr(rel), 0), "eig_ritz")
        return th, X, rel

    def lp_sample(self, X, theta, Xstar=None, target=0, floor=2.0):
        """eig_lp_sample: training sample of the learned preconditioner from Ritz pairs (X: torch
        FP64 n x m on the device, theta: m values; Xstar: torch FP64 n x k, for target 0).  Returns a
        dict of device tensors F (n*m x 6), r, z (n*m) FP32 and colw (m) FP64."""
        import numpy as np
        import torch
        n, m = X.shape
        assert X.dtype == torch.float64 and X.is_contiguous()
        th = np.ascontiguousarray(theta, dtype=np.float64)
        F = torch.empty(n * m, 6, dtype=torch.float32, device=X.device)
        r = torch.empty(n * m, dtype=torch.float32, device=X.device)
        z = torch.empty(n * m, dtype=torch.float32, device=X.device)
        colw = torch.empty(m, dtype=torch.float64, device=X.device)
        k = 0 if Xstar is None else int(Xstar.shape[1])
        check(self._lib.eig_lp_sample(self._h, X.data_ptr(), m, _ptr(th), None if Xstar is None else Xstar.data_ptr(),
                                      k, int(target), float(floor), F.data_ptr(), r.data_ptr(), z.data_ptr(),
                                      colw.data_ptr(), stream_ptr()), "eig_lp_sample")
        return dict(F=F, r=r, z=z, colw=colw, n=n, m=m)

    def lp_apply(self, params, R, theta, floor=2.0, W=None):
        """eig_lp_apply: W = K^{-1} R with the learned K (params: numpy FP32 vector)."""
        import numpy as np
        import torch
        p = np.ascontiguousarray(params, dtype=np.float32)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        if W is None:
            W = torch.empty_like(R)
        check(self._lib.eig_lp_apply(self._h, _ptr(p), R.data_ptr(), int(R.shape[1]), vec_dtype(R), _ptr(th),
                                     float(floor), W.data_ptr(), stream_ptr()), "eig_lp_apply")
        return W

    def close(self):
        if getattr(self, "_h", None):
            self._lib.eig_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------------------
# learned preconditioner: network kernels
# ---------------------------------------------------------------------------------------
N_LP_PARAMS = 1325
N_LP_TRAINED = 1313


def lp_forward(params, F):
    """eig_lp_forward: m for the feature rows F (torch FP32 count x 6 on the device)."""
    import numpy as np
    import torch
    p = np.ascontiguousarray(params, dtype=np.float32)
    out = torch.empty(F.shape[0], dtype=torch.float32, device=F.device)
    check(load().eig_lp_forward(_ptr(p), F.data_ptr(), int(F.shape[0]), out.data_ptr(), stream_ptr()),
          "eig_lp_forward")
    return out


def lp_grad(params_dev, sample, grad=None, workspace=None):
    """eig_lp_grad on a sample from Solver.lp_sample; params_dev: torch FP32 vector on the device.
    Returns the device FP64 vector [dL/dparams[12:], L]."""
    import torch
    lib = load()
    dev = params_dev.device
    if grad is None:
        grad = torch.empty(N_LP_TRAINED + 1, dtype=torch.float64, device=dev)
    if workspace is None:
        workspace = torch.empty(lib.eig_lp_grad_workspace_bytes(), dtype=torch.uint8, device=dev)
    check(lib.eig_lp_grad(params_dev.data_ptr(), sample["F"].data_ptr(), sample["r"].data_ptr(),
                          sample["z"].data_ptr(), sample["colw"].data_ptr(), int(sample["n"]), int(sample["m"]),
                          grad.data_ptr(), workspace.data_ptr(), stream_ptr()), "eig_lp_grad")
    return grad


def lp_adam(params_dev, grad, m1, m2, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """eig_lp_adam: one Adam step on params_dev (device FP32, in place)."""
    check(load().eig_lp_adam(params_dev.data_ptr(), grad.data_ptr(), m1.data_ptr(), m2.data_ptr(), int(t),
                             float(lr), float(beta1), float(beta2), float(eps), stream_ptr()), "eig_lp_adam")


# ---------------------------------------------------------------------------------------
# batches of instances, SpMM plan autotuner
# ---------------------------------------------------------------------------------------
class TuneResult(C.Structure):
    _fields_ = [("layout", C.c_int), ("row_block", C.c_int), ("col_block", C.c_int), ("ms", C.c_double)]


LAYOUT_NAMES = {v: k for k, v in LAYOUTS.items()}


def solve_batch(solvers, method="hybrid", X0s=None, opts=None, threads=0, lockstep=False):
    """eig_solve_batch_ex over Solver objects; X0s: list (per instance) or None; opts: one dict for
    all or a list of dicts.  Instances without a stream run on the batch's worker streams.
    lockstep: the running instances' products are launched together (EIG_BATCH_LOCKSTEP).
    Returns (status of the batch, [status], [stats dict])."""
    lib = load()
    cnt = len(solvers)
    per = isinstance(opts, (list, tuple)) or X0s is not None
    arr = (Opts * max(cnt, 1))()
    keeps = []
    for i in range(cnt if per else 1):
        od = dict(opts[i] if isinstance(opts, (list, tuple)) else (opts or {}))
        o, kp, _ = _make_opts(lib, None if X0s is None else X0s[i], od, solvers[i].n_ev, stream=False)
        arr[i] = o
        keeps.append(kp)
    hs = (C.c_void_p * max(cnt, 1))(*[s_._h for s_ in solvers])
    st = (C.c_int * max(cnt, 1))()
    stats = (Stats * max(cnt, 1))()
    import torch
    torch.cuda.synchronize()
    rc = lib.eig_solve_batch_ex(hs, cnt, METHODS[method] if isinstance(method, str) else int(method), arr,
                                1 if per else 0, int(threads), 1 if lockstep else 0, st, stats)
    del keeps
    out = [stats_dict(stats[i]) for i in range(cnt)]
    return rc, [int(st[i]) for i in range(cnt)], out


def autotune_spmm(H, nb, vec_type="f32", reps=5):
    """eig_autotune_spmm: the fastest SpMM plan shape for H with an nb-column block.  Returns
    (best, all) as dicts {layout, row_block, col_block, ms}."""
    import numpy as np
    lib = load()
    rp, cl, vl = (np.ascontiguousarray(H.rowptr), np.ascontiguousarray(H.col), np.ascontiguousarray(H.val))
    st = csr_struct(rp, cl, vl, H.storage, H.n, False)
    best = TuneResult()
    allr = (TuneResult * 8)()
    na = C.c_int(0)
    check(lib.eig_autotune_spmm(C.byref(st), int(nb), STORAGE[vec_type] if isinstance(vec_type, str) else vec_type,
                                int(reps), C.byref(best), allr, C.byref(na), stream_ptr()), "eig_autotune_spmm")

    def d(r):
        return {"layout": LAYOUT_NAMES.get(r.layout, r.layout), "row_block": r.row_block, "col_block": r.col_block,
                "ms": r.ms}
    return d(best), [d(allr[i]) for i in range(na.value)]


def create_batch(Hs, n_ev, block, layout="auto"):
    """eig_create_batch: Solver objects for the matrices Hs (all created, or none and an error)."""
    import numpy as np
    lib = load()
    arrs = [(np.ascontiguousarray(H.rowptr), np.ascontiguousarray(H.col), np.ascontiguousarray(H.val)) for H in Hs]
    sts = (CsrUpper * max(len(Hs), 1))()
    for i, (H, (rp, cl, vl)) in enumerate(zip(Hs, arrs)):
        sts[i] = csr_struct(rp, cl, vl, H.storage, H.n, False)
    hs = (C.c_void_p * max(len(Hs), 1))()
    check(lib.eig_create_batch(sts, len(Hs), int(n_ev), int(block), layout_code(layout), hs), "eig_create_batch")
    out = []
    for i, H in enumerate(Hs):
        S = Solver.__new__(Solver)
        S._lib, S._h, S.n, S.n_ev = lib, C.c_void_p(hs[i]), H.n, n_ev
        out.append(S)
    return out


def autotune_cheb(solver, degrees, X0=None, **opts):
    """eig_autotune_cheb: the Chebyshev degree with the fastest converged ChebFSI solve on this
    solver's matrix.  Returns (best degree or 0, [ms per degree], [converged per degree])."""
    import numpy as np
    lib = load()
    o, keeps, _ = _make_opts(lib, X0, opts, solver.n_ev)
    d = np.ascontiguousarray(degrees, dtype=np.int32)
    ms = np.zeros(d.size)
    cv = np.zeros(d.size, dtype=np.int32)
    best = C.c_int(0)
    rc = lib.eig_autotune_cheb(solver._h, _ptr(d), int(d.size), C.byref(o), C.byref(best), _ptr(ms), _ptr(cv))
    del keeps
    if rc not in (EIG_OK, EIG_ENOT_CONVERGED):
        raise EigError(rc, "eig_autotune_cheb")
    return best.value, ms.tolist(), cv.tolist()
