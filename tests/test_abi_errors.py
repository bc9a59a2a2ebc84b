"""CPU: the C ABI's documented argument checks and defaults, through the symbols of libeig.so.

Every call here is one that include/eig.h says returns EIG_EINVAL for bad arguments before
anything is launched (or a pure host function), so none of them needs a GPU: the library is
loaded without initialising CUDA, as in the export test.
"""
import ctypes as C

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2305_15552_gb300 import build, binding
    try:
        path = build.build()
    except RuntimeError as e:
        pytest.fail(f"build failed: {e}")
    return binding.load_symbols_only(path)


@pytest.fixture(scope="module")
def b():
    from paper_2305_15552_gb300 import binding
    return binding


def test_strerror_names_every_status(lib, b):
    names = ["EIG_OK", "EIG_EINVAL", "EIG_ENOMEM", "EIG_ECUDA", "EIG_ENOT_CONVERGED", "EIG_EBREAKDOWN",
             "EIG_ETIMEOUT", "EIG_EDUPLICATE", "EIG_EUNSUPPORTED"]
    for code, name in enumerate(names):
        assert lib.eig_strerror(code).decode().split(":")[0] == name
    assert lib.eig_strerror(len(names)).decode() == "unknown eig_status"


def test_default_opts_are_the_documented_ones(lib, b):
    """Defaults stated in eig.h: tol 1e-6 (Sec. 3.2), maxiter 500, LOBPCG front, tau rule at 1e-7,
    DIIS window 10, FP32 vectors, Jacobi K floored at 2.0, Chebyshev degree 10, no learned K, the
    safety net on, certification on, gap condition / thick-restart / decoupling at their defaults."""
    o = b.Opts()
    C.memset(C.byref(o), 0xFF, C.sizeof(o))        # every field is written, none kept
    lib.eig_default_opts(C.byref(o))
    assert o.tol == 1e-6 and o.maxiter == 500 and o.front == b.EIG_LOBPCG
    assert o.switch_tau == 1e-7 and o.switch_res == 0.0 and o.switch_after == 0 and o.switch_gap == 0.0
    assert o.s_max == 10 and o.vec_type == b.EIG_F32
    assert o.precond == 1 and o.rmm_precond == 0 and o.precond_floor == 2.0
    assert o.cheb_degree == 10 and o.lambda_ub == 0.0 and o.lanczos_maxbasis == 600
    assert o.lanczos_keep == 0 and o.rmm_decouple == 0
    assert not o.X0 and o.x0_cols == 0 and not o.stream and not o.lp_params
    assert o.certify == 1 and o.timing == 0 and o.rmm_fallback == 1 and o.rmm_maxiter == 0
    assert o.diis_tol == 0.0


def _csr(b, n=10):
    h = b.CsrUpper()
    h.n, h.nnz, h.val_type, h.on_device = n, n, b.EIG_F64, 0
    return h


@pytest.mark.parametrize("n_ev,block,layout", [(0, 4, 0), (5, 4, 0), (4, 33, 0), (11, 16, 0), (2, 4, 99),
                                               (2, 4, -1)])
def test_create_rejects_bad_sizes(lib, b, n_ev, block, layout):
    """eig_create: EIG_EINVAL for n_ev < 1, n_ev > block, block > 32, n_ev > n or an unknown
    layout, and the handle is left NULL."""
    h = C.c_void_p(1)
    H = _csr(b)
    assert lib.eig_create_ex2(C.byref(H), n_ev, block, layout, 0, 0, C.byref(h)) == b.EIG_EINVAL
    assert not h.value


def test_create_rejects_null_pointers(lib, b):
    H = _csr(b)
    assert lib.eig_create_ex2(None, 2, 4, 0, 0, 0, C.byref(C.c_void_p())) == b.EIG_EINVAL
    assert lib.eig_create_ex2(C.byref(H), 2, 4, 0, 0, 0, None) == b.EIG_EINVAL


def _bad_opts(b, lib, **kw):
    o = b.Opts()
    lib.eig_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize("kw", [dict(tol=0.0), dict(tol=-1.0), dict(maxiter=-1), dict(s_max=0), dict(s_max=21),
                                dict(vec_type=2), dict(precond=3), dict(rmm_precond=-1), dict(precond=2),
                                dict(rmm_precond=2)])
def test_solve_rejects_bad_options_before_touching_the_handle(lib, b, kw):
    """eig_solve validates the options first: a bad tolerance, iteration limit, DIIS window
    (1..20, Eqs. xsum-rmm), vector type or preconditioner (a learned K without parameters) is
    EIG_EINVAL, whatever the handle."""
    o = _bad_opts(b, lib, **kw)
    st = b.Stats()
    assert lib.eig_solve(C.c_void_p(1), b.EIG_HYBRID, C.byref(o), C.byref(st)) == b.EIG_EINVAL


def test_solve_rejects_start_block_without_columns(lib, b):
    x = (C.c_double * 4)()
    o = _bad_opts(b, lib)
    o.X0 = C.cast(x, C.c_void_p).value
    o.x0_cols = 0
    assert lib.eig_solve(C.c_void_p(1), b.EIG_LOBPCG, C.byref(o), None) == b.EIG_EINVAL


def test_null_handles(lib, b):
    assert lib.eig_solve(None, b.EIG_LOBPCG, None, None) == b.EIG_EINVAL
    assert lib.eig_ritz(None, None, None, None, 0) == b.EIG_EINVAL
    assert lib.eig_spmm(None, C.c_void_p(16), C.c_void_p(16), 8, b.EIG_F32, None) == b.EIG_EINVAL
    assert lib.eig_spmm(C.c_void_p(16), None, C.c_void_p(16), 8, b.EIG_F32, None) == b.EIG_EINVAL


def test_plan_create_rejects_unknown_layout(lib, b):
    H = _csr(b)
    p = C.c_void_p(1)
    assert lib.eig_spmm_plan_create_ex(C.byref(H), 0, 0, 99, 1, None, C.byref(p)) == b.EIG_EINVAL
    assert not p.value
    assert lib.eig_spmm_plan_create_ex(C.byref(H), 0, 0, 0, 1, None, None) == b.EIG_EINVAL


@pytest.mark.parametrize("n,nb,vt", [(0, 8, 1), (100, 0, 1), (100, 65, 1), (100, 8, 2), (100, 8, 7)])
def test_gram_rejects_bad_sizes(lib, b, n, nb, vt):
    """eig_gram: n >= 1, 1 <= nb <= 64, FP32 or FP64 blocks (Eq. rreig's Grams)."""
    p = C.c_void_p(256)
    assert lib.eig_gram(p, p, n, nb, vt, p, None) == b.EIG_EINVAL


def test_gram_rejects_null_pointers(lib, b):
    p = C.c_void_p(256)
    assert lib.eig_gram(None, p, 100, 8, b.EIG_F32, p, None) == b.EIG_EINVAL
    assert lib.eig_gram(p, p, 100, 8, b.EIG_F32, None, None) == b.EIG_EINVAL


@pytest.mark.parametrize("nb,parts", [(33, 512), (8, 0), (8, 513), (0, 64)])
def test_gram_noalloc_rejects_what_its_fixed_array_cannot_hold(lib, b, nb, parts):
    """The no-alloc Gram holds 512 partials of a 32 x 32 Gram: nb <= 32 and 1..512 partials."""
    p = C.c_void_p(256)
    assert lib.eig_gram_noalloc_parts(p, p, 100, nb, b.EIG_F32, p, parts, None) == b.EIG_EINVAL


@pytest.mark.parametrize("n,k", [(0, 4), (10, 0), (10, 65), (3, 4)])
def test_cholqr2_rejects_bad_sizes(lib, b, n, k):
    """CholQR2 of an n x k block needs 1 <= k <= 64 and n >= k."""
    p = C.c_void_p(256)
    assert lib.eig_cholqr2(p, n, k, b.EIG_F32, p, None) == b.EIG_EINVAL
