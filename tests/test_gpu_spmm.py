"""GPU parity of the symmetric half-stored SpMM (Y = H X, Sec. 1 / Eqs. upd1-upd2) against the
FP64 oracle, through the C ABI, for every device layout of the plan (mirrored tiles, half-stored
tiles, CSR)."""
import numpy as np
import pytest

import oracle as O
from gen import ci_matrix, laplacian_kron, diagonal_matrix, CSRUpper

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _plan(H, **kw):
    from paper_2305_15552_gb300.binding import SpmmPlan
    return SpmmPlan(H, **kw)


def _tol(H, X, Y_ref, dtype):
    """Elementwise bound: k * eps * (|H| |X|)_i, k = 2 * max row length (sum + products).
    FP64 vectors with FP32/BF16 values are summed in double-float (two FP32 words): unit
    roundoff 2^-44 per step instead of FP64's 2^-53."""
    absH = CSRUpper(H.n, H.rowptr, H.col, np.abs(H.values_f64()), "f64")
    bound = O.sym_upper_matmul(absH, np.abs(X))
    rowlen = np.diff(H.rowptr).max() * 2 + 2
    if dtype == torch.float32:
        eps = 2.0 ** -24
    else:
        eps = 2.0 ** -53 if H.storage == "f64" else 2.0 ** -44
    return rowlen * eps * bound + 1e-300


LAYOUTS = ["mirrored", "half", "csr"]


def _check(H, nb, dtype, seed=0, R=0, Cb=0, layout="auto", misalign=False):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((H.n, nb))
    Xt = torch.tensor(X, dtype=dtype, device="cuda")
    if misalign:
        # same values `misalign` elements past a 16-byte boundary
        buf = torch.empty(H.n * nb + misalign, dtype=dtype, device="cuda")
        buf[misalign:] = Xt.reshape(-1)
        Xt = buf[misalign:].view(H.n, nb)
        assert Xt.data_ptr() % 16 != 0
    Xe = Xt.double().cpu().numpy()
    P = _plan(H, row_block=R, col_block=Cb, layout=layout)
    Y = P.spmm(Xt)
    torch.cuda.synchronize()
    Yr = O.sym_upper_matmul(H, Xe)
    err = np.abs(Y.double().cpu().numpy() - Yr)
    tol = _tol(H, Xe, Yr, dtype)
    assert np.all(err <= tol), f"max err {err.max()} (tol at argmax {tol.ravel()[err.argmax()]})"
    # bitwise determinism
    Y2 = P.spmm(Xt)
    assert torch.equal(Y, Y2)
    P.close()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("nb", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("storage,dtype", [("f32", torch.float32), ("f64", torch.float64), ("f32", torch.float64),
                                            ("bf16", torch.float32), ("bf16", torch.float64)])
def test_ci_ragged(nb, storage, dtype, layout):
    H = ci_matrix(5000 + 37, 100, 64, seed=1, storage=storage)
    _check(H, nb, dtype, layout=layout)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_alignment(layout):
    """X and Y must be aligned to min(16, nb * element size) bytes: smaller offsets are rejected
    before any kernel runs; offsets that keep that alignment run (through plain loads of X_J in
    the mirrored kernel) and agree with the oracle."""
    from paper_2305_15552_gb300 import binding as b
    H = ci_matrix(3000 + 5, 150, 256, seed=3, storage="f32")
    P = _plan(H, layout=layout)
    buf = torch.zeros(H.n * 16 + 4, device="cuda")
    with pytest.raises(b.EigError) as e:
        P.spmm(buf[1:1 + H.n * 16].view(H.n, 16))
    assert e.value.status == b.EIG_EINVAL
    P.close()
    _check(H, 2, torch.float32, layout=layout, misalign=2)     # 8-byte rows at an 8-byte offset
    Hd = ci_matrix(3000 + 5, 150, 256, seed=3, storage="f64")
    _check(Hd, 1, torch.float64, layout=layout, misalign=1)    # 8-byte rows at an 8-byte offset


def test_layout_selection():
    """AUTO picks the mirrored layout at the default blocks; the mirrored layout needs 256 x 64
    tiles, other block sizes get the half-stored layout; every layout reports its bytes."""
    from paper_2305_15552_gb300 import binding as b
    H = ci_matrix(5000, 100, 64, seed=1, storage="f32")
    infos = {}
    for lay in ["auto", "mirrored", "half", "csr"]:
        P = _plan(H, layout=lay)
        infos[lay] = P.info()
        P.close()
    assert infos["auto"]["layout"] == b.LAYOUTS["mirrored"]
    assert infos["mirrored"]["layout"] == b.LAYOUTS["mirrored"]
    assert infos["half"]["layout"] == b.LAYOUTS["half"]
    assert infos["csr"]["layout"] == b.LAYOUTS["csr"]
    nnz_full = 2 * H.nnz - H.n          # every diagonal entry is stored
    assert infos["mirrored"]["layout_entries"] >= nnz_full
    assert infos["half"]["layout_entries"] >= H.nnz
    assert infos["csr"]["layout_entries"] == H.nnz
    P = _plan(H, row_block=128, col_block=64, layout="mirrored")
    assert P.info()["layout"] == b.LAYOUTS["half"]
    P.close()
    with pytest.raises(b.EigError):
        _plan(H, layout=7)


@pytest.mark.parametrize("R,Cb", [(256, 128), (256, 256), (128, 64), (512, 128), (64, 32)])
def test_block_shapes(R, Cb):
    H = ci_matrix(3001, 120, 256, seed=2, storage="f32")
    _check(H, 16, torch.float32, R=R, Cb=Cb)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_laplacian_f64(layout):
    H = laplacian_kron([13, 17, 19])
    _check(H, 8, torch.float64, layout=layout)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_diagonal_only_and_tiny(layout):
    _check(diagonal_matrix(np.linspace(-1, 1, 7)), 4, torch.float64, layout=layout)
    _check(diagonal_matrix(np.linspace(-1, 1, 1000), storage="f32"), 16, torch.float32, layout=layout)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_no_offdiagonal_entries_and_one_row(layout):
    n = 300
    H = CSRUpper(n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0), "f64")
    _check(H, 4, torch.float64, layout=layout)          # H = 0 (no stored entries at all)
    H1 = CSRUpper(1, np.array([0, 1], np.int64), np.array([0], np.int32), np.array([2.5]), "f64")
    _check(H1, 2, torch.float64, layout=layout)


def test_unsupported_type_combination():
    from paper_2305_15552_gb300 import binding
    P = _plan(diagonal_matrix(np.linspace(-1, 1, 100)))        # f64 values
    with pytest.raises(binding.EigError) as e:
        P.spmm(torch.ones(100, 4, device="cuda", dtype=torch.float32))
    assert e.value.status == binding.EIG_EUNSUPPORTED


@pytest.mark.parametrize("layout", LAYOUTS)
def test_empty_rows_and_dense_row(layout):
    n = 700
    rows, cols = [], []
    for i in range(n):
        if i % 7 == 3:
            continue                                   # empty row (no diagonal either)
        js = [i] + ([j for j in range(i + 1, n)] if i == 5 else [j for j in range(i + 1, n, 97)])
        for j in js:
            rows.append(i); cols.append(j)
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    val = np.random.default_rng(3).standard_normal(len(cols))
    H = CSRUpper(n, rowptr, np.array(cols, np.int32), val, "f64")
    H.check()
    _check(H, 8, torch.float64, layout=layout)
    _check(CSRUpper(n, rowptr, np.array(cols, np.int32), val.astype(np.float32), "f32"), 16, torch.float32,
           layout=layout)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_integer_values_bitwise(layout):
    """Small-integer H and X: every FP32 partial sum is exact, so GPU == oracle bitwise."""
    H = ci_matrix(4000, 100, 64, seed=4, storage="f64")
    vals = np.round(H.values_f64() * 10).astype(np.float32)
    Hi = CSRUpper(H.n, H.rowptr, H.col, vals, "f32")
    X = np.random.default_rng(5).integers(-4, 5, size=(H.n, 16)).astype(np.float32)
    P = _plan(Hi, layout=layout)
    Y = P.spmm(torch.tensor(X, device="cuda")).cpu().numpy()
    Yr = O.sym_upper_matmul(Hi, X.astype(np.float64))
    assert np.array_equal(Y.astype(np.float64), Yr)


def test_invalid_csr_rejected():
    from paper_2305_15552_gb300 import binding
    H = ci_matrix(500, 40, 64, seed=1, storage="f32")
    bad = CSRUpper(H.n, H.rowptr, H.col.copy(), H.val, "f32")
    bad.col[H.rowptr[10] + 1] = 3          # below the diagonal of row 10
    with pytest.raises(binding.EigError) as e:
        _plan(bad)
    assert e.value.status == binding.EIG_EINVAL


@pytest.fixture(scope="module")
def bench_matrix():
    return ci_matrix(2_000_000, 400, 256, seed=1, storage="f32")


@pytest.mark.parametrize("layout,nb", [("auto", 16), ("auto", 8), ("half", 16)])
def test_bench_size_sampled_rows(bench_matrix, layout, nb):
    """2M rows, ~400 nnz/row, 256-tiles, FP32 values and vectors (the time-to-solution workload,
    in the layout the solver uses and in the half-stored one): the whole product against the
    oracle on a sample of rows."""
    H = bench_matrix
    rng = np.random.default_rng(7)
    X = rng.standard_normal((H.n, nb)).astype(np.float32)
    P = _plan(H, layout=layout)
    Y = P.spmm(torch.tensor(X, device="cuda")).cpu().numpy()
    rows = np.sort(rng.choice(H.n, 2000, replace=False))
    Yr = O.sym_upper_matmul(H, X.astype(np.float64))
    err = np.abs(Y[rows].astype(np.float64) - Yr[rows])
    absH = CSRUpper(H.n, H.rowptr, H.col, np.abs(H.values_f64()), "f64")
    bound = O.sym_upper_matmul(absH, np.abs(X.astype(np.float64)))[rows]
    assert np.all(err <= 1000 * 2.0 ** -24 * bound + 1e-30)


@pytest.mark.parametrize("storage,dt,nb", [("f32", "f32", 16), ("f32", "f32", 8), ("f64", "f64", 8),
                                           ("f32", "f64", 32)])
def test_spmm_cheb_fused_step_matches_definition(storage, dt, nb):
    """eig_spmm_cheb (Chebyshev step in the SpMM epilogue, Alg. 3) against the oracle's product and
    Eq. (chebypoly) evaluated in FP64: later steps with Qp, the first step without, and locked
    columns copied through."""
    import torch
    from paper_2305_15552_gb300.binding import SpmmPlan
    H = ci_matrix(5003, 120, 64, seed=4, storage=storage)
    P = SpmmPlan(H, layout="mirrored")
    tdt = torch.float32 if dt == "f32" else torch.float64
    rng = np.random.default_rng(3)
    X = rng.standard_normal((H.n, nb))
    Q = rng.standard_normal((H.n, nb))
    Xd, Qd = torch.tensor(X, dtype=tdt, device="cuda"), torch.tensor(Q, dtype=tdt, device="cuda")
    Xr = Xd.double().cpu().numpy()
    Qr = Qd.double().cpu().numpy()
    HX = O.sym_upper_matmul(H, Xr)
    act = np.ones(nb, dtype=np.int32)
    act[1] = 0
    actd = torch.tensor(act, device="cuda")
    alpha, c = 2.0 / 7.5, 3.25
    tol = 3e-6 if dt == "f32" else 1e-12
    Y = P.spmm_cheb(Xd, alpha, c, Qp=Qd, active=actd).double().cpu().numpy()
    want = alpha * (HX - c * Xr) - Qr
    want[:, 1] = Xr[:, 1]
    np.testing.assert_allclose(Y, want, rtol=0, atol=tol * np.abs(want).max())
    assert np.array_equal(Y[:, 1], Xr[:, 1])
    Y1 = P.spmm_cheb(Xd, 1.0 / 7.5, c).double().cpu().numpy()
    np.testing.assert_allclose(Y1, (HX - c * Xr) / 7.5, rtol=0, atol=tol * np.abs(HX).max())
    # equal to the unfused product followed by the elementwise step
    HXg = P.spmm(Xd).double().cpu().numpy()
    Yu = alpha * (HXg - c * Xr) - Qr
    Yu[:, 1] = Xr[:, 1]
    # (the device may contract a multiply-add: a last-bit difference, seen only near cancellation)
    np.testing.assert_allclose(Y, Yu.astype(np.float32 if dt == "f32" else np.float64), rtol=2e-7 if dt == "f32" else 1e-15,
                               atol=(1e-7 if dt == "f32" else 1e-15) * np.abs(Yu).max())
    P.close()
