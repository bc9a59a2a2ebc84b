"""GPU parity of the symmetric half-stored SpMM (Y = H X, Sec. 1 / Eqs. upd1-upd2) against the
FP64 oracle, through the C ABI."""
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
    """Elementwise bound: k * eps * (|H| |X|)_i, k = 2 * max row length (sum + products)."""
    absH = CSRUpper(H.n, H.rowptr, H.col, np.abs(H.values_f64()), "f64")
    bound = O.sym_upper_matmul(absH, np.abs(X))
    rowlen = np.diff(H.rowptr).max() * 2 + 2
    eps = 2.0 ** -24 if dtype == torch.float32 else 2.0 ** -53
    return rowlen * eps * bound + 1e-300


def _check(H, nb, dtype, seed=0, R=0, Cb=0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((H.n, nb))
    Xt = torch.tensor(X, dtype=dtype, device="cuda")
    Xe = Xt.double().cpu().numpy()
    P = _plan(H, row_block=R, col_block=Cb)
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


@pytest.mark.parametrize("nb", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("storage,dtype", [("f32", torch.float32), ("f64", torch.float64), ("f32", torch.float64),
                                            ("bf16", torch.float32)])
def test_ci_ragged(nb, storage, dtype):
    H = ci_matrix(5000 + 37, 100, 64, seed=1, storage=storage)
    _check(H, nb, dtype)


@pytest.mark.parametrize("R,Cb", [(256, 128), (256, 256), (128, 64), (512, 128), (64, 32)])
def test_block_shapes(R, Cb):
    H = ci_matrix(3001, 120, 256, seed=2, storage="f32")
    _check(H, 16, torch.float32, R=R, Cb=Cb)


def test_laplacian_f64():
    H = laplacian_kron([13, 17, 19])
    _check(H, 8, torch.float64)


def test_diagonal_only_and_tiny():
    _check(diagonal_matrix(np.linspace(-1, 1, 7)), 4, torch.float64)
    _check(diagonal_matrix(np.linspace(-1, 1, 1000), storage="f32"), 16, torch.float32)


def test_unsupported_type_combination():
    from paper_2305_15552_gb300 import binding
    P = _plan(diagonal_matrix(np.linspace(-1, 1, 100)))        # f64 values
    with pytest.raises(binding.EigError) as e:
        P.spmm(torch.ones(100, 4, device="cuda", dtype=torch.float32))
    assert e.value.status == binding.EIG_EUNSUPPORTED


def test_empty_rows_and_dense_row():
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
    _check(H, 8, torch.float64)
    _check(CSRUpper(n, rowptr, np.array(cols, np.int32), val.astype(np.float32), "f32"), 16, torch.float32)


def test_integer_values_bitwise():
    """Small-integer H and X: every FP32 partial sum is exact, so GPU == oracle bitwise."""
    H = ci_matrix(4000, 100, 64, seed=4, storage="f64")
    vals = np.round(H.values_f64() * 10).astype(np.float32)
    Hi = CSRUpper(H.n, H.rowptr, H.col, vals, "f32")
    X = np.random.default_rng(5).integers(-4, 5, size=(H.n, 16)).astype(np.float32)
    P = _plan(Hi)
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


def test_bench_size_sampled_rows():
    """2M rows, ~400 nnz/row, 256-tiles, FP32 values and vectors (the time-to-solution workload):
    the whole product against the oracle on a sample of rows."""
    H = ci_matrix(2_000_000, 400, 256, seed=1, storage="f32")
    nb = 16
    rng = np.random.default_rng(7)
    X = rng.standard_normal((H.n, nb)).astype(np.float32)
    P = _plan(H)
    Y = P.spmm(torch.tensor(X, device="cuda")).cpu().numpy()
    rows = np.sort(rng.choice(H.n, 2000, replace=False))
    Yr = O.sym_upper_matmul(H, X.astype(np.float64))
    err = np.abs(Y[rows].astype(np.float64) - Yr[rows])
    absH = CSRUpper(H.n, H.rowptr, H.col, np.abs(H.values_f64()), "f64")
    bound = O.sym_upper_matmul(absH, np.abs(X.astype(np.float64)))[rows]
    assert np.all(err <= 1000 * 2.0 ** -24 * bound + 1e-30)
