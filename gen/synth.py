"""Synthetic stand-ins for the nuclear CI Hamiltonians of Sec. 3.1 (Tables 2 and 3).

The paper's matrices (6Li, 7Li, 11B, 12C with the Daejeon16 interaction) are not
available, so every workload is drawn here from a seeded recipe that keeps their
relevant structure:

* a half-stored symmetric sparse H (upper triangle incl. diagonal, Sec. 3.1: the
  nonzero counts of Tables 2-3 are "in half the symmetric matrices");
* rows sorted by a shell-like level index k whose degeneracy grows quadratically,
  g_k = (k+1)(k+2)/2, with H_ii = k + N(0, sigma_d^2) -- the lowest eigenvalues
  then sit in near-degenerate groups, like the low-lying nuclear states;
* off-diagonal couplings N(0, sigma_o^2) on a seeded block pattern: the matrix is
  cut into B x B tiles, every diagonal tile is active, each upper tile pair (I, J),
  J > I, is active independently with probability p, and inside an active tile each
  position is present with probability rho.  p is set so that the mean full-row
  count (1 + 2 mu) B rho equals the requested nnz/row, mu = p (nblk - 1) / 2.

Values are rounded to the storage type (f64, f32 or bf16) when they are drawn, so
the oracle and the GPU path solve exactly the same matrix.

Nothing here implements a step of an eigensolver.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_STORAGE = ("f64", "f32", "bf16")


def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest even); returns uint16 bit patterns."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    lsb = (u >> 16) & 1
    rounded = (u + np.uint32(0x7FFF) + lsb) >> 16
    return rounded.astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    """Widen bfloat16 bit patterns to float32 (exact)."""
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def round_to_storage(x: np.ndarray, storage: str) -> np.ndarray:
    """Round float64 values to the storage type; returns the storage array
    (float64, float32, or uint16 bfloat16 bit patterns)."""
    if storage == "f64":
        return np.asarray(x, dtype=np.float64)
    if storage == "f32":
        return np.asarray(x, dtype=np.float32)
    if storage == "bf16":
        return f32_to_bf16_bits(np.asarray(x, dtype=np.float32))
    raise ValueError(f"unknown storage type {storage!r}")


@dataclass
class CSRUpper:
    """Upper triangle (incl. diagonal) of a symmetric n x n matrix in CSR form.

    rowptr: int64[n+1]; col: int32[nnz] (sorted, col >= row, no duplicates);
    val: storage array (float64 / float32 / uint16 bf16 bits) of length nnz.
    """
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    storage: str = "f64"
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def values_f64(self) -> np.ndarray:
        if self.storage == "bf16":
            return bf16_bits_to_f32(self.val).astype(np.float64)
        return np.asarray(self.val, dtype=np.float64)

    def values_f32(self) -> np.ndarray:
        if self.storage == "bf16":
            return bf16_bits_to_f32(self.val)
        return np.asarray(self.val, dtype=np.float32)

    def diagonal_f64(self) -> np.ndarray:
        """H_ii (the first entry of every row is the diagonal in this layout when present)."""
        d = np.zeros(self.n)
        first = self.rowptr[:-1]
        has = (self.rowptr[1:] > first)
        idx = first[has]
        rows = np.nonzero(has)[0]
        isdiag = self.col[idx] == rows
        d[rows[isdiag]] = self.values_f64()[idx[isdiag]]
        return d

    def check(self) -> None:
        n = self.n
        assert self.rowptr.dtype == np.int64 and self.col.dtype == np.int32
        assert self.rowptr.shape == (n + 1,) and self.rowptr[0] == 0
        assert np.all(np.diff(self.rowptr) >= 0)
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(self.rowptr))
        assert np.all(self.col >= rows), "entry below the diagonal"
        assert np.all(self.col < n)
        # strictly increasing within rows
        same = rows[1:] == rows[:-1]
        assert np.all(np.diff(self.col.astype(np.int64))[same] > 0), "unsorted or duplicate column"


def ci_levels(n: int) -> np.ndarray:
    """Level index k of each row: rows sorted by level, level k holds (k+1)(k+2)/2 rows."""
    lev = np.empty(n, dtype=np.int64)
    start, k = 0, 0
    while start < n:
        g = (k + 1) * (k + 2) // 2
        lev[start:min(n, start + g)] = k
        start += g
        k += 1
    return lev


def ci_matrix(n: int, nnz_per_row: float, block: int, seed: int, storage: str = "f32",
              rho: float = 0.25, sigma_diag: float = 0.05, sigma_off: float = 0.1,
              chunk_rows: int = 1 << 16) -> CSRUpper:
    """Seeded CI-shaped half-stored symmetric matrix (recipe in the module docstring).

    nnz_per_row is the mean number of nonzeros of a FULL row (both triangles).
    """
    if storage not in _STORAGE:
        raise ValueError(storage)
    B = int(block)
    nblk = (n + B - 1) // B
    thr = int(round(rho * 256))
    rho_q = thr / 256.0
    mu = max(0.0, (nnz_per_row / (B * rho_q) - 1.0) / 2.0)
    p = min(1.0, 2.0 * mu / (nblk - 1)) if nblk > 1 else 0.0

    ss = np.random.SeedSequence([int(seed), n, B, int(round(nnz_per_row * 1000)), thr])
    s_tiles, s_pat, s_val, s_diag = ss.spawn(4)
    rng_t = np.random.Generator(np.random.Philox(s_tiles))
    rng_p = np.random.Generator(np.random.Philox(s_pat))
    rng_v = np.random.Generator(np.random.Philox(s_val))
    rng_d = np.random.Generator(np.random.Philox(s_diag))

    # active upper tiles per block row
    tiles = []
    for I in range(nblk):
        avail = nblk - 1 - I
        m = int(rng_t.binomial(avail, p)) if avail > 0 and p > 0 else 0
        if m > 0:
            J = np.sort(rng_t.choice(avail, size=m, replace=False)) + (I + 1)
        else:
            J = np.empty(0, dtype=np.int64)
        tiles.append(J.astype(np.int64))

    lev = ci_levels(n)
    diag = lev.astype(np.float64) + sigma_diag * rng_d.standard_normal(n)

    counts = np.zeros(n, dtype=np.int64)
    col_parts, off_mask_parts = [], []
    # group block rows so that each numpy call works on ~chunk_rows rows
    bpc = max(1, chunk_rows // B)
    for I0 in range(0, nblk, bpc):
        for I in range(I0, min(nblk, I0 + bpc)):
            r0, r1 = I * B, min(n, (I + 1) * B)
            nr = r1 - r0
            segs = [(r0, r1)] + [(int(J) * B, min(n, (int(J) + 1) * B)) for J in tiles[I]]
            colmap = np.concatenate([np.arange(a, b, dtype=np.int64) for a, b in segs])
            W = colmap.size
            raw = np.frombuffer(rng_p.bytes(nr * W), dtype=np.uint8).reshape(nr, W)
            present = raw < thr
            # diagonal tile: keep strictly-upper draws, force the diagonal itself
            dt = present[:, :nr]
            dt &= np.triu(np.ones((nr, nr), dtype=bool), k=1)
            dt[np.arange(nr), np.arange(nr)] = True
            ri, ci = np.nonzero(present)
            counts[r0:r1] = np.bincount(ri, minlength=nr)
            cg = colmap[ci]
            col_parts.append(cg.astype(np.int32))
            off_mask_parts.append(cg != (ri + r0))
    col = np.concatenate(col_parts) if col_parts else np.empty(0, np.int32)
    offm = np.concatenate(off_mask_parts) if off_mask_parts else np.empty(0, bool)
    del col_parts, off_mask_parts
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])

    nnz = col.size
    vals = np.empty(nnz, dtype=np.float64)
    n_off = int(offm.sum())
    vals[offm] = sigma_off * rng_v.standard_normal(n_off)
    vals[~offm] = diag  # diagonal entries appear once per row, in row order
    val = round_to_storage(vals, storage)
    H = CSRUpper(n=n, rowptr=rowptr, col=col, val=val, storage=storage,
                 meta=dict(kind="ci", seed=seed, block=B, rho=rho_q, mu=mu, p=p,
                           nnz_per_row=nnz_per_row, sigma_diag=sigma_diag, sigma_off=sigma_off))
    return H


def laplacian_kron(dims, storage: str = "f64", shift: float = 0.0) -> CSRUpper:
    """Kronecker-sum Laplacian T_a (+) T_b (+) T_c (T_m = tridiag(-1, 2, -1)), upper CSR.

    Its spectrum is known in closed form (laplacian_kron_eigs), which pins the oracle.
    """
    dims = [int(d) for d in dims]
    n = int(np.prod(dims))
    strides = [int(np.prod(dims[i + 1:])) for i in range(len(dims))]
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for s in strides:
        coords.append(rem // s)
        rem = rem % s
    rows_l, cols_l, vals_l = [idx], [idx], [np.full(n, 2.0 * len(dims) + shift)]
    for d, s in enumerate(strides):
        ok = coords[d] + 1 < dims[d]
        rows_l.append(idx[ok]); cols_l.append(idx[ok] + s); vals_l.append(np.full(int(ok.sum()), -1.0))
    rows = np.concatenate(rows_l); cols = np.concatenate(cols_l); vals = np.concatenate(vals_l)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return CSRUpper(n=n, rowptr=rowptr, col=cols.astype(np.int32), val=round_to_storage(vals, storage),
                    storage=storage, meta=dict(kind="laplacian", dims=dims, shift=shift))


def laplacian_kron_eigs(dims, shift: float = 0.0) -> np.ndarray:
    """Closed-form sorted spectrum of laplacian_kron(dims): sum_d (2 - 2 cos(pi k_d / (m_d + 1)))."""
    lam = np.zeros(1)
    for m in dims:
        e = 2.0 - 2.0 * np.cos(np.pi * np.arange(1, m + 1) / (m + 1))
        lam = (lam[:, None] + e[None, :]).ravel()
    return np.sort(lam + shift)


def diagonal_matrix(d: np.ndarray, storage: str = "f64") -> CSRUpper:
    n = d.size
    return CSRUpper(n=n, rowptr=np.arange(n + 1, dtype=np.int64), col=np.arange(n, dtype=np.int32),
                    val=round_to_storage(np.asarray(d, np.float64), storage), storage=storage,
                    meta=dict(kind="diagonal"))


def principal_submatrix(H: CSRUpper, n0: int) -> CSRUpper:
    """Leading n0 x n0 principal block (rows/cols < n0): the analogue of the smaller
    N_max - 2 model space used for initial guesses (Sec. 3.1, Table 3)."""
    n0 = int(n0)
    rp = H.rowptr[: n0 + 1]
    seg_col = H.col[: int(rp[-1])]
    keep = seg_col < n0
    rows = np.repeat(np.arange(n0, dtype=np.int64), np.diff(rp))
    cnt = np.bincount(rows[keep], minlength=n0)
    rowptr = np.zeros(n0 + 1, dtype=np.int64)
    np.cumsum(cnt, out=rowptr[1:])
    return CSRUpper(n=n0, rowptr=rowptr, col=seg_col[keep].copy(), val=H.val[: int(rp[-1])][keep].copy(),
                    storage=H.storage, meta=dict(H.meta, principal_of=H.n))


def random_block(n: int, k: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Seeded N(0,1) n x k block (row-major)."""
    rng = np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), int(n), int(k), 7])))
    return rng.standard_normal((n, k)).astype(dtype)


def pad_rows(X: np.ndarray, n: int) -> np.ndarray:
    """Zero-pad a block to n rows (the smaller-model-space guess of Sec. 3.1)."""
    out = np.zeros((n, X.shape[1]), dtype=X.dtype)
    out[: X.shape[0]] = X
    return out


def family_perturbation(H0: CSRUpper, seed: int, sigma: float = 0.1) -> np.ndarray:
    """Values of a symmetric perturbation V on the stored pattern of H0 (diagonal included),
    N(0, sigma^2), float64, one per stored entry of H0's upper triangle."""
    ss = np.random.SeedSequence([int(seed), H0.n, H0.nnz, 0x7F4A])
    rng = np.random.Generator(np.random.Philox(ss))
    return sigma * rng.standard_normal(H0.nnz)


def family_member(H0: CSRUpper, V: np.ndarray, g: float, storage: str = None) -> CSRUpper:
    """H(g) = H0 + g V on H0's pattern, values rounded to `storage` (default: H0's)."""
    st = storage or H0.storage
    val = round_to_storage(H0.values_f64() + float(g) * np.asarray(V, dtype=np.float64), st)
    meta = dict(H0.meta)
    meta.update(kind="family", g=float(g))
    return CSRUpper(n=H0.n, rowptr=H0.rowptr, col=H0.col, val=val, storage=st, meta=meta)
