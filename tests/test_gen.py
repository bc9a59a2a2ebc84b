"""The shared seeded generator: structure, determinism, storage rounding."""
import numpy as np

from gen import (ci_matrix, ci_levels, laplacian_kron, laplacian_kron_eigs, principal_submatrix,
                 f32_to_bf16_bits, bf16_bits_to_f32, random_block)


def test_levels_quadratic_degeneracy():
    lev = ci_levels(30)
    # g_k = (k+1)(k+2)/2 = 1, 3, 6, 10, ...
    assert list(np.bincount(lev)[:4]) == [1, 3, 6, 10]


def test_ci_matrix_structure_and_determinism():
    H = ci_matrix(5000, 100, 64, seed=3, storage="f32")
    H.check()
    H2 = ci_matrix(5000, 100, 64, seed=3, storage="f32")
    assert np.array_equal(H.col, H2.col) and np.array_equal(H.val, H2.val)
    full = (2 * H.nnz - H.n) / H.n
    assert 85 < full < 115
    # first entry of every row is the diagonal, value near its level
    d = H.diagonal_f64()
    lev = ci_levels(H.n)
    assert np.all(np.abs(d - lev) < 0.4)
    assert H.val.dtype == np.float32
    H3 = ci_matrix(5000, 100, 64, seed=4, storage="f32")
    assert not np.array_equal(H.col[:1000], H3.col[:1000])


def test_ragged_last_block():
    H = ci_matrix(1000 + 37, 60, 64, seed=1, storage="f64")
    H.check()
    assert H.n == 1037


def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.0078125, -3.14159, 0.1], dtype=np.float32)
    b = f32_to_bf16_bits(x)
    y = bf16_bits_to_f32(b)
    assert y[0] == 1.0 and y[2] == 1.0078125
    assert y[1] == 1.0  # tie rounds to even
    assert np.all(np.abs(y - x) <= np.abs(x) * 2.0 ** -8)
    H = ci_matrix(2000, 80, 64, seed=2, storage="bf16")
    assert H.val.dtype == np.uint16
    v = H.values_f32()
    assert np.array_equal(f32_to_bf16_bits(v), H.val)


def test_laplacian_structure():
    H = laplacian_kron([3, 4, 5])
    H.check()
    assert H.n == 60
    # 3-D: diagonal 6, one -1 per neighbour (upper part)
    assert H.nnz == 60 + (2 * 4 * 5) + (3 * 3 * 5) + (3 * 4 * 4)
    e = laplacian_kron_eigs([3, 4, 5])
    assert e.size == 60 and np.all(np.diff(e) >= 0)


def test_principal_submatrix():
    H = ci_matrix(3000, 80, 64, seed=1, storage="f64")
    H0 = principal_submatrix(H, 700)
    H0.check()
    assert H0.n == 700
    assert np.all(H0.col < 700)


def test_random_block_seeded():
    a = random_block(100, 4, 9)
    b = random_block(100, 4, 9)
    assert np.array_equal(a, b) and a.shape == (100, 4)


def test_family_member_is_h0_plus_g_v_on_the_same_pattern():
    from gen import family_perturbation, family_member
    H0 = ci_matrix(3000, 80, 64, seed=5, storage="f64")
    V = family_perturbation(H0, seed=9)
    assert V.shape == (H0.nnz,) and abs(V.std() - 0.1) < 0.01
    np.testing.assert_array_equal(V, family_perturbation(H0, seed=9))
    assert not np.array_equal(V, family_perturbation(H0, seed=10))
    Hg = family_member(H0, V, 0.75)
    assert Hg.rowptr is H0.rowptr and Hg.col is H0.col
    np.testing.assert_array_equal(Hg.values_f64(), H0.values_f64() + 0.75 * V)
    np.testing.assert_array_equal(family_member(H0, V, 0.0).values_f64(), H0.values_f64())
    H32 = family_member(H0, V, 1.25, storage="f32")
    assert H32.val.dtype == np.float32
    np.testing.assert_array_equal(H32.val, (H0.values_f64() + 1.25 * V).astype(np.float32))
