"""Pins for the CPU oracle: closed forms, hand-computed examples, invariants
and cross-checks between its independent forms.  None of these uses the CUDA
path.  Every oracle function is pinned by at least one check that does not
re-derive its own formula:

* closed forms on the 1-D grid and on product grids (both metrics);
* hand-computed tiny examples (tests/golden/hand_examples.txt), including the
  two constructions of the Omega(nd) lower bound;
* invariants of distance matrices: symmetry z^T A w = w^T A z, zero diagonal,
  linearity in z, translation / reflection invariance, permutation
  equivariance, scaling by |a| (l1) and a^2 (squared l2), additivity over
  coordinates;
* rank <= d + 2 of the squared-l2 matrix; metric axioms of the l1 matrix;
* agreement of the definition (double loop) with the sort-based form of
  Algorithms 1-2 and with the p = 2 identity, exact on integers.
"""
import numpy as np
import pytest

import oracle
from paper_2210_15114_gb300 import inputs
from conftest import load_hand_examples


def g1(i, m):
    """sum_j |i - j| over j in [0, m): i(i+1)/2 + (m-1-i)(m-i)/2."""
    return i * (i + 1) // 2 + (m - 1 - i) * (m - i) // 2


def g2(i, m):
    """sum_j (i - j)^2 over j in [0, m)."""
    return i * (i + 1) * (2 * i + 1) // 6 + (m - 1 - i) * (m - i) * (2 * m - 2 * i - 1) // 6


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("dtype", [np.float64, np.int64])
def test_l1_grid_closed_form(dtype):
    n = 4096
    X = inputs.grid_1d(n).astype(dtype)
    z = np.ones(n, dtype=dtype)
    i = np.arange(n, dtype=np.int64)
    want = g1(i, n)
    np.testing.assert_array_equal(oracle.l1_rows(X, z), want.astype(dtype))
    np.testing.assert_array_equal(oracle.l1_sort(X, z), want.astype(dtype))


@pytest.mark.parametrize("dtype", [np.float64, np.int64])
def test_l2sq_grid_closed_form(dtype):
    n = 4096
    X = inputs.grid_1d(n).astype(dtype)
    z = np.ones(n, dtype=dtype)
    i = np.arange(n, dtype=np.int64)
    want = g2(i, n)
    np.testing.assert_array_equal(oracle.l2sq_rows(X, z), want.astype(dtype))
    np.testing.assert_array_equal(oracle.l2sq_identity(X, z), want.astype(dtype))


def test_product_grid_closed_forms():
    # Points (a, b), a in [0, n1), b in [0, n2): a product grid, so the
    # row sums separate per coordinate.
    n1, n2 = 37, 23
    a, b = np.meshgrid(np.arange(n1), np.arange(n2), indexing="ij")
    X = np.stack([a.ravel(), b.ravel()], axis=1).astype(np.int64)
    z = np.ones(len(X), dtype=np.int64)
    A, B = X[:, 0], X[:, 1]
    want1 = n2 * g1(A, n1) + n1 * g1(B, n2)
    want2 = n2 * g2(A, n1) + n1 * g2(B, n2)
    np.testing.assert_array_equal(oracle.l1_rows(X, z), want1)
    np.testing.assert_array_equal(oracle.l1_sort(X, z), want1)
    np.testing.assert_array_equal(oracle.l2sq_rows(X, z), want2)
    np.testing.assert_array_equal(oracle.l2sq_identity(X, z), want2)
    # the same grid in FP64, with the points shuffled
    perm = np.random.default_rng(3).permutation(len(X))
    np.testing.assert_array_equal(oracle.l1_sort(X[perm].astype(np.float64), z),
                                  want1[perm].astype(np.float64))


# --------------------------------------------------------------- hand examples
@pytest.mark.parametrize("ex", load_hand_examples(), ids=lambda e: e["name"])
def test_hand_examples(ex):
    X, z = ex["X"], ex["z"]
    for fn in (oracle.l1_rows, oracle.l1_sort):
        np.testing.assert_array_equal(fn(X, z), ex["l1"])
        np.testing.assert_array_equal(fn(X.astype(np.float64), z.astype(np.float64)),
                                      ex["l1"].astype(np.float64))
    for fn in (oracle.l2sq_rows, oracle.l2sq_identity):
        np.testing.assert_array_equal(fn(X, z), ex["l2sq"])
        np.testing.assert_array_equal(fn(X.astype(np.float64), z.astype(np.float64)),
                                      ex["l2sq"].astype(np.float64))


def test_lower_bound_construction_sum():
    # Theorem "lb_for_ub": n-1 identical points and one point at distance 1.
    # The entries of A 1 sum to 2(n-1): the outlier's row gives n-1 and every
    # other row gives 1.
    n, d = 513, 6
    X = np.full((n, d), 4, dtype=np.int64)
    X[200, 3] += 1
    one = np.ones(n, dtype=np.int64)
    for fn in (oracle.l1_rows, oracle.l1_sort, oracle.l2sq_rows, oracle.l2sq_identity):
        r = fn(X, one)
        assert r.sum() == 2 * (n - 1)
        assert r[200] == n - 1
        assert np.all(np.delete(r, 200) == 1)
    Xs = np.full((n, d), 4, dtype=np.int64)
    for fn in (oracle.l1_rows, oracle.l1_sort, oracle.l2sq_rows, oracle.l2sq_identity):
        assert np.all(fn(Xs, one) == 0)


# ----------------------------------------------------------------- invariants
FORMS = {
    "l1_rows": (oracle.l1_rows, 1),
    "l1_sort": (oracle.l1_sort, 1),
    "l2sq_rows": (oracle.l2sq_rows, 2),
    "l2sq_identity": (oracle.l2sq_identity, 2),
}


@pytest.fixture(scope="module")
def rand_small():
    rng = np.random.default_rng(11)
    X = rng.normal(size=(300, 5))
    Z = rng.normal(size=(300, 3))
    W = rng.normal(size=(300, 3))
    return X, Z, W


@pytest.mark.parametrize("form", list(FORMS))
def test_symmetry(form, rand_small):
    fn, _ = FORMS[form]
    X, Z, W = rand_small
    lhs = np.einsum("ij,ij->j", W, fn(X, Z))
    rhs = np.einsum("ij,ij->j", Z, fn(X, W))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-11)


@pytest.mark.parametrize("form", list(FORMS))
def test_zero_diagonal_and_columns(form, rand_small):
    # A e_i is column i of A: zero at i, equal to the distances elsewhere.
    fn, p = FORMS[form]
    X, _, _ = rand_small
    n = len(X)
    for i in (0, 17, n - 1):
        e = np.zeros(n)
        e[i] = 1.0
        col = fn(X, e)
        assert abs(col[i]) <= 1e-12 * np.abs(col).max()
        diff = X - X[i]
        want = np.abs(diff).sum(1) if p == 1 else (diff ** 2).sum(1)
        np.testing.assert_allclose(col, want, rtol=1e-11, atol=1e-11 * want.max())


@pytest.mark.parametrize("form", list(FORMS))
def test_linearity(form, rand_small):
    fn, _ = FORMS[form]
    X, Z, W = rand_small
    np.testing.assert_allclose(fn(X, 3.0 * Z - 0.5 * W), 3.0 * fn(X, Z) - 0.5 * fn(X, W),
                               rtol=1e-10, atol=1e-10 * np.abs(fn(X, Z)).max())


@pytest.mark.parametrize("form", list(FORMS))
def test_translation_reflection_scaling(form):
    # Integer data keep every transformed product exact.
    fn, p = FORMS[form]
    rng = np.random.default_rng(5)
    X = rng.integers(-50, 50, size=(257, 4)).astype(np.int64)
    Z = rng.integers(-9, 10, size=(257, 2)).astype(np.int64)
    base = fn(X, Z)
    np.testing.assert_array_equal(fn(X + np.array([1000, -7, 3, 0]), Z), base)
    np.testing.assert_array_equal(fn(-X, Z), base)
    Xr = X.copy()
    Xr[:, 2] *= -1
    np.testing.assert_array_equal(fn(Xr, Z), base)
    np.testing.assert_array_equal(fn(-3 * X, Z), (3 ** p) * base)


@pytest.mark.parametrize("form", list(FORMS))
def test_permutation_equivariance(form, rand_small):
    fn, _ = FORMS[form]
    X, Z, _ = rand_small
    P = np.random.default_rng(9).permutation(len(X))
    np.testing.assert_allclose(fn(X[P], Z[P]), fn(X, Z)[P], rtol=1e-11,
                               atol=1e-11 * np.abs(fn(X, Z)).max())


@pytest.mark.parametrize("form", list(FORMS))
def test_additive_over_coordinates(form):
    fn, _ = FORMS[form]
    rng = np.random.default_rng(6)
    X = rng.integers(0, 40, size=(200, 5)).astype(np.int64)
    Z = rng.integers(-5, 6, size=(200, 2)).astype(np.int64)
    total = sum(fn(X[:, [c]], Z) for c in range(X.shape[1]))
    np.testing.assert_array_equal(fn(X, Z), total)


def test_dense_matrix_structure():
    # Build the dense matrices column by column (Z = identity) from the
    # definition.  l1: a metric (symmetric, zero diagonal, nonnegative,
    # triangle inequality).  squared l2: rank <= d + 2 (Section 1.2: two
    # rank-one terms plus a Gram matrix of rank d).
    rng = np.random.default_rng(8)
    n, d = 160, 4
    X = rng.normal(size=(n, d))
    I = np.eye(n)
    A1 = oracle.l1_rows(X, I)
    A2 = oracle.l2sq_rows(X, I)
    for A in (A1, A2):
        np.testing.assert_allclose(A, A.T, rtol=1e-13, atol=1e-13)
        assert np.all(np.diag(A) == 0)
        assert np.all(A >= 0)
    tri = A1[:, None, :] - (A1[:, :, None] + A1[None, :, :])   # A_ij - A_ik - A_kj
    assert tri.max() <= 1e-12
    s2 = np.linalg.svd(A2, compute_uv=False)
    assert s2[d + 2] <= 1e-12 * s2[0]
    assert s2[d + 1] >= 1e-6 * s2[0]
    s1 = np.linalg.svd(A1, compute_uv=False)
    assert s1[d + 2] >= 1e-3 * s1[0]     # the l1 matrix is not of that form


# ---------------------------------------------- independent forms must agree
def test_forms_agree_fp64():
    X, z = inputs.workload_small_f64()
    want = oracle.l1_rows(X, z)
    assert oracle.relative_error(oracle.l1_sort(X, z), want) <= 1e-13
    want2 = oracle.l2sq_rows(X, z)
    assert oracle.relative_error(oracle.l2sq_identity(X, z), want2) <= 1e-12


@pytest.mark.parametrize("span", [8, 1 << 16])
def test_forms_agree_integer_exact(span):
    # span 8 gives heavy ties; 2^16 matches the integer workload's range.
    rng = np.random.default_rng(span)
    X = rng.integers(0, span, size=(700, 6)).astype(np.int32)
    Z = rng.integers(-100, 101, size=(700, 3)).astype(np.int32)
    np.testing.assert_array_equal(oracle.l1_sort(X, Z), oracle.l1_rows(X, Z))
    np.testing.assert_array_equal(oracle.l2sq_identity(X, Z), oracle.l2sq_rows(X, Z))


def test_forms_agree_signed_zeros_and_fp32():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(400, 3)).astype(np.float32)
    X[::7, 0] = 0.0
    X[3::7, 0] = -0.0
    X[::5, 1] = X[0, 1]                 # ties
    Z = rng.normal(size=(400, 2)).astype(np.float32)
    want = oracle.l1_rows(X, Z)
    assert oracle.relative_error(oracle.l1_sort(X, Z), want) <= 1e-13


def test_sampled_rows_match_full():
    X, z = inputs.workload_small_f64()
    rows = inputs.sample_rows(len(X), 20)
    np.testing.assert_array_equal(oracle.l1_rows(X, z, rows), oracle.l1_rows(X, z)[rows])
    np.testing.assert_array_equal(oracle.l2sq_rows(X, z, rows), oracle.l2sq_rows(X, z)[rows])


def test_preprocessing_order_is_stable_sort():
    col = np.array([3, 1, 3, 0, 1, 3], dtype=np.int64)
    np.testing.assert_array_equal(oracle.preprocessing_order(col), [3, 1, 4, 0, 2, 5])
