"""Pins of the variant oracles (Appendix A: total variation, ||x - y||_p^p,
approximate l2 through the Gaussian l2 -> l1 embedding).

  * ||.||_p^p at p = 1, 2 equals the separately written C definitions of the
    l1 and squared-l2 products (bit for bit on integers);
  * the 1D grid closed form for p = 4 (Faulhaber's sum of fourth powers);
  * the even-p expansion equals the definition exactly on integers, and the
    printed algorithm's omissions (no y_j, no binomial coefficients, t from
    1) are caught;
  * total variation: point masses on disjoint outcomes are at distance 1,
    and TV of distributions lies in [0, 1];
  * the embedding: T(e_1) is G's first column / (beta m) by hand; the mean
    ||T(x)||_1 approaches ||x||_2 (E|g . x| = beta ||x||_2); the Frobenius
    error of the approximate l2 matrix shrinks like 1/sqrt(m) and is a few
    percent at m = 4096, and dropping beta is caught.
"""
from math import comb

import numpy as np
import pytest

import oracle


def test_lpp_matches_c_definitions():
    rng = np.random.default_rng(0)
    X = rng.integers(-50, 50, size=(80, 4))
    Z = rng.integers(-9, 10, size=(80, 3))
    np.testing.assert_array_equal(oracle.lpp_rows(X, Z, 1), oracle.l1_rows(X, Z))
    np.testing.assert_array_equal(oracle.lpp_rows(X, Z, 2), oracle.l2sq_rows(X, Z))


def faulhaber4(N):
    # sum_{m=1}^{N} m^4 = N (N+1) (2N+1) (3N^2 + 3N - 1) / 30
    return N * (N + 1) * (2 * N + 1) * (3 * N * N + 3 * N - 1) // 30


def test_lpp_grid_closed_form():
    n = 500
    X = np.arange(n).reshape(n, 1)
    i = np.arange(n)
    want = faulhaber4(i) + faulhaber4(n - 1 - i)
    np.testing.assert_array_equal(oracle.lpp_rows(X, np.ones(n, dtype=np.int64), 4), want)
    np.testing.assert_array_equal(oracle.lpp_even_expansion(X, np.ones(n, dtype=np.int64), 4), want)


@pytest.mark.parametrize("p", [2, 4, 6])
def test_even_expansion_matches_definition(p):
    rng = np.random.default_rng(p)
    X = rng.integers(-30, 30, size=(70, 3))
    Z = rng.integers(-9, 10, size=(70, 2))
    np.testing.assert_array_equal(oracle.lpp_even_expansion(X, Z, p), oracle.lpp_rows(X, Z, p))
    Xf = rng.normal(size=(70, 3))
    Zf = rng.normal(size=(70, 2))
    assert oracle.relative_error(oracle.lpp_even_expansion(Xf, Zf, p), oracle.lpp_rows(Xf, Zf, p)) < 1e-12


def printed_even_p(X, Z, p):
    # the printed algorithm: S_{i,t} = sum_j x_j(i)^(p-t) (-1)^(p-t), t = 1..p
    out = np.zeros((len(X), Z.shape[1]))
    for i in range(X.shape[1]):
        x = X[:, i].astype(np.float64)
        for t in range(1, p + 1):
            S = np.sum(x ** (p - t) * (-1.0) ** (p - t))
            out += (x ** t)[:, None] * S
    return out


def test_printed_even_p_is_caught():
    rng = np.random.default_rng(3)
    X = rng.integers(-5, 5, size=(40, 2))
    Z = rng.integers(-3, 4, size=(40, 1))
    assert not np.allclose(printed_even_p(X, Z, 4), oracle.lpp_rows(X, Z, 4))


def test_tv_of_distributions():
    P = np.eye(3)                               # point masses on disjoint outcomes
    np.testing.assert_allclose(oracle.tv_rows(P, np.eye(3)), 1.0 - np.eye(3))
    rng = np.random.default_rng(4)
    D = rng.dirichlet(np.ones(6), size=50)
    A = oracle.tv_rows(D, np.eye(50))
    assert np.all(A >= 0) and np.all(A <= 1 + 1e-12)
    np.testing.assert_allclose(A, A.T, atol=1e-14)


def test_embedding_by_hand():
    G = np.array([[1.0, 2.0], [-3.0, 0.5], [0.0, 4.0]])
    T = oracle.l2_embed(np.array([[1.0, 0.0]]), G)
    np.testing.assert_allclose(T[0], G[:, 0] / (np.sqrt(2 / np.pi) * 3))


def test_embedding_norm_and_matrix_error():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(1, 7))
    G = rng.normal(size=(40000, 7))
    assert abs(np.abs(oracle.l2_embed(x, G)).sum() / np.linalg.norm(x) - 1) < 0.01
    X = rng.normal(size=(120, 5))
    exact = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    errs = []
    for m in (256, 4096):
        G = rng.normal(size=(m, 5))
        B = oracle.l2_approx(X, G, np.eye(120))
        errs.append(np.linalg.norm(B - exact) / np.linalg.norm(exact))
    assert errs[1] < 0.03 and errs[1] < errs[0]
    # dropping beta scales every entry by beta: a 25 % error
    G = rng.normal(size=(4096, 5))
    Tb = oracle.l2_embed(X, G) * np.sqrt(2 / np.pi)
    B_wrong = oracle.l1_sort(Tb, np.eye(120))
    assert np.linalg.norm(B_wrong - exact) / np.linalg.norm(exact) > 0.15


@pytest.mark.parametrize("p", [1, 3, 5])
def test_odd_p_sorted_form_matches_definition(p):
    rng = np.random.default_rng(p + 40)
    X = rng.integers(-20, 20, size=(90, 3))          # many ties
    Z = rng.integers(-9, 10, size=(90, 2))
    np.testing.assert_array_equal(oracle.lpp_odd_sort(X, Z, p), oracle.lpp_rows(X, Z, p))
    Xf = rng.normal(size=(90, 3))
    Zf = rng.normal(size=(90, 2))
    assert oracle.relative_error(oracle.lpp_odd_sort(Xf, Zf, p), oracle.lpp_rows(Xf, Zf, p)) < 1e-12
    if p == 1:
        np.testing.assert_array_equal(oracle.lpp_odd_sort(X, Z, 1), oracle.l1_rows(X, Z))


def test_odd_p_grid_closed_form():
    # x_i = i on a 1D grid, z = 1: sum_j |i - j|^p = S_p(i) + S_p(n-1-i) with
    # S_p(N) = 1^p + ... + N^p: Nicomachus for p = 3, Faulhaber's polynomials
    # for p = 5 and 7 (exact integers; the grid sizes keep every sum < 2^63)
    sums = {
        3: (400, lambda N: (N * (N + 1) // 2) ** 2),
        5: (400, lambda N: N * N * (N + 1) ** 2 * (2 * N * N + 2 * N - 1) // 12),
        7: (150, lambda N: N * N * (N + 1) ** 2 * (3 * N ** 4 + 6 * N ** 3 - N * N - 4 * N + 2) // 24),
    }
    for p, (n, S) in sums.items():
        assert S(4) == sum(t ** p for t in range(1, 5))        # the polynomial itself
        X = np.arange(n).reshape(n, 1)
        want = np.array([S(i) + S(n - 1 - i) for i in range(n)], dtype=np.int64)
        np.testing.assert_array_equal(oracle.lpp_odd_sort(X, np.ones(n, dtype=np.int64), p), want)
        np.testing.assert_array_equal(oracle.lpp_rows(X, np.ones(n, dtype=np.int64), p), want)

