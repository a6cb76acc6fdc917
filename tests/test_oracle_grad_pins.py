"""Pins of the gradient oracle (the gradient of L = sum_q w_q^T A(X) z_q with
respect to X, which the paper does not state; the oracle applies the chain
rule to the definition with sgn(0) = 0 for l1).

Each pin comes from outside the oracle's own formula:
  * closed forms on the 1D grid x_i = i with w = z = 1, derived by hand below;
  * central finite differences of L, where L is evaluated through the product
    oracle (itself pinned by the product tests).  For squared l2, L is
    quadratic in every coordinate, so a central difference is exact up to
    rounding.  For l1 on integer coordinates (gaps >= 1, h = 1e-3), a central
    difference is exact too, and gives 0 at a tie -- the sgn(0) = 0 reading;
  * torch autograd through an explicit FP64 formula of L (torch's |.| has
    derivative 0 at 0);
  * invariants: translation invariance (every column of G sums to 0),
    symmetry in (w, z), Euler's relation for homogeneous functions
    (sum x . G = L for l1, 2L for squared l2), scaling, linearity in w.
Mutants with planted mistakes must fail at least one pin.
"""
import numpy as np
import pytest

import oracle

GRADS = {
    ("l1", "rows"): oracle.l1_grad_rows,
    ("l1", "sort"): oracle.l1_grad_sort,
    ("l2sq", "rows"): oracle.l2sq_grad_rows,
    ("l2sq", "closed"): oracle.l2sq_grad_closed,
}
PRODUCT = {"l1": oracle.l1_rows, "l2sq": oracle.l2sq_rows}


def loss(metric, X, W, Z):
    """L = sum_q w_q^T (A z_q), with A z from the product oracle."""
    AZ = PRODUCT[metric](X, Z)
    return float(np.sum(np.asarray(W, dtype=np.float64) * AZ))


# -------------------------------------------------------------- closed forms
# Grid x_i = i (d = 1), w = z = 1:
#   l1:   dL/dx_i = sum_j 2 sgn(i - j) = 2 (i - (n - 1 - i)) = 2 (2i - n + 1)
#   l2sq: dL/dx_i = sum_j 2 * 2 (i - j) = 4 (n i - n(n-1)/2) = 2 n (2i - n + 1)
@pytest.mark.parametrize("key", list(GRADS))
@pytest.mark.parametrize("integer", [True, False])
def test_grid_closed_form(key, integer):
    metric, _ = key
    n = 4096 if key[1] != "rows" else 1500
    X = np.arange(n).reshape(n, 1)
    ones = np.ones((n, 1), dtype=np.int64)
    if not integer:
        X = X.astype(np.float64)
        ones = ones.astype(np.float64)
    G = GRADS[key](X, ones, ones)
    i = np.arange(n)
    want = 2 * (2 * i - n + 1) if metric == "l1" else 2 * n * (2 * i - n + 1)
    np.testing.assert_array_equal(G[:, 0], want)


# --------------------------------------------------------- finite differences
def fd_gradient(metric, X, W, Z, h):
    X = np.asarray(X, dtype=np.float64)
    G = np.zeros_like(X)
    for i in range(X.shape[0]):
        for c in range(X.shape[1]):
            Xp = X.copy(); Xp[i, c] += h
            Xm = X.copy(); Xm[i, c] -= h
            G[i, c] = (loss(metric, Xp, W, Z) - loss(metric, Xm, W, Z)) / (2 * h)
    return G


@pytest.fixture(scope="module")
def tie_heavy():
    rng = np.random.default_rng(11)
    X = rng.integers(0, 5, size=(24, 3)).astype(np.float64)   # many ties
    W = rng.normal(size=(24, 2))
    Z = rng.normal(size=(24, 2))
    return X, W, Z


@pytest.mark.parametrize("key", list(GRADS))
def test_central_differences(key, tie_heavy):
    metric, _ = key
    X, W, Z = tie_heavy
    if metric == "l2sq":                 # exact for any data: use a non-grid X too
        X = X + np.random.default_rng(12).uniform(-0.3, 0.3, size=X.shape)
    G = GRADS[key](X, W, Z)
    F = fd_gradient(metric, X, W, Z, 1e-3)
    assert np.abs(G - F).max() <= 1e-8 * max(1.0, np.abs(F).max())


# ------------------------------------------------------------ torch autograd
@pytest.mark.parametrize("key", list(GRADS))
def test_torch_autograd(key):
    torch = pytest.importorskip("torch")
    metric, _ = key
    rng = np.random.default_rng(13)
    X = rng.integers(0, 7, size=(64, 3)).astype(np.float64)
    W = rng.normal(size=(64, 2))
    Z = rng.normal(size=(64, 2))
    Xt = torch.tensor(X, requires_grad=True)
    diff = Xt[:, None, :] - Xt[None, :, :]
    A = diff.abs().sum(-1) if metric == "l1" else (diff * diff).sum(-1)
    L = (torch.tensor(W) * (A @ torch.tensor(Z))).sum()
    L.backward()
    np.testing.assert_allclose(GRADS[key](X, W, Z), Xt.grad.numpy(), rtol=0, atol=1e-9)


# ---------------------------------------------------------------- invariants
@pytest.fixture(scope="module")
def rand_pts():
    rng = np.random.default_rng(14)
    return rng.normal(size=(50, 4)), rng.normal(size=(50, 3)), rng.normal(size=(50, 3))


@pytest.mark.parametrize("key", list(GRADS))
def test_invariants(key, rand_pts):
    metric, _ = key
    X, W, Z = rand_pts
    g = GRADS[key]
    G = g(X, W, Z)
    scale = np.abs(G).max()
    # translation invariance: L(X + 1 t^T) = L(X), so every column of G sums to 0
    assert np.abs(G.sum(axis=0)).max() <= 1e-10 * scale * len(X)
    # symmetric in (w, z)
    assert np.abs(g(X, Z, W) - G).max() <= 1e-10 * scale
    # Euler: L is homogeneous of degree 1 (l1) or 2 (squared l2) in X
    deg = 1 if metric == "l1" else 2
    L = loss(metric, X, W, Z)
    assert abs(np.sum(X * G) - deg * L) <= 1e-10 * max(1.0, abs(L)) * len(X)
    # scaling: G(aX) = sgn(a) G(X) (l1), a G(X) (squared l2)
    a = -2.5
    want = (np.sign(a) if metric == "l1" else a) * G
    assert np.abs(g(a * X, W, Z) - want).max() <= 1e-10 * scale * abs(a)
    # linear in w
    W2 = np.random.default_rng(15).normal(size=W.shape)
    assert np.abs(g(X, W + W2, Z) - G - g(X, W2, Z)).max() <= 1e-10 * scale * 4
    # translation of the points leaves G unchanged
    assert np.abs(g(X + 3.0, W, Z) - G).max() <= 1e-9 * scale


def test_forms_agree_integer_exact():
    rng = np.random.default_rng(16)
    X = rng.integers(-50, 50, size=(200, 5))
    W = rng.integers(-9, 10, size=(200, 2))
    Z = rng.integers(-9, 10, size=(200, 2))
    np.testing.assert_array_equal(oracle.l1_grad_rows(X, W, Z), oracle.l1_grad_sort(X, W, Z))
    np.testing.assert_array_equal(oracle.l2sq_grad_rows(X, W, Z), oracle.l2sq_grad_closed(X, W, Z))


def test_sampled_rows_match_full():
    rng = np.random.default_rng(17)
    X, W, Z = rng.normal(size=(80, 3)), rng.normal(size=(80, 1)), rng.normal(size=(80, 1))
    rows = np.array([0, 5, 79, 33])
    for m in ("l1", "l2sq"):
        full = GRADS[(m, "rows")](X, W, Z)
        np.testing.assert_array_equal(GRADS[(m, "rows")](X, W, Z, rows), full[rows])


# ------------------------------------------------------------------- mutants
def _mutant(metric, mutation):
    """A plausible wrong gradient, written out in numpy."""
    def g(X, W, Z):
        X = np.asarray(X, dtype=np.float64)
        W = np.asarray(W, dtype=np.float64).reshape(len(X), -1)
        Z = np.asarray(Z, dtype=np.float64).reshape(len(X), -1)
        if X.ndim == 1:
            X = X[:, None]
        diff = X[:, None, :] - X[None, :, :]                 # x_i - x_j
        if metric == "l1":
            phi = np.sign(diff)
            if mutation == "sgn0_plus_one":
                phi = np.where(diff == 0, 1.0, phi)
                np.einsum("iic->ic", phi)[:] = 0.0
        else:
            phi = 2 * diff if mutation != "no_factor_2" else diff
        weight = W @ Z.T + Z @ W.T                            # w_i z_j + z_i w_j
        if mutation == "one_sided":
            weight = W @ Z.T
        if mutation == "flipped_sign":
            phi = -phi
        return np.einsum("ij,ijc->ic", weight, phi)
    return g


def _pins_pass(metric, g):
    try:
        n = 300
        X = np.arange(n, dtype=np.float64).reshape(n, 1)
        ones = np.ones((n, 1))
        i = np.arange(n)
        want = 2 * (2 * i - n + 1) if metric == "l1" else 2 * n * (2 * i - n + 1)
        if not np.array_equal(g(X, ones, ones)[:, 0], want):
            return False
        rng = np.random.default_rng(11)
        Xt = rng.integers(0, 5, size=(24, 3)).astype(np.float64)
        W, Z = rng.normal(size=(24, 2)), rng.normal(size=(24, 2))
        G = g(Xt, W, Z)
        if np.abs(G.sum(axis=0)).max() > 1e-9 * np.abs(G).max() * 24:
            return False
        F = fd_gradient(metric, Xt, W, Z, 1e-3)
        return np.abs(G - F).max() <= 1e-8 * max(1.0, np.abs(F).max())
    except Exception:
        return False


def test_unmutated_numpy_form_passes():
    assert _pins_pass("l1", _mutant("l1", None))
    assert _pins_pass("l2sq", _mutant("l2sq", None))


@pytest.mark.parametrize("metric,mutation", [("l1", "sgn0_plus_one"), ("l1", "one_sided"),
                                             ("l1", "flipped_sign"), ("l2sq", "no_factor_2"),
                                             ("l2sq", "one_sided"), ("l2sq", "flipped_sign")])
def test_gradient_mutants_are_caught(metric, mutation):
    assert not _pins_pass(metric, _mutant(metric, mutation))
