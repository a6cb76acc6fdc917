"""Strength of the oracle's pins: each plausible mistake, planted in a copy of
an oracle form (on the CPU), must fail at least one pin that does not depend
on the oracle itself (closed forms, hand-computed examples, invariants).

The planted mistakes include the two typos of the printed p = 2 query
(Appendix A squares y_j in S1 and S2), so the pins also justify the reading
the oracle takes there.
"""
import numpy as np
import pytest

import oracle
from conftest import load_hand_examples
from test_oracle_pins import g1, g2


def _l1_sort_variant(X, Z, mutation):
    X = np.asarray(X, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    sq = Z.ndim == 1
    if sq:
        Z = Z[:, None]
    n, d = X.shape
    out = np.zeros(Z.shape)
    zero = np.zeros((1, Z.shape[1]))
    for i in range(d):
        order = np.argsort(X[:, i], kind="stable")
        if mutation == "descending":
            order = order[::-1]
        xs = X[order, i]
        ys = Z if mutation == "unsorted_y" else Z[order]
        B = np.concatenate([zero, np.cumsum(xs[:, None] * ys, axis=0)])
        C = np.concatenate([zero, np.cumsum(ys, axis=0)])
        q = np.empty(n, dtype=np.int64)
        q[order] = np.arange(n)
        if mutation == "rank_as_perm":
            q = order.copy()
        S1, S2, S3, S4 = B[q], B[n] - B[q], C[q], C[n] - C[q]
        if mutation == "swap_S1_S2":
            S1, S2 = S2, S1
        if mutation == "swap_S3_S4":
            S3, S4 = S4, S3
        if mutation == "drop_S2":
            S2 = 0.0 * S2
        xk = X[:, i, None]
        if mutation == "x_from_sorted":
            xk = xs[:, None]
        out += xk * (S3 - S4) + S2 - S1
    return out[:, 0] if sq else out


def _l2sq_variant(X, Z, mutation):
    X = np.asarray(X, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    sq_ = Z.ndim == 1
    if sq_:
        Z = Z[:, None]
    nrm = (X * X).sum(1)
    v = X.T @ Z
    S1 = (Z * Z).sum(0) if mutation == "printed_S1_y_squared" else Z.sum(0)
    S2 = nrm @ (Z * Z) if mutation == "printed_S2_y_squared" else nrm @ Z
    two = 1.0 if mutation == "drop_factor_2" else 2.0
    if mutation == "sign_S2":
        S2 = -S2
    if mutation == "norm_of_wrong_point":
        nrm = nrm[::-1]
    out = nrm[:, None] * S1[None] + S2[None] - two * (X @ v)
    return out[:, 0] if sq_ else out


def _brute_variant(X, Z, metric, mutation):
    X = np.asarray(X, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    sq = Z.ndim == 1
    if sq:
        Z = Z[:, None]
    diff = X[:, None, :] - X[None, :, :]
    if metric == 1:
        D = diff.sum(-1) if mutation == "no_abs" else np.abs(diff).sum(-1)
    else:
        D = np.abs(diff).sum(-1) ** 2 if mutation == "square_of_sum" else (diff ** 2).sum(-1)
    if mutation == "weight_own_z":
        out = D.sum(1)[:, None] * Z
    elif mutation == "max_not_sum":
        out = np.abs(diff).max(-1) @ Z
    else:
        out = D @ Z
    return out[:, 0] if sq else out


def _pins_pass(fn, p):
    """True when every oracle-independent pin holds for fn (p = 1 or 2)."""
    closed = g1 if p == 1 else g2
    key = "l1" if p == 1 else "l2sq"
    try:
        for ex in load_hand_examples():
            if not np.array_equal(np.rint(fn(ex["X"], ex["z"])), ex[key]):
                return False
        n = 64
        X = np.arange(n, dtype=np.float64)[:, None]
        if not np.array_equal(fn(X, np.ones(n)), closed(np.arange(n), n).astype(float)):
            return False
        n1, n2 = 7, 5
        a, b = np.meshgrid(np.arange(n1), np.arange(n2), indexing="ij")
        G = np.stack([a.ravel(), b.ravel()], 1).astype(np.float64)
        want = n2 * closed(G[:, 0].astype(int), n1) + n1 * closed(G[:, 1].astype(int), n2)
        if not np.allclose(fn(G, np.ones(len(G))), want):
            return False
        rng = np.random.default_rng(1)
        Xr = rng.normal(size=(40, 3))
        z, w = rng.normal(size=40), rng.normal(size=40)
        if not np.isclose(w @ fn(Xr, z), z @ fn(Xr, w), rtol=1e-9):
            return False
    except Exception:
        return False
    return True


def test_unmutated_forms_pass_the_pins():
    assert _pins_pass(oracle.l1_sort, 1)
    assert _pins_pass(oracle.l1_rows, 1)
    assert _pins_pass(oracle.l2sq_identity, 2)
    assert _pins_pass(oracle.l2sq_rows, 2)
    assert _pins_pass(lambda X, Z: _l1_sort_variant(X, Z, None), 1)
    assert _pins_pass(lambda X, Z: _l2sq_variant(X, Z, None), 2)
    assert _pins_pass(lambda X, Z: _brute_variant(X, Z, 1, None), 1)
    assert _pins_pass(lambda X, Z: _brute_variant(X, Z, 2, None), 2)


@pytest.mark.parametrize("mutation", ["descending", "unsorted_y", "rank_as_perm",
                                      "swap_S1_S2", "swap_S3_S4", "drop_S2",
                                      "x_from_sorted"])
def test_l1_sort_mutants_are_caught(mutation):
    assert not _pins_pass(lambda X, Z: _l1_sort_variant(X, Z, mutation), 1)


@pytest.mark.parametrize("mutation", ["printed_S1_y_squared", "printed_S2_y_squared",
                                      "drop_factor_2", "sign_S2", "norm_of_wrong_point"])
def test_l2sq_identity_mutants_are_caught(mutation):
    assert not _pins_pass(lambda X, Z: _l2sq_variant(X, Z, mutation), 2)


@pytest.mark.parametrize("metric,mutation", [(1, "no_abs"), (1, "weight_own_z"),
                                             (1, "max_not_sum"), (2, "square_of_sum"),
                                             (2, "weight_own_z")])
def test_definition_mutants_are_caught(metric, mutation):
    assert not _pins_pass(lambda X, Z: _brute_variant(X, Z, metric, mutation), metric)
