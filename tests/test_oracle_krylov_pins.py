"""Pins of the block Krylov oracle (top singular values and low-rank
approximation of a distance matrix through products A Z only).

  * a dense symmetric eigendecomposition of the explicit matrix (numpy's
    eigh, small n): the Ritz values equal the eigenvalues of largest modulus
    and the rank-r approximation error is within 1% of the optimal one
    (Eckart-Young: the optimal error is the norm of the discarded
    eigenvalues);
  * Cauchy interlacing: Ritz values of a compression never exceed the
    eigenvalues of the same rank from the top;
  * squared l2: A = B C B^T with B = [1, s, X] (s_i = ||x_i||^2) and
    C = [[0,1,0],[1,0,0],[0,0,-2I]] -- rank <= d + 2 -- so the nonzero
    eigenvalues are those of L^T C L (B^T B = L L^T), and a Krylov space of
    dimension >= d + 2 reproduces A to rounding;
  * mutants (no Rayleigh-Ritz product, selection by signed value) fail.
"""
import numpy as np
import pytest

import oracle


def dense(metric, X):
    D = X[:, None, :] - X[None, :, :]
    return np.abs(D).sum(-1) if metric == "l1" else (D * D).sum(-1)


def top_by_modulus(ev, r):
    return ev[np.argsort(-np.abs(ev))][:r]


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_ritz_values_match_dense_eigenvalues(metric):
    rng = np.random.default_rng(1)
    X = rng.normal(size=(512, 6))
    A = dense(metric, X)
    Pi = rng.normal(size=(512, 12))
    theta, U = oracle.block_krylov(lambda Z: A @ Z, Pi, q=6, rank=8)
    ev = np.linalg.eigvalsh(A)
    want = top_by_modulus(ev, 8)
    np.testing.assert_allclose(theta, want, rtol=1e-6, atol=1e-9 * np.abs(want[0]))
    # near-optimal rank-8 approximation
    err = np.linalg.norm(A - (U * theta) @ U.T)
    opt = np.sqrt(np.sum(np.sort(np.abs(ev))[::-1][8:] ** 2))
    assert err <= 1.01 * opt + 1e-9 * np.linalg.norm(A)
    # U has orthonormal columns
    np.testing.assert_allclose(U.T @ U, np.eye(8), atol=1e-10)


def test_interlacing_from_the_top():
    rng = np.random.default_rng(2)
    X = rng.normal(size=(300, 3))
    A = dense("l1", X)
    theta, _ = oracle.block_krylov(lambda Z: A @ Z, rng.normal(size=(300, 2)), q=2, rank=4)
    ev = np.sort(np.linalg.eigvalsh(A))[::-1]
    pos = np.sort(theta[theta > 0])[::-1]
    assert np.all(pos <= ev[:len(pos)] * (1 + 1e-12))
    neg = np.sort(theta[theta < 0])
    assert np.all(neg >= np.sort(ev)[:len(neg)] * (1 + 1e-12))


def test_l2sq_low_rank_is_recovered_exactly():
    rng = np.random.default_rng(3)
    n, d = 700, 4
    X = rng.normal(size=(n, d))
    A = dense("l2sq", X)
    theta, U = oracle.block_krylov(lambda Z: A @ Z, rng.normal(size=(n, 4)), q=3, rank=12)
    assert np.linalg.norm(A - (U * theta) @ U.T) <= 1e-10 * np.linalg.norm(A)
    # the compressed form gives the d + 2 nonzero eigenvalues
    Xc = X - X.mean(axis=0)
    B = np.concatenate([np.ones((n, 1)), (Xc * Xc).sum(1, keepdims=True), Xc], axis=1)
    C = np.zeros((d + 2, d + 2))
    C[0, 1] = C[1, 0] = 1.0
    C[2:, 2:] = -2 * np.eye(d)
    np.testing.assert_allclose(B @ C @ B.T, A - 0, rtol=0, atol=1e-9 * np.abs(A).max())
    L = np.linalg.cholesky(B.T @ B)
    nz = top_by_modulus(np.linalg.eigvalsh(L.T @ C @ L), d + 2)
    np.testing.assert_allclose(theta[:d + 2], nz, rtol=1e-9)
    assert np.all(np.abs(theta[d + 2:]) <= 1e-9 * np.abs(theta[0]))


def _mutant(product, Pi, q, rank, mutation):
    W = product(Pi)
    blocks, prods = [], []
    for _ in range(q):
        for B in blocks:
            W = W - B @ (B.T @ W)
        Qi, _ = np.linalg.qr(W)
        blocks.append(Qi)
        W = product(Qi)
        prods.append(W)
    Q = np.concatenate(blocks, 1)
    AQ = np.concatenate(prods, 1)
    M = Q.T @ (Q if mutation == "no_rayleigh_product" else AQ)
    th, V = np.linalg.eigh(0.5 * (M + M.T))
    order = np.argsort(-th)[:rank] if mutation == "signed_order" else np.argsort(-np.abs(th))[:rank]
    return th[order], Q @ V[:, order]


@pytest.mark.parametrize("mutation", ["no_rayleigh_product", "signed_order"])
def test_krylov_mutants_are_caught(mutation):
    rng = np.random.default_rng(1)
    X = rng.normal(size=(512, 6))
    A = dense("l1", X)
    theta, _ = _mutant(lambda Z: A @ Z, rng.normal(size=(512, 12)), 6, 8, mutation)
    want = top_by_modulus(np.linalg.eigvalsh(A), 8)
    assert not np.allclose(theta, want, rtol=1e-6)
