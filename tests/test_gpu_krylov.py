"""The block Krylov iteration on the GPU (products through dm_matmat) against
the pinned CPU oracle and the mathematics.

  * small n: the same start block Pi gives Ritz values equal to the oracle's
    (FP64) within 1e-4, and the top ones equal the eigenvalues of the dense
    matrix;
  * full size (n = 2^22, d = 16, 10-cluster mixture, k = 40, q = 8, rank 32):
    squared l2 -- the top d + 2 = 18 Ritz values equal the nonzero
    eigenvalues of the compressed form (FP64, on the host) within 1e-4 and
    the other 14 are zero to 1e-5 of the largest; l1 -- the top Ritz pairs
    satisfy ||A u - theta u|| <= 1e-3 |theta_1| (one more product), and U
    has orthonormal columns.
"""
import numpy as np
import pytest

import oracle
from paper_2210_15114_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_15114_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.fixture(scope="module")
def ctx(dm):
    return dm.dm_create(0)


def dense(metric, X):
    X = X.astype(np.float64)
    D = X[:, None, :] - X[None, :, :]
    return np.abs(D).sum(-1) if metric == "l1" else (D * D).sum(-1)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_krylov_small_matches_oracle_and_dense(dm, ctx, metric):
    from paper_2210_15114_gb300.krylov import block_krylov
    X, Pi = inputs.workload_krylov(n=2048, d=8, k=10)
    plan = dm.dm_prepare(ctx, metric, torch.from_numpy(X).cuda())
    theta, U = block_krylov(plan, torch.from_numpy(Pi).cuda(), q=4, rank=8)
    theta = theta.cpu().numpy()
    prod = (oracle.l1_sort if metric == "l1" else oracle.l2sq_identity)
    want, _ = oracle.block_krylov(lambda Z: prod(X, Z), Pi, q=4, rank=8)
    np.testing.assert_allclose(theta, want, rtol=1e-4)
    ev = np.linalg.eigvalsh(dense(metric, X))
    top = ev[np.argsort(-np.abs(ev))][:4]
    np.testing.assert_allclose(theta[:4], top, rtol=1e-4)
    Uh = U.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(Uh.T @ Uh, np.eye(8), atol=1e-4)


@pytest.fixture(scope="module")
def full():
    return inputs.workload_krylov()


def test_krylov_full_size_l2sq_compressed_form(dm, ctx, full):
    from paper_2210_15114_gb300.krylov import block_krylov
    X, Pi = full
    n, d = X.shape
    plan = dm.dm_prepare(ctx, "l2sq", torch.from_numpy(X).cuda())
    theta, _ = block_krylov(plan, torch.from_numpy(Pi).cuda(), q=8, rank=32)
    theta = theta.cpu().numpy()
    Xc = X.astype(np.float64)
    Xc -= Xc.mean(axis=0)
    B = np.concatenate([np.ones((n, 1)), (Xc * Xc).sum(1, keepdims=True), Xc], axis=1)
    C = np.zeros((d + 2, d + 2))
    C[0, 1] = C[1, 0] = 1.0
    C[2:, 2:] = -2 * np.eye(d)
    L = np.linalg.cholesky(B.T @ B)
    ev = np.linalg.eigvalsh(L.T @ C @ L)
    ev = ev[np.argsort(-np.abs(ev))]
    np.testing.assert_allclose(theta[:d + 2], ev, rtol=1e-4)
    assert np.all(np.abs(theta[d + 2:]) <= 1e-5 * abs(theta[0]))


def test_krylov_full_size_l1_ritz_residuals(dm, ctx, full):
    from paper_2210_15114_gb300.krylov import block_krylov
    X, Pi = full
    plan = dm.dm_prepare(ctx, "l1", torch.from_numpy(X).cuda())
    theta, U = block_krylov(plan, torch.from_numpy(Pi).cuda(), q=8, rank=32)
    AU = dm.dm_matmat(plan, U.contiguous()).double()
    Ud = U.double()
    th = theta.to(Ud.device)
    res = torch.linalg.norm(AU[:, :8] - Ud[:, :8] * th[:8], dim=0).cpu().numpy()
    assert np.all(res <= 1e-3 * abs(theta[0].item())), res / abs(theta[0].item())
    G = (Ud.T @ Ud).cpu().numpy()
    np.testing.assert_allclose(G, np.eye(32), atol=1e-4)
