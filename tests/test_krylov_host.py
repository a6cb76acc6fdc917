"""Host-side steps of the block Krylov iteration (torch on the CPU): the
orthonormalization of a block against the earlier basis, for full-rank,
rank-deficient and zero blocks.  The products A Z and the dense tall-skinny
products (dm_dense_tn / dm_dense_nn) are the library's and are tested on the
GPU; here the dense products are replaced by torch products on the CPU, which
checks the iteration's logic, not the kernels."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2210_15114_gb300 import krylov  # noqa: E402

N, K = 3000, 10


@pytest.fixture(autouse=True)
def dense_on_cpu(monkeypatch):
    from paper_2210_15114_gb300 import binding

    def tn(ctx, A, B, alpha=1.0, out=None):
        return alpha * (A.T @ B)

    def nn(ctx, A, T, out=None, alpha=1.0, beta=0.0):
        r = alpha * (A @ T)
        if out is None:
            return r
        out.mul_(beta).add_(r)
        return out

    monkeypatch.setattr(binding, "dm_dense_tn", tn)
    monkeypatch.setattr(binding, "dm_dense_nn", nn)


def _basis(n, m, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.linalg.qr(torch.randn(n, m, generator=g, dtype=torch.float64)).Q.float()


def _check_orthonormal(Q, prev, tol=2e-6):
    I = torch.eye(Q.shape[1])
    assert torch.allclose(Q.T.double() @ Q.double(), I.double(), atol=tol)
    if prev.shape[1]:
        assert float((prev.T.double() @ Q.double()).abs().max()) < tol


def _in_span(A, Q, tol):
    # ||A - Q Q^T A|| / ||A||
    Ad, Qd = A.double(), Q.double()
    r = Ad - Qd @ (Qd.T @ Ad)
    return float(torch.linalg.norm(r) / torch.linalg.norm(Ad)) < tol


@pytest.fixture
def gen():
    return torch.Generator().manual_seed(7)


def test_full_rank_block(gen):
    prev = _basis(N, 6, 1)
    g = torch.Generator().manual_seed(2)
    W = krylov._project_out(None, torch.randn(N, K, generator=g), prev)
    Q = krylov._orthonormalize(None, W, prev, gen)
    _check_orthonormal(Q, prev)
    assert _in_span(W, Q, 1e-5)


def test_rank_deficient_block_keeps_resolved_directions(gen):
    prev = _basis(N, 6, 3)
    g = torch.Generator().manual_seed(4)
    low = torch.randn(N, 4, generator=g) @ torch.randn(4, K, generator=g)   # rank 4
    W = krylov._project_out(None, low + 1e-9 * torch.randn(N, K, generator=g), prev)
    assert krylov._cholqr2(None, W) is None                 # deficient: the fallback runs
    Q = krylov._orthonormalize(None, W, prev, gen)
    assert Q.shape == (N, K)
    _check_orthonormal(Q, prev)
    assert _in_span(W, Q, 1e-5)                       # the rank-4 range is kept


def test_long_deficient_block_needs_no_householder(gen, monkeypatch):
    # n = 2^20: the filled block must pass the Cholesky QR test (fill on the
    # scale of the resolved columns), so Householder QR is never reached
    n = 1 << 20
    g = torch.Generator().manual_seed(8)
    prev = torch.zeros(n, 0)
    W = torch.randn(n, 3, generator=g) @ torch.randn(3, 8, generator=g)
    def no_qr(*a, **k):
        raise AssertionError("Householder fallback used")
    monkeypatch.setattr(torch.linalg, "qr", no_qr)
    Q = krylov._orthonormalize(None, W, prev, gen)
    _check_orthonormal(Q, prev, tol=1e-5)
    assert _in_span(W, Q, 1e-5)


def test_zero_block_gets_fill(gen):
    prev = _basis(N, 6, 5)
    Q = krylov._orthonormalize(None, torch.zeros(N, K), prev, gen)
    _check_orthonormal(Q, prev)


def test_fill_is_seeded():
    prev = _basis(N, 3, 6)
    W = torch.zeros(N, K)
    a = krylov._orthonormalize(None, W, prev, torch.Generator().manual_seed(9))
    b = krylov._orthonormalize(None, W, prev, torch.Generator().manual_seed(9))
    assert torch.equal(a, b)


def _dense(metric, X):
    D = X[:, None, :] - X[None, :, :]
    return np.abs(D).sum(-1) if metric == "l1" else (D * D).sum(-1)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_block_krylov_host_steps_with_a_dense_product(monkeypatch, metric):
    # the iteration's host steps end to end, the library product replaced by
    # a dense FP32 product on the CPU: the top Ritz values equal the dense
    # eigenvalues; squared l2 (rank d + 2 = 6 < the block width 10) takes the
    # rank-deficient path on every block after the first
    from paper_2210_15114_gb300 import binding
    rng = np.random.default_rng(3)
    X = rng.normal(size=(500, 4))
    A = torch.from_numpy(_dense(metric, X).astype(np.float32))

    def product(plan, Z, out=None):
        r = A @ Z
        if out is None:
            return r
        out.copy_(r)
        return out

    monkeypatch.setattr(binding, "dm_matmat", product)
    synced = []
    monkeypatch.setattr(binding, "dm_sync", lambda ctx: synced.append(ctx))
    Pi = torch.from_numpy(rng.normal(size=(500, 10)).astype(np.float32))
    theta, U = krylov.block_krylov(types.SimpleNamespace(ctx="ctx"), Pi, q=3, rank=8)
    assert synced == ["ctx"]          # device-side errors are collected once, at the end
    ev = np.linalg.eigvalsh(_dense(metric, X))
    ev = ev[np.argsort(-np.abs(ev))]
    top = 6 if metric == "l2sq" else 4
    np.testing.assert_allclose(theta[:top].numpy(), ev[:top], rtol=1e-4)
    if metric == "l2sq":
        assert np.all(np.abs(theta[6:].numpy()) <= 1e-4 * abs(float(theta[0])))
    Ud = U.double()
    np.testing.assert_allclose((Ud.T @ Ud).numpy(), np.eye(8), atol=1e-4)
