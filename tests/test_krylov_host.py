"""Host-side steps of the block Krylov iteration (torch on the CPU): the
orthonormalization of a block against the earlier basis, for full-rank,
rank-deficient and zero blocks.  The products A Z are the library's and are
tested on the GPU; these steps are dense linear algebra on tall blocks."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2210_15114_gb300 import krylov  # noqa: E402

N, K = 3000, 10


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
    W = krylov._project_out(torch.randn(N, K, generator=g), prev)
    Q = krylov._orthonormalize(W, prev, gen)
    _check_orthonormal(Q, prev)
    assert _in_span(W, Q, 1e-5)


def test_rank_deficient_block_keeps_resolved_directions(gen):
    prev = _basis(N, 6, 3)
    g = torch.Generator().manual_seed(4)
    low = torch.randn(N, 4, generator=g) @ torch.randn(4, K, generator=g)   # rank 4
    W = krylov._project_out(low + 1e-9 * torch.randn(N, K, generator=g), prev)
    assert krylov._cholqr2(W) is None                 # deficient: the fallback runs
    Q = krylov._orthonormalize(W, prev, gen)
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
    Q = krylov._orthonormalize(W, prev, gen)
    _check_orthonormal(Q, prev, tol=1e-5)
    assert _in_span(W, Q, 1e-5)


def test_zero_block_gets_fill(gen):
    prev = _basis(N, 6, 5)
    Q = krylov._orthonormalize(torch.zeros(N, K), prev, gen)
    _check_orthonormal(Q, prev)


def test_fill_is_seeded():
    prev = _basis(N, 3, 6)
    W = torch.zeros(N, K)
    a = krylov._orthonormalize(W, prev, torch.Generator().manual_seed(9))
    b = krylov._orthonormalize(W, prev, torch.Generator().manual_seed(9))
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
