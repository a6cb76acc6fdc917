"""The autograd wrapper's routing, on the CPU: the library calls are replaced
by dense FP64 stand-ins (the product A(X) Z and the gradient of
sum_q w_q^T A(X) z_q through torch autograd of the dense formula), and the
wrapper's gradients with respect to X and Z are compared with torch autograd
through the dense formula itself.  This checks the wiring -- which tensor goes
to dm_grad as W and which as Z, and that dL/dZ is A dL/dout -- not the
kernels, which the GPU tests check against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2210_15114_gb300 import autograd as dag  # noqa: E402
from paper_2210_15114_gb300 import binding  # noqa: E402


def dense_A(X, metric):
    D = X[:, None, :] - X[None, :, :]
    return D.abs().sum(-1) if metric == "l1" else (D * D).sum(-1)


class FakePlan:
    def __init__(self, X, metric):
        self.X, self.metric = X.detach(), metric


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_wrapper_routes_gradients(monkeypatch, metric):
    def prepare(ctx, m, X):
        return FakePlan(X, m)

    def matmat(plan, Z, out=None):
        return dense_A(plan.X, plan.metric) @ Z

    def grad(plan, W, Z):
        with torch.enable_grad():     # backward passes run with grad mode off
            Xr = plan.X.clone().requires_grad_(True)
            L = (W * (dense_A(Xr, plan.metric) @ Z)).sum()
            (G,) = torch.autograd.grad(L, Xr)
        return G

    monkeypatch.setattr(binding, "dm_prepare", prepare)
    monkeypatch.setattr(binding, "dm_matmat", matmat)
    monkeypatch.setattr(binding, "dm_grad", grad)
    monkeypatch.setattr(binding, "dm_sync", lambda ctx: None)

    rng = np.random.default_rng(5)
    X0 = torch.from_numpy(rng.normal(size=(40, 3)))
    Z0 = torch.from_numpy(rng.normal(size=(40, 2)))
    R = torch.from_numpy(rng.normal(size=(40, 2)))        # dL/dout

    X = X0.clone().requires_grad_(True)
    Z = Z0.clone().requires_grad_(True)
    out = dag.DistanceProduct.apply(X, Z, metric, None)
    gX, gZ = torch.autograd.grad((out * R).sum(), (X, Z))

    Xr = X0.clone().requires_grad_(True)
    Zr = Z0.clone().requires_grad_(True)
    wX, wZ = torch.autograd.grad((dense_A(Xr, metric) @ Zr * R).sum(), (Xr, Zr))
    assert torch.allclose(gX, wX, rtol=1e-12, atol=1e-12)
    assert torch.allclose(gZ, wZ, rtol=1e-12, atol=1e-12)
