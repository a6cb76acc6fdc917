"""Parity of dm_grad (the gradient of sum_q w_q^T A(X) z_q with respect to X)
with the CPU oracle, through the C ABI.

Tolerances (Frobenius relative error of G against the FP64 oracle on the same
input values): 1e-5 for FP32, 1e-12 for FP64; int32 inputs give exact int64
gradients, compared bit for bit.  Every case is compared on
every entry; the full-size workload (n = 2^21, d = 64, k = 1, uniform and
tie-heavy) against the oracle's sorted-order gradient (l1, the coordinates on
parallel host processes) or its closed form (squared l2), with sampled rows
checked once more against the definition, plus two properties that hold at
any size: translation invariance (every column of G sums to zero) and
Euler's relation sum X . G = deg * w^T A z (deg 1 for l1, 2 for squared l2).
"""
import numpy as np
import pytest

import oracle
from oracle import parallel
from paper_2210_15114_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {np.float32: 1e-5, np.float64: 1e-12}
GRAD = {"l1": oracle.l1_grad_rows, "l2sq": oracle.l2sq_grad_rows}


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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_grad(dm, ctx, metric, X, W, Z):
    plan = dm.dm_prepare(ctx, metric, dev(X))
    G = dm.dm_grad(plan, dev(W), dev(Z))
    dm.dm_sync(ctx)
    return G.cpu().numpy()


def check(got, want, dtype):
    if np.issubdtype(np.dtype(dtype), np.integer):
        np.testing.assert_array_equal(got, want)
    else:
        err = oracle.relative_error(got, want)
        assert err <= TOL[np.dtype(dtype).type], f"relative error {err:.3e}"


def make(kind, n, d, k, dtype, seed=0):
    rng = np.random.default_rng(seed)
    if dtype == np.int32:
        if kind == "ties":
            X = rng.integers(0, 5, size=(n, d))
        else:
            X = rng.integers(0, 1 << 16, size=(n, d))
        W = rng.integers(-100, 101, size=(n, k))
        Z = rng.integers(-100, 101, size=(n, k))
        return X.astype(np.int32), W.astype(np.int32), Z.astype(np.int32)
    if kind == "ties":
        X = rng.integers(0, 5, size=(n, d)).astype(np.float64)
    elif kind == "grid":
        X = rng.integers(0, 1024, size=(n, d)).astype(np.float64)
    else:
        X = rng.normal(0, 3, size=(n, d))
    W = rng.normal(size=(n, k))
    Z = rng.normal(size=(n, k))
    return X.astype(dtype), W.astype(dtype), Z.astype(dtype)


SIZES = [1, 2, 3, 100, 2047, 2048, 2049, 4100]


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int32])
def test_grad_sizes(dm, ctx, metric, n, dtype):
    X, W, Z = make("normal", n, 3, 2, dtype, seed=n)
    check(gpu_grad(dm, ctx, metric, X, W, Z), GRAD[metric](X, W, Z), dtype)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
@pytest.mark.parametrize("kind", ["ties", "grid"])
@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int32])
def test_grad_tie_groups_across_tiles(dm, ctx, metric, kind, dtype):
    # 5 (or 1024) distinct values over 9000 points: tie groups span many tiles
    X, W, Z = make(kind, 9000, 4, 1, dtype, seed=5)
    check(gpu_grad(dm, ctx, metric, X, W, Z), GRAD[metric](X, W, Z), dtype)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
@pytest.mark.parametrize("k", [1, 3, 8])
@pytest.mark.parametrize("d", [1, 8, 17])
def test_grad_widths(dm, ctx, metric, k, d):
    X, W, Z = make("normal", 3001, d, k, np.float32, seed=d * 10 + k)
    check(gpu_grad(dm, ctx, metric, X, W, Z), GRAD[metric](X, W, Z), np.float32)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_grad_identical_points_is_zero(dm, ctx, metric):
    X = np.full((5000, 3), 2.5, dtype=np.float32)
    W, Z = make("normal", 5000, 1, 2, np.float32)[1:]
    G = gpu_grad(dm, ctx, metric, X, W, Z)
    assert np.all(G == 0)


def test_grad_signed_zeros_tie(dm, ctx):
    # -0.0 and +0.0 are one value: a tie (sgn(0) = 0), whatever their keys
    rng = np.random.default_rng(3)
    X = rng.choice(np.array([-0.0, 0.0, 1.0, -1.0], dtype=np.float32), size=(3000, 2))
    W, Z = make("normal", 3000, 1, 1, np.float32, seed=4)[1:]
    check(gpu_grad(dm, ctx, "l1", X, W, Z), oracle.l1_grad_rows(X, W, Z), np.float32)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_grad_leading_dimensions(dm, ctx, metric):
    X, W, Z = make("normal", 2500, 5, 3, np.float32, seed=9)
    Wp = torch.zeros((2500, 7), dtype=torch.float32, device="cuda")
    Zp = torch.zeros((2500, 6), dtype=torch.float32, device="cuda")
    Wp[:, :3] = dev(W)
    Zp[:, :3] = dev(Z)
    Gp = torch.full((2500, 9), 7.0, dtype=torch.float32, device="cuda")
    plan = dm.dm_prepare(ctx, metric, dev(X))
    dm.dm_grad(plan, Wp[:, :3], Zp[:, :3], out=Gp[:, :5])
    dm.dm_sync(ctx)
    G = Gp.cpu().numpy()
    check(G[:, :5], GRAD[metric](X, W, Z), np.float32)
    assert np.all(G[:, 5:] == 7.0)


def test_grad_invalid_arguments(dm, ctx):
    X, W, Z = make("normal", 100, 3, 2, np.float32)
    plan = dm.dm_prepare(ctx, "l1", dev(X))
    with pytest.raises(dm.DMError):
        dm.dm_grad(plan, dev(W), dev(Z[:, :1]))          # shapes differ
    with pytest.raises(dm.DMError):
        dm.dm_grad(plan, dev(W.astype(np.float64)), dev(Z.astype(np.float64)))


# ------------------------------------------------------------- full size
@pytest.fixture(scope="module", params=[False, True], ids=["uniform", "tie_heavy"])
def full(request):
    return inputs.workload_gradient(tie_heavy=request.param)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_grad_full_size_whole_block(dm, ctx, full, metric):
    X, W, Z = full
    n = len(X)
    Xd, Wd, Zd = dev(X), dev(W), dev(Z)
    plan = dm.dm_prepare(ctx, metric, Xd)
    G = dm.dm_grad(plan, Wd, Zd)
    Az = dm.dm_matmat(plan, Zd)
    dm.dm_sync(ctx)
    Gh = G.cpu().numpy().astype(np.float64)
    whole = parallel.l1_grad_sort(X, W, Z) if metric == "l1" else oracle.l2sq_grad_closed(X, W, Z)
    check(Gh, whole, np.float32)
    rows = inputs.sample_rows(n, 6)
    check(Gh[rows], GRAD[metric](X, W, Z, rows), np.float32)
    # translation invariance: columns of G sum to zero
    col = np.abs(Gh.sum(axis=0))
    scale = np.sqrt((Gh ** 2).sum(axis=0) * n)
    assert np.all(col <= 1e-5 * scale), (col / scale).max()
    # Euler: sum X . G = deg * w^T (A z)
    deg = 1 if metric == "l1" else 2
    L = float(np.dot(W[:, 0].astype(np.float64), Az.cpu().numpy().astype(np.float64)[:, 0]))
    lhs = float(np.sum(X.astype(np.float64) * Gh))
    assert abs(lhs - deg * L) <= 1e-5 * np.abs(X.astype(np.float64) * Gh).sum()


# ----------------------------------------------------------------- autograd
def test_autograd_matches_oracle_and_gradcheck(dm):
    from paper_2210_15114_gb300.autograd import DistanceProduct
    # gradcheck repeats the backward pass and wants identical bits: the l1
    # query's fixed-order accumulation gives them
    ctx = dm.dm_create(0)
    dm.dm_set_deterministic(ctx, True)
    rng = np.random.default_rng(21)
    for metric in ("l1", "l2sq", "tv"):
        X = torch.tensor(rng.normal(size=(40, 3)), device="cuda", requires_grad=True)
        Z = torch.tensor(rng.normal(size=(40, 2)), device="cuda", requires_grad=True)
        assert torch.autograd.gradcheck(lambda a, b: DistanceProduct.apply(a, b, metric, ctx), (X, Z),
                                        eps=1e-6, atol=1e-6, rtol=1e-5)
        out = DistanceProduct.apply(X, Z, metric, ctx)
        Wt = torch.tensor(rng.normal(size=(40, 2)), device="cuda")
        (out * Wt).sum().backward()
        Xn, Zn, Wn = (t.detach().cpu().numpy() for t in (X, Z, Wt))
        scale = 0.5 if metric == "tv" else 1.0
        base = "l1" if metric == "tv" else metric
        np.testing.assert_allclose(X.grad.cpu().numpy(), scale * GRAD[base](Xn, Wn, Zn), rtol=0, atol=1e-9)
        AW = scale * (oracle.l1_rows if base == "l1" else oracle.l2sq_rows)(Xn, Wn)
        np.testing.assert_allclose(Z.grad.cpu().numpy(), AW, rtol=0, atol=1e-9)
