"""Batches of independent point sets (dm_batch_*) against the CPU oracle.

Every set of a batch is checked on its own: against the definition where
n^2 (d + k) is small, otherwise the oracle's sort-based form (l1) or p = 2
identity (squared l2) -- FP32 within 1e-5, FP64 within 1e-12, int32 exact.
The graph is replayed after the inputs change in place, with fixed lanes and
with the autotuner's choice, and the full-size workload (512 sets, n
log-uniform in [1024, 262144], d in 2..64, k in 1..32) is checked on sampled
rows of a sample of sets.
"""
import numpy as np
import pytest

import oracle
from paper_2210_15114_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {np.float32: 1e-5, np.float64: 1e-12}


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


def reference(metric, X, Z):
    n, d = X.shape
    if n * n * (d + Z.shape[1]) <= 2e8:
        return (oracle.l1_rows if metric == "l1" else oracle.l2sq_rows)(X, Z)
    return oracle.l1_sort(X, Z) if metric == "l1" else oracle.l2sq_identity(X, Z)


def check(got, want, dtype):
    if np.issubdtype(np.dtype(dtype), np.integer):
        np.testing.assert_array_equal(got, want)
    else:
        err = oracle.relative_error(got, want)
        assert err <= TOL[np.dtype(dtype).type], f"relative error {err:.3e}"


def small_sets(dtype, nsets=24):
    return inputs.workload_batch(nsets=nsets, n_lo=1, n_hi=6000, d_lo=1, d_hi=9, k_lo=1, k_hi=6,
                                 seed0=77, dtype=dtype)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int32])
@pytest.mark.parametrize("lanes", [1, 3, 0])
def test_batch_matches_oracle(dm, ctx, metric, dtype, lanes):
    sets = small_sets(dtype)
    Xs = [torch.from_numpy(X).cuda() for X, _ in sets]
    Zs = [torch.from_numpy(Z).cuda() for _, Z in sets]
    b = dm.dm_batch_create(ctx, metric, Xs, Zs, lanes=lanes)
    assert 1 <= dm.dm_batch_lanes(b) <= 16
    outs = dm.dm_batch_run(b)
    dm.dm_sync(ctx)
    for (X, Z), o in zip(sets, outs):
        check(o.cpu().numpy(), reference(metric, X, Z), dtype)
    # change the inputs in place and replay the same graph
    rng = np.random.default_rng(5)
    new = []
    for (X, Z), Xd, Zd in zip(sets, Xs, Zs):
        if np.issubdtype(np.dtype(dtype), np.integer):
            X2 = rng.integers(-500, 500, size=X.shape).astype(dtype)
            Z2 = rng.integers(-9, 10, size=Z.shape).astype(dtype)
        else:
            X2 = rng.normal(size=X.shape).astype(dtype)
            Z2 = rng.normal(size=Z.shape).astype(dtype)
        Xd.copy_(torch.from_numpy(X2))
        Zd.copy_(torch.from_numpy(Z2))
        new.append((X2, Z2))
    outs = dm.dm_batch_run(b)
    dm.dm_sync(ctx)
    for (X, Z), o in zip(new, outs):
        check(o.cpu().numpy(), reference(metric, X, Z), dtype)
    dm.dm_batch_destroy(b)


@pytest.mark.parametrize("lanes", [1, 4])
def test_batch_l2sq_tensor_engine(dm, lanes):
    # the graph captures the tensor-core contraction when the context asks
    # for it; FP32 sets of uneven size, replayed twice
    c = dm.dm_create(0)
    dm.dm_set_engine(c, "tensor")
    sets = small_sets(np.float32)
    Xs = [torch.from_numpy(X).cuda() for X, _ in sets]
    Zs = [torch.from_numpy(Z).cuda() for _, Z in sets]
    b = dm.dm_batch_create(c, "l2sq", Xs, Zs, lanes=lanes)
    for _ in range(2):
        outs = dm.dm_batch_run(b)
        dm.dm_sync(c)
        for (X, Z), o in zip(sets, outs):
            check(o.cpu().numpy(), reference("l2sq", X, Z), np.float32)
    dm.dm_batch_destroy(b)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_batch_total_variation(dm, ctx, dtype):
    sets = [(inputs.simplex_points(n, d, seed=s, dtype=dtype), inputs.gaussian_queries(n, k, seed=s, dtype=dtype))
            for s, (n, d, k) in enumerate([(1, 3, 1), (700, 5, 2), (5000, 8, 3), (2049, 2, 4)])]
    Xs = [torch.from_numpy(X).cuda() for X, _ in sets]
    Zs = [torch.from_numpy(Z).cuda() for _, Z in sets]
    b = dm.dm_batch_create(ctx, "tv", Xs, Zs, lanes=2)
    outs = dm.dm_batch_run(b)
    dm.dm_sync(ctx)
    for (X, Z), o in zip(sets, outs):
        check(o.cpu().numpy(), oracle.tv_rows(X, Z), dtype)
    dm.dm_batch_destroy(b)


def test_batch_equals_single_calls_exactly_on_integers(dm, ctx):
    sets = small_sets(np.int32, nsets=10)
    Xs = [torch.from_numpy(X).cuda() for X, _ in sets]
    Zs = [torch.from_numpy(Z).cuda() for _, Z in sets]
    for metric in ("l1", "l2sq"):
        b = dm.dm_batch_create(ctx, metric, Xs, Zs, lanes=4)
        outs = [o.clone() for o in dm.dm_batch_run(b)]
        for Xd, Zd, o in zip(Xs, Zs, outs):
            plan = dm.dm_prepare(ctx, metric, Xd)
            single = dm.dm_matmat(plan, Zd)
            assert torch.equal(single, o)
        dm.dm_batch_destroy(b)


def test_batch_reports_nonfinite_through_sync(dm, ctx):
    sets = small_sets(np.float32, nsets=5)
    Xs = [torch.from_numpy(X).cuda() for X, _ in sets]
    Zs = [torch.from_numpy(Z).cuda() for _, Z in sets]
    Xs[3][0, 0] = float("nan")
    b = dm.dm_batch_create(ctx, "l1", Xs, Zs, lanes=2)
    dm.dm_sync(ctx)                # capturing with fixed lanes runs nothing
    dm.dm_batch_run(b)
    with pytest.raises(dm.DMError):
        dm.dm_sync(ctx)
    dm.dm_sync(ctx)                # the error word was cleared
    dm.dm_batch_destroy(b)


def test_batch_invalid_arguments(dm, ctx):
    X = torch.zeros((10, 2), device="cuda")
    Z = torch.zeros((10, 1), device="cuda")
    with pytest.raises(dm.DMError):
        dm.dm_batch_create(ctx, "l1", [X], [Z, Z])
    with pytest.raises(dm.DMError):
        dm.dm_batch_create(ctx, "l1", [X, X.double()], [Z, Z.double()])


def test_batch_full_size_sampled(dm, ctx):
    sets = inputs.workload_batch()
    Xs = [torch.from_numpy(X).cuda() for X, _ in sets]
    Zs = [torch.from_numpy(Z).cuda() for _, Z in sets]
    rng = np.random.default_rng(9)
    pick = rng.choice(len(sets), size=12, replace=False)
    for metric in ("l1", "l2sq"):
        b = dm.dm_batch_create(ctx, metric, Xs, Zs, lanes=0)
        outs = dm.dm_batch_run(b)
        dm.dm_sync(ctx)
        for s in pick:
            X, Z = sets[s]
            rows = inputs.sample_rows(len(X), 6)
            want = (oracle.l1_rows if metric == "l1" else oracle.l2sq_rows)(X, Z, rows)
            check(outs[s].cpu().numpy()[rows], want, np.float32)
        dm.dm_batch_destroy(b)
