"""The variants of Appendix A on the GPU against the CPU oracle:
total variation (half the l1 product, and half its gradient), ||x - y||_p^p
for even p (the binomial expansion on centred coordinates) and odd p (p + 1
prefix sums in sorted order, Theorem "odd_p"), and the approximate l2
product through the Gaussian l2 -> l1 embedding.

FP32 within 1e-5 and FP64 within 1e-12 of the oracle on the same inputs
(for the embedding: the oracle's FP64 map of the same FP32 points and G),
int32 exact; the embedding's approximation of the exact l2 product is also
checked (a few percent at m = 1024, as Theorem "l2_approx" allows).
"""
import numpy as np
import pytest

import oracle
from oracle import parallel
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check(got, want, dtype, tol=None):
    if np.issubdtype(np.dtype(dtype), np.integer):
        np.testing.assert_array_equal(got, want)
    else:
        err = oracle.relative_error(got, want)
        assert err <= (tol or TOL[np.dtype(dtype).type]), f"relative error {err:.3e}"


# ------------------------------------------------------------ total variation
@pytest.mark.parametrize("n", [1, 100, 3001])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_tv_product_and_gradient(dm, ctx, n, dtype):
    X = inputs.simplex_points(n, 10, dtype=dtype)
    Z = inputs.gaussian_queries(n, 4, dtype=dtype)
    plan = dm.dm_prepare(ctx, "tv", dev(X))
    out = dm.dm_matmat(plan, dev(Z))
    W = inputs.gaussian_queries(n, 4, seed=9, dtype=dtype)
    G = dm.dm_grad(plan, dev(W), dev(Z))
    dm.dm_sync(ctx)
    check(out.cpu().numpy(), oracle.tv_rows(X, Z), dtype)
    check(G.cpu().numpy(), 0.5 * oracle.l1_grad_rows(X, W, Z), dtype)


def test_tv_rejects_integers(dm, ctx):
    with pytest.raises(dm.DMError):
        dm.dm_prepare(ctx, "tv", dev(np.zeros((10, 2), dtype=np.int32)))


# --------------------------------------------------------------- ||.||_p^p
@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int32])
@pytest.mark.parametrize("n", [1, 257, 4000])
def test_lpp_matches_definition(dm, ctx, p, dtype, n):
    rng = np.random.default_rng(p * 100 + n)
    if dtype == np.int32:
        hi = {2: 1 << 15, 3: 3000, 4: 1000, 5: 200, 6: 100, 7: 20}[p]
        X = rng.integers(-hi, hi, size=(n, 5)).astype(dtype)
        Z = rng.integers(-100, 101, size=(n, 3)).astype(dtype)
    else:
        X = rng.normal(0, 3, size=(n, 5)).astype(dtype)
        Z = rng.normal(size=(n, 3)).astype(dtype)
    plan = dm.dm_prepare_lpp(ctx, dev(X), p)
    out = dm.dm_matmat(plan, dev(Z))
    dm.dm_sync(ctx)
    want = oracle.lpp_rows(X, Z, p)
    check(out.cpu().numpy(), want, dtype)


def test_lpp_p2_equals_l2sq_plan(dm, ctx):
    X = np.random.default_rng(1).integers(0, 1 << 16, size=(3000, 7)).astype(np.int32)
    Z = np.random.default_rng(2).integers(-100, 101, size=(3000, 5)).astype(np.int32)
    a = dm.dm_matmat(dm.dm_prepare_lpp(ctx, dev(X), 2), dev(Z))
    b = dm.dm_matmat(dm.dm_prepare(ctx, "l2sq", dev(X)), dev(Z))
    assert torch.equal(a, b)


@pytest.mark.parametrize("p", [3, 5])
@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int32])
def test_lpp_odd_ties_across_tiles(dm, ctx, p, dtype):
    # four distinct values per coordinate: tie groups of about 1500 points
    # that span several 1024-position tiles; ties contribute |0|^p = 0
    rng = np.random.default_rng(31 + p)
    n = 6003
    X = rng.integers(-2, 2, size=(n, 4)).astype(dtype)
    X[:, 3] = 7                                   # one coordinate all tied
    Z = (rng.integers(-50, 51, size=(n, 5)) if dtype == np.int32
         else rng.normal(size=(n, 5))).astype(dtype)
    plan = dm.dm_prepare_lpp(ctx, dev(X), p)
    out = dm.dm_matmat(plan, dev(Z))
    dm.dm_sync(ctx)
    check(out.cpu().numpy(), oracle.lpp_rows(X, Z, p), dtype)


@pytest.mark.parametrize("p,n", [(3, 3000), (5, 1200), (7, 150)])
def test_lpp_odd_grid_closed_form(dm, ctx, p, n):
    # x_i = i, z = 1: sum_j |i - j|^p = S_p(i) + S_p(n - 1 - i), S_p the power
    # sums (Nicomachus / Faulhaber), exact in int64 from int32 points
    S = {3: lambda N: (N * (N + 1) // 2) ** 2,
         5: lambda N: N * N * (N + 1) ** 2 * (2 * N * N + 2 * N - 1) // 12,
         7: lambda N: N * N * (N + 1) ** 2 * (3 * N ** 4 + 6 * N ** 3 - N * N - 4 * N + 2) // 24}[p]
    X = np.arange(n, dtype=np.int32)[:, None]
    out = dm.dm_matmat(dm.dm_prepare_lpp(ctx, dev(X), p), dev(np.ones((n, 1), dtype=np.int32)))
    dm.dm_sync(ctx)
    want = np.array([[S(i) + S(n - 1 - i)] for i in range(n)], dtype=np.int64)
    np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_lpp_odd_strided_output(dm, ctx):
    # out is a column slice of a wider block (ldo > k): the columns outside
    # the slice are left as they were
    rng = np.random.default_rng(5)
    X = rng.normal(size=(2500, 6)).astype(np.float64)
    Z = rng.normal(size=(2500, 3))
    big = torch.full((2500, 8), 3.5, dtype=torch.float64, device="cuda")
    plan = dm.dm_prepare_lpp(ctx, dev(X), 3)
    dm.dm_matmat(plan, dev(Z), out=big[:, 2:5])
    dm.dm_sync(ctx)
    got = big.cpu().numpy()
    check(got[:, 2:5], oracle.lpp_rows(X, Z, 3), np.float64)
    assert np.all(got[:, :2] == 3.5) and np.all(got[:, 5:] == 3.5)


def test_lpp_odd_plan_is_the_l1_sort(dm, ctx):
    # an odd-p plan holds the same sorted coordinates as the l1 plan
    X = np.random.default_rng(8).integers(-50, 50, size=(3000, 3)).astype(np.int32)
    a = dm.dm_prepare_lpp(ctx, dev(X), 3)
    b = dm.dm_prepare(ctx, "l1", dev(X))
    va, pa = dm.dm_plan_export(a)
    vb, pb = dm.dm_plan_export(b)
    assert torch.equal(va, vb) and torch.equal(pa, pb)


def test_lpp_invalid_powers(dm, ctx):
    X = dev(np.zeros((10, 2), dtype=np.float32))
    for p in (0, 1, 17, 18):
        with pytest.raises(dm.DMError):
            dm.dm_prepare_lpp(ctx, X, p)


# ----------------------------------------------------- approximate l2 (embed)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n,d,m", [(1, 3, 8), (3001, 8, 64), (2500, 20, 130)])
def test_l2_embed_matches_oracle(dm, ctx, dtype, n, d, m):
    rng = np.random.default_rng(n + m)
    X = rng.normal(size=(n, d)).astype(dtype)
    Z = rng.normal(size=(n, 3)).astype(dtype)
    G = inputs.embedding_matrix(m, d, dtype=dtype)
    plan = dm.dm_prepare_l2_embed(ctx, dev(X), dev(G))
    out = dm.dm_matmat(plan, dev(Z))
    dm.dm_sync(ctx)
    tol = 1e-5 if dtype == np.float32 else 1e-12
    check(out.cpu().numpy(), oracle.l2_approx(X, G, Z), dtype, tol)


def test_l2_embed_approximates_l2(dm, ctx):
    rng = np.random.default_rng(7)
    n, d, m = 2000, 10, 1024
    X = rng.normal(size=(n, d)).astype(np.float32)
    Z = rng.normal(size=(n, 2)).astype(np.float32)
    G = inputs.embedding_matrix(m, d)
    plan = dm.dm_prepare_l2_embed(ctx, dev(X), dev(G))
    out = dm.dm_matmat(plan, dev(Z)).cpu().numpy()
    Xd = X.astype(np.float64)
    exact = np.sqrt(((Xd[:, None, :] - Xd[None, :, :]) ** 2).sum(-1)) @ Z.astype(np.float64)
    assert oracle.relative_error(out, exact) < 0.05


# ---------------------------------------------------------------- full size
def test_variants_full_size_whole_block(dm, ctx):
    # every variant on the step's workload (n = 2^20, d = 32, k = 16), the
    # whole block against the oracle's O(n d log n) or O(n d p k) forms, and
    # sampled rows once more against the definitions
    X, Z = inputs.workload_mixture_f32()
    rows = inputs.sample_rows(len(X), 4)
    Xd, Zd = dev(X), dev(Z)
    # ||.||_4^4 (even-p expansion) and ||.||_3^3 (odd p through sorted order)
    out = dm.dm_matmat(dm.dm_prepare_lpp(ctx, Xd, 4), Zd).cpu().numpy()
    check(out, oracle.lpp_even_expansion(X, Z, 4), np.float32)
    check(out[rows], oracle.lpp_rows(X, Z, 4, rows), np.float32)
    out = dm.dm_matmat(dm.dm_prepare_lpp(ctx, Xd, 3), Zd).cpu().numpy()
    check(out, parallel.lpp_odd_sort(X, Z, 3), np.float32)
    check(out[rows], oracle.lpp_rows(X, Z, 3, rows), np.float32)
    # approximate l2 with m = 256: Algorithms 1-2 on the mapped points
    G = inputs.embedding_matrix(256, X.shape[1])
    out = dm.dm_matmat(dm.dm_prepare_l2_embed(ctx, Xd, dev(G)), Zd).cpu().numpy()
    T = oracle.l2_embed(X, G)
    check(out, parallel.l1_sort(T, Z), np.float32)
    check(out[rows], oracle.l1_rows(T, Z, rows), np.float32)
    # total variation on distributions
    P = inputs.simplex_points(len(X), X.shape[1])
    out = dm.dm_matmat(dm.dm_prepare(ctx, "tv", dev(P)), Zd).cpu().numpy()
    check(out, 0.5 * parallel.l1_sort(P, Z), np.float32)
    check(out[rows], oracle.tv_rows(P, Z, rows), np.float32)
    dm.dm_sync(ctx)
