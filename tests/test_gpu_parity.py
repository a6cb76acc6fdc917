"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (Frobenius relative error over the whole block, against the FP64
oracle evaluated on the same input values): 1e-12 for FP64 inputs, 1e-5 for
FP32 inputs; int32 inputs are bit-exact (int64 results).  Every case, the
full-size workloads (n = 2^20, d = 32, k = 16) included, is compared on the
whole output block: small cases against the definition, large ones against
the oracle's sort-based form of Algorithms 1-2 (l1) or the p = 2 identity of
Appendix A (squared l2), which are pinned to the definition.  At full size
each FP32 element is also held to an error bound of its own,
|out_ij - (AZ)_ij| <= 1e-5 (A|Z|)_ij, the scale that bounds the rounding of a
sum of the terms A_il Z_lj in any order; a seeded sample of rows is checked
once more against the definition, and w^T (A z) = z^T (A w) is checked.
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


@pytest.fixture(scope="module")
def ctx_ordered(dm):
    c = dm.dm_create(0)
    dm.dm_set_deterministic(c, True)
    return c


@pytest.fixture(params=["atomic", "ordered"])
def mctx(request, ctx, ctx_ordered):
    """Both accumulation modes of the l1 query (squared l2 ignores it)."""
    return ctx if request.param == "atomic" else ctx_ordered


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_product(dm, ctx, metric, X, Z):
    plan = dm.dm_prepare(ctx, metric, dev(X))
    out = dm.dm_matmat(plan, dev(Z))
    dm.dm_sync(ctx)
    return out.cpu().numpy()


def reference(metric, X, Z):
    # The definition (double loop) where it is cheap; otherwise the oracle's
    # sort-based form (l1) or p = 2 identity (squared l2), both pinned to the
    # definition.  (At n = 1 the exact product is 0, which only the definition
    # reproduces exactly; the identity leaves an FP64 cancellation residue.)
    n = len(X)
    d = 1 if np.ndim(X) == 1 else X.shape[1]
    k = 1 if np.ndim(Z) == 1 else Z.shape[1]
    if n * n * (d + k) <= 2e8:
        return (oracle.l1_rows if metric == "l1" else oracle.l2sq_rows)(X, Z)
    return oracle.l1_sort(X, Z) if metric == "l1" else oracle.l2sq_identity(X, Z)


def check(got, want, dtype):
    if np.issubdtype(np.dtype(dtype), np.integer):
        np.testing.assert_array_equal(got, want)
    else:
        err = oracle.relative_error(got, want)
        assert err <= TOL[dtype], f"relative error {err:.3e}"


# ------------------------------------------------------------ small configs
@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_small_fp64_workload(dm, ctx, metric):
    # n = 4096, d = 8, U[0,1) FP64, one N(0,1) query, every row vs the definition.
    X, z = inputs.workload_small_f64()
    plan = dm.dm_prepare(ctx, metric, dev(X))
    fn = dm.dm_matvec_l1 if metric == "l1" else dm.dm_matvec_l2sq
    out = fn(plan, dev(z[:, 0]))
    dm.dm_sync(ctx)
    want = (oracle.l1_rows if metric == "l1" else oracle.l2sq_rows)(X, z[:, 0])
    assert oracle.relative_error(out.cpu().numpy(), want) <= 1e-12


@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.int32])
@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_grid_closed_form(dm, ctx, metric, dtype):
    n = 4096
    X = inputs.grid_1d(n).astype(dtype)
    z = np.ones(n, dtype=dtype)
    i = np.arange(n, dtype=np.int64)
    if metric == "l1":
        want = i * (i + 1) // 2 + (n - 1 - i) * (n - i) // 2
    else:
        want = i * (i + 1) * (2 * i + 1) // 6 + (n - 1 - i) * (n - i) * (2 * n - 2 * i - 1) // 6
    out = gpu_product(dm, ctx, metric, X, z.reshape(n, 1))[:, 0]
    if dtype == np.float32:
        assert oracle.relative_error(out, want) <= 1e-5
    else:
        np.testing.assert_array_equal(out, want.astype(out.dtype))


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
@pytest.mark.parametrize("n", [1, 2, 3, 767, 768, 769, 1537, 4095, 4097, 20011])
def test_fp32_mixture_sizes(dm, mctx, metric, n):
    X, Z = inputs.workload_mixture_f32(n=n, d=32, k=16)
    check(gpu_product(dm, mctx, metric, X, Z), reference(metric, X, Z), np.float32)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
@pytest.mark.parametrize("k", [1, 2, 3, 5, 8, 16, 17, 40])
def test_query_block_widths(dm, mctx, metric, k):
    X, Z = inputs.workload_mixture_f32(n=5000, d=7, k=k)
    check(gpu_product(dm, mctx, metric, X, Z), reference(metric, X, Z), np.float32)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
@pytest.mark.parametrize("dtype", [np.float64, np.int32])
@pytest.mark.parametrize("k", [1, 3, 16, 20])
def test_other_types(dm, mctx, metric, dtype, k):
    ctx = mctx
    n, d = 6007, 5
    if dtype == np.int32:
        X = inputs.integer_points(n, d, 3, 0, 1 << 16)
        Z = inputs.integer_queries(n, k, 4)
    else:
        X = inputs.uniform_points(n, d, 3, dtype=np.float64)
        Z = inputs.gaussian_queries(n, k, 4, dtype=np.float64)
    check(gpu_product(dm, ctx, metric, X, Z), reference(metric, X, Z), dtype)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_integer_ties_exact(dm, mctx, metric):
    ctx = mctx
    rng = np.random.default_rng(21)
    X = rng.integers(0, 6, size=(9000, 4)).astype(np.int32)
    Z = rng.integers(-100, 101, size=(9000, 3)).astype(np.int32)
    check(gpu_product(dm, ctx, metric, X, Z), reference(metric, X, Z), np.int32)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_fp32_ties_signed_zeros_negatives(dm, ctx, metric):
    rng = np.random.default_rng(22)
    X = rng.normal(size=(7000, 6)).astype(np.float32)
    X[::3, 0] = 0.0
    X[1::3, 0] = -0.0
    X[:, 1] = np.round(X[:, 1] * 4) / 4
    X[:, 2] = -np.abs(X[:, 2])
    Z = rng.normal(size=(7000, 4)).astype(np.float32)
    check(gpu_product(dm, ctx, metric, X, Z), reference(metric, X, Z), np.float32)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_fp32_offset_coordinates(dm, ctx, metric):
    # Large common offset: the product is translation invariant; the kernels
    # work in shifted frames.
    X = (1000.0 + inputs.uniform_points(8000, 6, 5)).astype(np.float32)
    Z = inputs.gaussian_queries(8000, 3, 6)
    check(gpu_product(dm, ctx, metric, X, Z), reference(metric, X, Z), np.float32)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_identical_points_give_zero(dm, ctx, metric):
    X = np.full((3000, 5), 2.5, dtype=np.float32)
    Z = inputs.gaussian_queries(3000, 4, 2)
    out = gpu_product(dm, ctx, metric, X, Z)
    assert np.all(out == 0)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_leading_dimensions(dm, mctx, metric):
    ctx = mctx
    n, d, k = 4000, 6, 5
    Xb = inputs.gaussian_mixture(n, d + 3, 4, 9)
    Zb = inputs.gaussian_queries(n, k + 2, 10)
    X, Z = Xb[:, :d], Zb[:, :k]
    Xd = dev(Xb)[:, :d]
    Zd = dev(Zb)[:, :k]
    outb = torch.full((n, k + 4), 7.0, device="cuda")
    plan = dm.dm_prepare(ctx, metric, Xd)
    dm.dm_matmat(plan, Zd, out=outb[:, :k])
    dm.dm_sync(ctx)
    got = outb.cpu().numpy()
    check(got[:, :k], reference(metric, X, Z), np.float32)
    assert np.all(got[:, k:] == 7.0)


def test_sort_matches_stable_argsort(dm, ctx):
    for n, dtype in [(1, np.float32), (2, np.float32), (4095, np.float32), (4096, np.float32),
                     (4097, np.float32), (30001, np.float32), (3000, np.float64),
                     (5000, np.int32)]:
        if dtype == np.int32:
            X = inputs.integer_points(n, 5, 1, -50, 50)
        else:
            X = inputs.gaussian_mixture(n, 5, 3, 1).astype(dtype)
            X[::4, 3] = X[0, 3]                        # ties
        plan = dm.dm_prepare(ctx, "l1", dev(X))
        vals, perm = dm.dm_plan_export(plan)
        dm.dm_sync(ctx)
        vals, perm = vals.cpu().numpy(), perm.cpu().numpy()
        for c in range(X.shape[1]):
            order = oracle.preprocessing_order(X[:, c])
            np.testing.assert_array_equal(perm[c], order)
            np.testing.assert_array_equal(vals[c], X[order, c])


def test_sort_signed_zeros_valid(dm, ctx):
    X = np.zeros((5000, 1), dtype=np.float32)
    X[::2, 0] = -0.0
    X[::7, 0] = 1.5
    X[::11, 0] = -2.0
    plan = dm.dm_prepare(ctx, "l1", dev(X))
    vals, perm = dm.dm_plan_export(plan)
    dm.dm_sync(ctx)
    vals, perm = vals.cpu().numpy()[0], perm.cpu().numpy()[0]
    assert np.all(np.diff(vals) >= 0)
    assert np.array_equal(np.sort(perm), np.arange(5000))
    np.testing.assert_array_equal(vals, X[perm, 0])


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_deterministic(dm, ctx, ctx_ordered, metric):
    # Ordered accumulation: identical bits run to run.  L2-reduction mode:
    # the same values up to the order of the d additions.
    X, Z = inputs.workload_mixture_f32(n=50000, d=12, k=16)
    a = gpu_product(dm, ctx_ordered, metric, X, Z)
    b = gpu_product(dm, ctx_ordered, metric, X, Z)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    c = gpu_product(dm, ctx, metric, X, Z)
    assert oracle.relative_error(c, a) <= 1e-6


def test_matvec_entry_points_reject_wrong_metric(dm, ctx):
    X = inputs.uniform_points(100, 2, 1, dtype=np.float32)
    z = dev(np.ones(100, dtype=np.float32))
    p1 = dm.dm_prepare(ctx, "l1", dev(X))
    p2 = dm.dm_prepare(ctx, "l2sq", dev(X))
    with pytest.raises(dm.DMError):
        dm.dm_matvec_l2sq(p1, z)
    with pytest.raises(dm.DMError):
        dm.dm_matvec_l1(p2, z)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_nonfinite_rejected(dm, ctx, metric):
    # l1 reports it from dm_prepare (which synchronizes), squared l2 from the
    # next dm_sync.
    X = inputs.uniform_points(1000, 3, 1, dtype=np.float32)
    X[17, 1] = np.nan
    with pytest.raises(dm.DMError) as e:
        dm.dm_prepare(ctx, metric, dev(X))
        dm.dm_sync(ctx)
    assert e.value.status == dm.DM_ERR_NONFINITE
    X[17, 1] = np.inf
    with pytest.raises(dm.DMError):
        dm.dm_prepare(ctx, metric, dev(X))
        dm.dm_sync(ctx)
    # the context stays usable
    X[17, 1] = 0.5
    Z = inputs.gaussian_queries(1000, 2, 1)
    check(gpu_product(dm, ctx, metric, X, Z), reference(metric, X, Z), np.float32)


def test_invalid_arguments(dm, ctx):
    X = dev(inputs.uniform_points(100, 2, 1, dtype=np.float32))
    with pytest.raises(dm.DMError) as e:
        dm.dm_prepare(ctx, "l1", X[:0])
    assert e.value.status == dm.DM_ERR_INVALID_ARG
    plan = dm.dm_prepare(ctx, "l1", X)
    with pytest.raises(dm.DMError):
        dm.dm_matmat(plan, dev(np.ones((100, 2), dtype=np.float64)))


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int32])
def test_bruteforce_kernel(dm, ctx, metric, dtype):
    n, d, k = 3001, 9, 17
    if dtype == np.int32:
        X = inputs.integer_points(n, d, 2, 0, 1000)
        Z = inputs.integer_queries(n, k, 3)
    else:
        X = inputs.gaussian_mixture(n, d, 4, 2).astype(dtype)
        Z = inputs.gaussian_queries(n, k, 3).astype(dtype)
    out = dm.dm_bruteforce(ctx, metric, dev(X), dev(Z))
    dm.dm_sync(ctx)
    want = (oracle.l1_rows if metric == "l1" else oracle.l2sq_rows)(X, Z)
    check(out.cpu().numpy(), want, dtype)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_host_entry_point(dm, ctx, metric):
    X, Z = inputs.workload_mixture_f32(n=12000, d=10, k=6)
    got = dm.dm_matmat_host(ctx, metric, X, Z)
    check(got, reference(metric, X, Z), np.float32)


def test_host_entry_point_async(dm, ctx):
    # two contexts, calls issued from one thread (copies in issue order on the
    # host link), results read after dm_sync; a second round with new Z and
    # the same buffers, then a blocking call on the first context
    X, Z = inputs.workload_mixture_f32(n=30011, d=12, k=5)
    Z2 = (Z[::-1] * 0.5 + 1.0).copy()
    ctx2 = dm.dm_create(0)
    try:
        for Zq in (Z, Z2):
            o1 = dm.dm_matmat_host_async(ctx, "l1", X, Zq)
            o2 = dm.dm_matmat_host_async(ctx2, "l2sq", X, Zq)
            dm.dm_sync(ctx)
            dm.dm_sync(ctx2)
            check(o1, reference("l1", X, Zq), np.float32)
            check(o2, reference("l2sq", X, Zq), np.float32)
        o3 = dm.dm_matmat_host_async(ctx, "l2sq", X, Z)
        o4 = dm.dm_matmat_host(ctx, "l1", X, Z2)       # waits for the first call's copy of Z
        dm.dm_sync(ctx)
        check(o3, reference("l2sq", X, Z), np.float32)
        check(o4, reference("l1", X, Z2), np.float32)
    finally:
        dm.dm_destroy(ctx2)


@pytest.mark.parametrize("metrics", [("l1", "l2sq"), ("l2sq", "l1"), ("l1",), ("l2sq", "l2sq", "l1")])
def test_host_entry_point_multi(dm, ctx, metrics):
    # one copy of X and Z for every product, products on peer contexts; twice
    # in a row (the second call reuses the peers and buffers), then FP64 and
    # int32 inputs on the same context
    X, Z = inputs.workload_mixture_f32(n=20011, d=9, k=7)
    for Zq in (Z, (Z * -0.25 + 0.5).astype(np.float32)):
        outs = dm.dm_matmat_host_multi(ctx, list(metrics), X, Zq)
        for m, o in zip(metrics, outs):
            check(o, reference(m, X, Zq), np.float32)
    X64, Z64 = X.astype(np.float64), Z.astype(np.float64)
    for m, o in zip(metrics, dm.dm_matmat_host_multi(ctx, list(metrics), X64, Z64)):
        check(o, reference(m, X64, Z64), np.float64)
    Xi = inputs.integer_points(5003, 4, 2, 0, 1000)
    Zi = inputs.integer_queries(5003, 3, 3)
    for m, o in zip(metrics, dm.dm_matmat_host_multi(ctx, list(metrics), Xi, Zi)):
        check(o, reference(m, Xi, Zi), np.int32)


def test_host_entry_point_multi_rejects(dm, ctx):
    X, Z = inputs.workload_mixture_f32(n=100, d=3, k=2)
    with pytest.raises(dm.DMError):
        dm.dm_matmat_host_multi(ctx, [], X, Z)
    with pytest.raises(dm.DMError):
        dm.dm_matmat_host_multi(ctx, ["l1", "tv"], X, Z)          # TV has its own entry points
    with pytest.raises(dm.DMError):
        dm.dm_matmat_host_multi(ctx, ["l1"] * 9, X, Z)             # at most 8 products
    with pytest.raises(dm.DMError):
        dm.dm_matmat_host_multi(ctx, ["l1", "l2sq"], X, Z, outs=[np.empty((100, 2), np.float32)])


# ----------------------------------------------------------- full size
@pytest.fixture(scope="module")
def full_fp32():
    return inputs.workload_mixture_f32()


@pytest.fixture(scope="module")
def full_int():
    return inputs.workload_integer()


def sort_form(metric, X, Z):
    """The oracle's O(n d log n) form of the whole block: Algorithms 1-2 with
    the coordinates on parallel host processes (l1), or the p = 2 identity."""
    return parallel.l1_sort(X, Z) if metric == "l1" else oracle.l2sq_identity(X, Z)


@pytest.fixture(scope="module")
def full_fp32_ref(full_fp32):
    X, Z = full_fp32
    absZ = np.abs(Z)
    return {m: (sort_form(m, X, Z), sort_form(m, X, absZ)) for m in ("l1", "l2sq")}


@pytest.fixture(scope="module")
def full_int_ref(full_int):
    X, Z = full_int
    return {m: sort_form(m, X, Z) for m in ("l1", "l2sq")}


def check_elementwise(got, want, scale, tol):
    """|got - want| <= tol * scale element by element (scale = A |Z|)."""
    bad = np.abs(got.astype(np.float64) - want) > tol * scale
    assert not bad.any(), (f"{int(bad.sum())} elements out of bound, first at "
                           f"{np.argwhere(bad)[0].tolist()}")


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_full_size_fp32_whole_block(dm, mctx, metric, full_fp32, full_fp32_ref):
    X, Z = full_fp32
    want, scale = full_fp32_ref[metric]
    out = gpu_product(dm, mctx, metric, X, Z)
    assert np.all(np.isfinite(out))
    err = oracle.relative_error(out, want)
    assert err <= 1e-5, f"relative error {err:.3e}"
    check_elementwise(out, want, scale, 1e-5)
    # second opinion on sampled rows: the definition, row by row
    rows = inputs.sample_rows(len(X), 8)
    assert oracle.relative_error(out[rows], (oracle.l1_rows if metric == "l1" else oracle.l2sq_rows)(X, Z, rows)) <= 1e-5


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_full_size_int_whole_block_exact(dm, mctx, metric, full_int, full_int_ref):
    X, Z = full_int
    out = gpu_product(dm, mctx, metric, X, Z)
    np.testing.assert_array_equal(out, full_int_ref[metric])
    rows = inputs.sample_rows(len(X), 4)
    np.testing.assert_array_equal(out[rows], (oracle.l1_rows if metric == "l1" else oracle.l2sq_rows)(X, Z, rows))


@pytest.mark.parametrize("dtype,k", [(np.float32, 12), (np.float64, 6), (np.int32, 10)])
def test_l1_large_n_narrow_column_groups(dm, mctx, dtype, k):
    # n above the size where one full column group's copies of Z and of the
    # output outgrow L2: the l1 query takes half-width groups (4 FP32 / int32,
    # 2 FP64 columns), with a ragged last group and a ragged last tile
    n, d = (1 << 21) + 37, 3
    rng = np.random.default_rng(211)
    if dtype == np.int32:
        X = rng.integers(0, 1 << 16, size=(n, d)).astype(dtype)
        Z = rng.integers(-100, 101, size=(n, k)).astype(dtype)
    else:
        X = rng.normal(0, 4, size=(n, d)).astype(dtype)
        Z = rng.normal(size=(n, k)).astype(dtype)
    out = gpu_product(dm, mctx, "l1", X, Z)
    want = parallel.l1_sort(X, Z)
    if dtype == np.int32:
        np.testing.assert_array_equal(out, want)
    else:
        assert oracle.relative_error(out, want) <= TOL[dtype]
    rows = np.concatenate([inputs.sample_rows(n, 4), [0, n - 1]])
    check(out[rows], oracle.l1_rows(X, Z, rows), dtype)


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_full_size_symmetry(dm, ctx, metric, full_fp32):
    # w^T (A z) = z^T (A w) for the symmetric A, at full size.
    X, Z = full_fp32
    plan = dm.dm_prepare(ctx, metric, dev(X))
    Zd = dev(Z)
    out = dm.dm_matmat(plan, Zd).double()
    dm.dm_sync(ctx)
    G = Zd.double().T @ out                       # G[a,b] = z_a^T A z_b
    asym = (G - G.T).abs().max().item()
    assert asym <= 1e-5 * G.abs().max().item()


@pytest.mark.parametrize("dtype,d,k", [(np.float32, 64, 100), (np.float64, 40, 70), (np.int32, 64, 33)])
def test_l2sq_wide_blocks_in_column_chunks(dm, ctx, dtype, d, k):
    # wider blocks than one reduce launch takes run in column chunks
    rng = np.random.default_rng(d + k)
    if dtype == np.int32:
        X = rng.integers(0, 1 << 16, size=(3000, d)).astype(dtype)
        Z = rng.integers(-100, 101, size=(3000, k)).astype(dtype)
    else:
        X = rng.normal(0, 4, size=(3000, d)).astype(dtype)
        Z = rng.normal(size=(3000, k)).astype(dtype)
    check(gpu_product(dm, ctx, "l2sq", X, Z), reference("l2sq", X, Z), dtype)


# ------------------------------------------------ squared-l2 engine switch
@pytest.fixture(scope="module")
def ctx_tensor(dm):
    c = dm.dm_create(0)
    dm.dm_set_engine(c, "tensor")
    return c


@pytest.mark.parametrize("n,d,k", [(1, 1, 1), (63, 3, 5), (1000, 8, 16), (3001, 32, 17),
                                   (2048, 126, 16), (70001, 16, 40), (5000, 30, 64)])
def test_l2sq_tensor_engine(dm, ctx_tensor, n, d, k):
    # the tensor engine at shapes its kernels partly refuse: k not a multiple
    # of 4 or above 32, d + 2 = 128 (the CUDA-core reduce then takes over),
    # ragged n
    rng = np.random.default_rng(n + d + k)
    X = rng.normal(0, 3, size=(n, d)).astype(np.float32)
    Z = rng.normal(size=(n, k)).astype(np.float32)
    out = gpu_product(dm, ctx_tensor, "l2sq", X, Z)
    assert oracle.relative_error(out, oracle.l2sq_identity(X, Z)) <= 1e-5
    rows = np.unique(np.concatenate([inputs.sample_rows(n, 16), [0, n - 1]]))
    assert oracle.relative_error(out[rows], oracle.l2sq_rows(X, Z, rows)) <= 1e-5


@pytest.mark.parametrize("n,d,k", [(1, 4, 1), (127, 8, 5), (128, 12, 16), (129, 20, 31), (4097, 28, 32),
                                   (70001, 32, 16), (300, 32, 17), (5000, 4, 3)])
def test_l2sq_tensor_apply_shapes(dm, ctx_tensor, n, d, k):
    # the apply on tcgen05 (d a multiple of 4 up to 32, k up to 32): ragged
    # tiles of 128 points, k padded to 16 / 32, one-point tiles; the whole
    # block against the p = 2 identity, on points shifted far from the origin
    rng = np.random.default_rng(7 * n + d + k)
    X = (rng.normal(0, 3, size=(n, d)) + 50.0).astype(np.float32)
    Z = rng.normal(size=(n, k)).astype(np.float32)
    out = gpu_product(dm, ctx_tensor, "l2sq", X, Z)
    want = oracle.l2sq_identity(X, Z) if n > 1 else oracle.l2sq_rows(X, Z)
    assert oracle.relative_error(out, want) <= 1e-5


@pytest.mark.parametrize("n,d,k", [(1, 4, 4), (63, 8, 8), (64, 12, 16), (65, 28, 12), (1000, 32, 4),
                                   (4097, 32, 32), (70001, 16, 20), (3000, 44, 16), (2500, 60, 32),
                                   (129, 60, 4), (100003, 32, 16)])
def test_l2sq_tensor_reduce_shapes(dm, ctx, n, d, k):
    # the tensor-core reduce (the default engine for these shapes: d and k
    # multiples of 4, d <= 60, k <= 16 or d >= 48, and the tensor engine
    # beyond): 64-point chunks cut off at n, 2 (d + 2) rows of hi and lo
    # packed into the 128-row tile, k rounded up to 8; points shifted far from
    # the origin (the centring) -- whole block against the p = 2 identity,
    # under the default engine and under DM_ENGINE_TENSOR_CORES
    rng = np.random.default_rng(11 * n + d + k)
    X = (rng.normal(0, 3, size=(n, d)) + 50.0).astype(np.float32)
    Z = rng.normal(size=(n, k)).astype(np.float32)
    want = oracle.l2sq_identity(X, Z) if n > 1 else oracle.l2sq_rows(X, Z)
    for c in (ctx, dm.dm_create(0)):
        if c is not ctx:
            dm.dm_set_engine(c, "tensor")
        out = gpu_product(dm, c, "l2sq", X, Z)
        assert oracle.relative_error(out, want) <= 1e-5


def test_l2sq_tensor_reduce_without_norms(dm, ctx):
    # the reduce without the s row (the squared-l2 gradient packs (z, w) as
    # 2k columns; k = 2 and 8 give 4 and 16 packed columns) and with
    # precomputed features and no shift (even p: d p = 16 columns)
    rng = np.random.default_rng(23)
    n, d = 5003, 8
    X = rng.normal(size=(n, d)).astype(np.float32)
    plan = dm.dm_prepare(ctx, "l2sq", dev(X))
    for k in (2, 8):
        W = rng.normal(size=(n, k)).astype(np.float32)
        Z = rng.normal(size=(n, k)).astype(np.float32)
        G = dm.dm_grad(plan, dev(W), dev(Z)).cpu().numpy()
        assert oracle.relative_error(G, oracle.l2sq_grad_closed(X, W, Z)) <= 1e-5
    X4 = rng.normal(size=(n, 4)).astype(np.float32)
    Z4 = rng.normal(size=(n, 4)).astype(np.float32)
    out = dm.dm_matmat(dm.dm_prepare_lpp(ctx, dev(X4), 4), dev(Z4)).cpu().numpy()
    assert oracle.relative_error(out, oracle.lpp_even_expansion(X4, Z4, 4)) <= 1e-5
    dm.dm_sync(ctx)


def test_l2sq_tensor_apply_strided_points_fall_back(dm, ctx_tensor):
    # rows of X not contiguous (ldx > d): the CUDA-core apply takes over
    rng = np.random.default_rng(3)
    Xw = rng.normal(size=(2000, 12)).astype(np.float32)
    Z = rng.normal(size=(2000, 6)).astype(np.float32)
    plan = dm.dm_prepare(ctx_tensor, "l2sq", dev(Xw)[:, :8])
    out = dm.dm_matmat(plan, dev(Z)).cpu().numpy()
    dm.dm_sync(ctx_tensor)
    assert oracle.relative_error(out, oracle.l2sq_identity(Xw[:, :8], Z)) <= 1e-5


def test_l2sq_tensor_engine_full_size(dm, ctx_tensor, full_fp32, full_fp32_ref):
    X, Z = full_fp32
    want, scale = full_fp32_ref["l2sq"]
    out = gpu_product(dm, ctx_tensor, "l2sq", X, Z)
    assert oracle.relative_error(out, want) <= 1e-5
    check_elementwise(out, want, scale, 1e-5)


def test_tensor_engine_gradient_and_even_p(dm, ctx_tensor):
    rng = np.random.default_rng(17)
    X = rng.normal(size=(4000, 6)).astype(np.float32)
    W = rng.normal(size=(4000, 3)).astype(np.float32)
    Z = rng.normal(size=(4000, 3)).astype(np.float32)
    plan = dm.dm_prepare(ctx_tensor, "l2sq", dev(X))
    G = dm.dm_grad(plan, dev(W), dev(Z)).cpu().numpy()
    assert oracle.relative_error(G, oracle.l2sq_grad_rows(X, W, Z)) <= 1e-5
    out = dm.dm_matmat(dm.dm_prepare_lpp(ctx_tensor, dev(X), 4), dev(Z)).cpu().numpy()
    assert oracle.relative_error(out, oracle.lpp_rows(X, Z, 4)) <= 1e-5
    dm.dm_sync(ctx_tensor)


def test_engine_rejects_unknown(dm, ctx):
    with pytest.raises(dm.DMError):
        dm.dm_set_engine(ctx, "fpga")
    lib = dm.load()
    assert lib.dm_set_engine(ctx.handle, 7) == 1


@pytest.mark.parametrize("metric", ["l1", "l2sq"])
def test_strided_vector_query_and_result(dm, ctx, metric):
    # a column view of a wider block as the query and another as the result:
    # the binding passes the element stride as the leading dimension
    X, Z = inputs.workload_mixture_f32(n=3001, d=5, k=4)
    plan = dm.dm_prepare(ctx, metric, dev(X))
    Zd = dev(Z)
    outfull = torch.zeros((3001, 3), dtype=torch.float32, device="cuda")
    dm.dm_matmat(plan, Zd[:, 1], out=outfull[:, 2])
    dm.dm_sync(ctx)
    got = outfull.cpu().numpy()
    assert oracle.relative_error(got[:, 2], reference(metric, X, Z[:, 1])) <= 1e-5
    assert not got[:, :2].any()
    with pytest.raises(dm.DMError):
        dm.dm_matmat(plan, Zd[:3000])                      # rows differ from the plan's n
