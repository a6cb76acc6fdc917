"""The dense tall-skinny products of the block Krylov iteration (dm_dense_tn,
dm_dense_nn) through the C ABI, against FP64 products of the same FP32 values
on the host: relative error (Frobenius) <= 1e-5, at ragged sizes (row counts
off the 32-row chunks, column counts off the 128 x 48 / 64 tiles), on strided
column slices of wider blocks (the Krylov basis), both copy paths (16-byte
and element-wise) and the alpha / beta forms the iteration uses."""
import numpy as np
import pytest

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


def rel(got, want):
    got = np.asarray(got, dtype=np.float64)
    return np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300)


@pytest.mark.parametrize("n,m,k", [(1, 1, 1), (31, 3, 10), (1000, 40, 40), (100003, 130, 40),
                                   (70001, 280, 40), (40000, 320, 320), (5000, 41, 65)])
def test_dense_tn(dm, ctx, n, m, k):
    rng = np.random.default_rng(n + m + k)
    A = rng.normal(size=(n, m)).astype(np.float32)
    B = rng.normal(size=(n, k)).astype(np.float32)
    C = dm.dm_dense_tn(ctx, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), alpha=0.5)
    dm.dm_sync(ctx)
    assert rel(C.cpu().numpy(), 0.5 * A.astype(np.float64).T @ B.astype(np.float64)) <= 1e-5


@pytest.mark.parametrize("n,m,k", [(1, 1, 1), (127, 3, 10), (1000, 40, 40), (100003, 280, 40),
                                   (4097, 320, 32), (3000, 33, 64)])
def test_dense_nn(dm, ctx, n, m, k):
    rng = np.random.default_rng(7 * n + m + k)
    A = rng.normal(size=(n, m)).astype(np.float32)
    T = rng.normal(size=(m, k)).astype(np.float32)
    C0 = rng.normal(size=(n, k)).astype(np.float32)
    out = torch.from_numpy(C0.copy()).cuda()
    dm.dm_dense_nn(ctx, torch.from_numpy(A).cuda(), torch.from_numpy(T).cuda(), out=out, alpha=-1.0, beta=1.0)
    got = dm.dm_dense_nn(ctx, torch.from_numpy(A).cuda(), torch.from_numpy(T).cuda())
    dm.dm_sync(ctx)
    A64, T64 = A.astype(np.float64), T.astype(np.float64)
    assert rel(out.cpu().numpy(), C0.astype(np.float64) - A64 @ T64) <= 1e-5
    assert rel(got.cpu().numpy(), A64 @ T64) <= 1e-5


def test_dense_on_basis_slices(dm, ctx):
    # the iteration's operands: column slices of an n x 320 basis (leading
    # dimension 320), projections W - P (P^T W) in place
    rng = np.random.default_rng(3)
    n = 50021
    Q = rng.normal(size=(n, 320)).astype(np.float32)
    W = rng.normal(size=(n, 40)).astype(np.float32)
    Qd, Wd = torch.from_numpy(Q).cuda(), torch.from_numpy(W).cuda()
    P = Qd[:, :200]
    T = dm.dm_dense_tn(ctx, P, Wd)
    dm.dm_dense_nn(ctx, P, T, out=Wd, alpha=-1.0, beta=1.0)
    dm.dm_sync(ctx)
    P64, W64 = Q[:, :200].astype(np.float64), W.astype(np.float64)
    want = W64 - P64 @ (P64.T @ W64)
    assert rel(Wd.cpu().numpy(), want) <= 1e-5


def test_dense_rejects(dm, ctx):
    A = torch.zeros((10, 3), device="cuda")
    with pytest.raises(dm.DMError):
        dm.dm_dense_tn(ctx, A, torch.zeros((9, 2), device="cuda"))        # rows differ
    with pytest.raises(dm.DMError):
        dm.dm_dense_nn(ctx, A, torch.zeros((3, 65), device="cuda"))       # k > 64
    with pytest.raises(dm.DMError):
        dm.dm_dense_tn(ctx, A.double(), A.double())                         # FP32 only


@pytest.mark.parametrize("n", [1, 129, 100003])
@pytest.mark.parametrize("m", [1, 5, 17, 33, 280])
@pytest.mark.parametrize("k", [1, 3, 40, 64])
def test_dense_nn_ragged_strided_rows(dm, ctx, n, m, k):
    # A as the first m columns of a block whose width is a multiple of 4
    # (16-byte aligned rows at a leading dimension above m): chunks of A's
    # columns cut off at m, tiles of rows cut off at n
    rng = np.random.default_rng(n + 7 * m + 31 * k)
    width = m + (-m) % 4
    Aw = rng.normal(size=(n, width)).astype(np.float32)
    T = rng.normal(size=(m, k)).astype(np.float32)
    C0 = rng.normal(size=(n, k)).astype(np.float32)
    Ad = torch.from_numpy(Aw).cuda()[:, :m]
    out = torch.from_numpy(C0.copy()).cuda()
    dm.dm_dense_nn(ctx, Ad, torch.from_numpy(T).cuda(), out=out, alpha=-0.5, beta=2.0)
    dm.dm_sync(ctx)
    want = 2.0 * C0.astype(np.float64) - 0.5 * Aw[:, :m].astype(np.float64) @ T.astype(np.float64)
    assert rel(out.cpu().numpy(), want) <= 1e-5
