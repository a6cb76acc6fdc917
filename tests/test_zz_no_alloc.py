"""The squared-l2 product through dm_l2sq_matmat_noalloc, the entry point that
takes all of its scratch from a fixed device array instead of allocating.

Compared with the allocating path (dm_prepare with DM_L2SQ, then dm_matmat)
on the same device inputs, and with the CPU oracle's p = 2 identity
(Appendix A) on the whole block, on two calls in a row (the second reuses the
scratch the first left behind): relative error <= 1e-5 for FP32, <= 1e-12
for FP64, and identical int64 results for int32 inputs.  The file is named
to run last so that the entry point is also exercised after every other GPU
test of the session; it needs nothing from them and passes alone too.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2210_15114_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {np.float32: 1e-5, np.float64: 1e-12}
DM_OK, DM_ERR_INVALID_ARG, DM_ERR_UNSUPPORTED = 0, 1, 2


@pytest.fixture(scope="module")
def dm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_15114_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(got, want):
    got = got.astype(np.float64)
    want = want.astype(np.float64)
    return np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300)


def call_noalloc(dm, X, Z, out):
    """One call through the C ABI with torch's current stream."""
    lib = dm.load()
    stream = torch.cuda.current_stream().cuda_stream
    n, d = X.shape
    k = Z.shape[1]
    return lib.dm_l2sq_matmat_noalloc(
        dm.dtype_code(X.dtype), ctypes.c_void_p(X.data_ptr()), n, d, X.stride(0),
        ctypes.c_void_p(Z.data_ptr()), k, Z.stride(0),
        ctypes.c_void_p(out.data_ptr()), out.stride(0), ctypes.c_void_p(stream))


CASES = [
    # (label, points, queries)
    ("f32_mixture_n70001_d24_k16",
     lambda: inputs.gaussian_mixture(70001, 24, 16, dtype=np.float32),
     lambda: inputs.gaussian_queries(70001, 16, dtype=np.float32)),
    ("f64_uniform_n5003_d7_k3",
     lambda: inputs.uniform_points(5003, 7, dtype=np.float64),
     lambda: inputs.gaussian_queries(5003, 3, dtype=np.float64)),
    ("i32_max_sizes_n4099_d32_k32",
     lambda: inputs.integer_points(4099, 32),
     lambda: inputs.integer_queries(4099, 32)),
]


@pytest.mark.parametrize("label,make_x,make_z", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_allocating_path(dm, label, make_x, make_z):
    X, Z = make_x(), make_z()
    Xd, Zd = dev(X), dev(Z)
    ctx = dm.dm_create(0)
    plan = dm.dm_prepare(ctx, "l2sq", Xd)
    want = dm.dm_matmat(plan, Zd)
    dm.dm_sync(ctx)
    want = want.cpu().numpy()
    exact = oracle.l2sq_identity(X, Z)
    out_dtype = torch.int64 if X.dtype == np.int32 else Xd.dtype
    for call in range(2):
        out = torch.full((len(X), Z.shape[1]), -7, dtype=out_dtype, device="cuda")
        assert call_noalloc(dm, Xd, Zd, out) == DM_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        if X.dtype == np.int32:
            np.testing.assert_array_equal(got, want, err_msg=f"call {call}")
            np.testing.assert_array_equal(got, exact, err_msg=f"call {call} vs oracle")
        else:
            err = rel(got, want)
            assert err <= TOL[X.dtype.type], f"call {call}: relative error {err:.3e}"
            err = rel(got, exact)
            assert err <= TOL[X.dtype.type], f"call {call}: relative error {err:.3e} vs oracle"
    dm.dm_plan_destroy(plan)
    dm.dm_destroy(ctx)


def test_noalloc_python_wrapper(dm):
    X = inputs.gaussian_mixture(3001, 5, 4, dtype=np.float32)
    Z = inputs.gaussian_queries(3001, 2, dtype=np.float32)
    Xd, Zd = dev(X), dev(Z)
    ctx = dm.dm_create(0)
    plan = dm.dm_prepare(ctx, "l2sq", Xd)
    want = dm.dm_matmat(plan, Zd)
    dm.dm_sync(ctx)
    out = torch.empty_like(Zd)
    dm.dm_l2sq_matmat_noalloc(Xd, Zd, out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), want.cpu().numpy()) <= 1e-5
    dm.dm_plan_destroy(plan)
    dm.dm_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_the_static_scratch(dm):
    X = dev(inputs.gaussian_mixture(100, 33, 4, dtype=np.float32))
    Z = dev(inputs.gaussian_queries(100, 33, dtype=np.float32))
    out = torch.empty((100, 33), dtype=torch.float32, device="cuda")
    # d = 33 > 32
    assert call_noalloc(dm, X, Z[:, :4].contiguous(), out[:, :4].contiguous()) == DM_ERR_UNSUPPORTED
    # k = 33 > 32
    assert call_noalloc(dm, X[:, :8].contiguous(), Z, out) == DM_ERR_UNSUPPORTED
    # a bad size is an argument error, reported before anything is launched
    lib = dm.load()
    assert lib.dm_l2sq_matmat_noalloc(0, ctypes.c_void_p(X.data_ptr()), 0, 8, 8,
                                      ctypes.c_void_p(Z.data_ptr()), 4, 4,
                                      ctypes.c_void_p(out.data_ptr()), 4, None) == DM_ERR_INVALID_ARG
