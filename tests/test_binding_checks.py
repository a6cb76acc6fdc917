"""Argument checks of the Python binding that raise before any library call:
shapes, element types and devices of query blocks and results (a mismatch
would otherwise read or write outside the caller's buffers on the device).
CPU only: the checks run on plan metadata and CPU tensors."""
import types

import numpy as np

import pytest

torch = pytest.importorskip("torch")

from paper_2210_15114_gb300 import binding  # noqa: E402


def fake_plan(n=10, d=3, dtype=binding.DM_F32):
    ctx = types.SimpleNamespace(device=0, handle=None)
    return types.SimpleNamespace(n=n, d=d, dtype=dtype, ctx=ctx, handle=None)


@pytest.mark.parametrize("Z,out", [
    (torch.zeros(9, 2), None),                                  # rows differ from n
    (torch.zeros(10, 2, dtype=torch.float64), None),            # element type of Z
    (torch.zeros(10, 2), torch.zeros(10, 3)),                   # out shape
    (torch.zeros(10, 2), torch.zeros(10, 2, dtype=torch.float64)),   # out type
    (torch.zeros(10), torch.zeros(10, 1)),                      # 1-D Z, 2-D out
    (torch.zeros(10, 2), torch.zeros(10, 2)),                   # not on the device
])
def test_matmat_rejects_mismatches(Z, out):
    with pytest.raises(binding.DMError) as e:
        binding._query_args(fake_plan(), Z, out)
    assert e.value.status == binding.DM_ERR_INVALID_ARG


def test_int32_plans_take_int64_results():
    plan = fake_plan(dtype=binding.DM_I32)
    with pytest.raises(binding.DMError):
        binding._query_args(plan, torch.zeros(10, 2, dtype=torch.int32), torch.zeros(10, 2, dtype=torch.int32))


def test_strided_vector_becomes_a_column_with_its_stride():
    Zfull = torch.zeros(10, 4)
    z = Zfull[:, 1]
    z2 = binding._as2d(z)
    assert z2.shape == (10, 1) and binding._ld(z2) == 4 and z2.data_ptr() == z.data_ptr()


def test_noalloc_wrapper_checks_before_the_call():
    X = torch.zeros(10, 3)
    with pytest.raises(binding.DMError):
        binding.dm_l2sq_matmat_noalloc(X, torch.zeros(10, 2, dtype=torch.float64), torch.zeros(10, 2))
    with pytest.raises(binding.DMError):
        binding.dm_l2sq_matmat_noalloc(X, torch.zeros(9, 2), torch.zeros(10, 2))
    with pytest.raises(binding.DMError):
        binding.dm_l2sq_matmat_noalloc(X, torch.zeros(10, 2), torch.zeros(10, 3))
    with pytest.raises(binding.DMError):
        binding.dm_l2sq_matmat_noalloc(torch.zeros(10, 3, dtype=torch.int32),
                                       torch.zeros(10, 2, dtype=torch.int32),
                                       torch.zeros(10, 2, dtype=torch.int32))
    with pytest.raises(binding.DMError):     # CPU tensors
        binding.dm_l2sq_matmat_noalloc(X, torch.zeros(10, 2), torch.zeros(10, 2))


@pytest.mark.parametrize("X,Z,out", [
    (np.zeros((10, 3), np.float32), np.zeros((9, 2), np.float32), None),          # rows differ
    (np.zeros((10, 3), np.float32), np.zeros((10, 2), np.float64), None),         # element types differ
    (np.zeros((10, 3), np.float32), np.zeros((10, 2), np.float32), np.zeros((10, 3), np.float32)),
    (np.zeros((10, 3), np.float32), np.zeros((10, 2), np.float32), np.zeros((10, 2), np.float64)),
    (np.zeros((10, 3), np.int32), np.zeros((10, 2), np.int32), np.zeros((10, 2), np.int32)),   # int64 results
    (torch.zeros(10, 3), torch.zeros(10, 2), None),                                # not numpy
])
def test_host_calls_check_before_the_call(X, Z, out):
    ctx = types.SimpleNamespace(device=0, handle=None)
    for fn in (binding.dm_matmat_host, binding.dm_matmat_host_async):
        with pytest.raises(binding.DMError) as e:
            fn(ctx, "l1", X, Z, out)
        assert e.value.status == binding.DM_ERR_INVALID_ARG
    with pytest.raises(binding.DMError):
        binding.dm_matmat_host_multi(ctx, ["l1", "l2sq"], X, Z, None if out is None else [out, out])
