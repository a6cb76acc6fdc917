"""Lifetime of contexts against their plans and batches, and the bounded
device-side wait (through the C ABI).

* A context destroyed while plans and a batch made from it are alive: later
  calls on them fail with DM_ERR_INVALID_ARG, and destroying them afterwards
  (in any order) releases everything; run in a child process that must exit
  0, since a use after free would show as a crash at teardown.
* A radix-pass CTA whose predecessor tile never publishes its digit counts
  (the decoupled look-back of Algorithm 1's sort) gives up after the
  context's wait limit, dm_sync reports DM_ERR_TIMEOUT, and the same context
  then computes a correct product.
* The tensor-core squared-l2 kernels (two roles meeting on mbarriers) with a
  wait limit of one round: every call either reports DM_ERR_TIMEOUT (a
  role's wait ran out, the CTA drained its own copies and MMAs and freed its
  tensor memory) or returns a correct product; the context then computes
  correct products at the default limit.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2210_15114_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_15114_gb300 import binding, build
    build.build()
    binding.load()
    return binding


CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import torch
from paper_2210_15114_gb300 import binding as dm
dm.load()
ctx = dm.dm_create(0)
X = torch.rand(5000, 4, device="cuda")
Z = torch.rand(5000, 3, device="cuda")
p1 = dm.dm_prepare(ctx, "l1", X)
p2 = dm.dm_prepare(ctx, "l2sq", X)
b = dm.dm_batch_create(ctx, "l1", [X, X[:3000]], [Z, Z[:3000]], lanes=2)
dm.dm_matmat(p1, Z)
dm.dm_batch_run(b)
dm.dm_sync(ctx)
dm.dm_destroy(ctx)                       # children still alive
for call in (lambda: dm.dm_matmat(p1, Z), lambda: dm.dm_grad(p2, Z, Z), lambda: dm.dm_batch_run(b)):
    try:
        call()
        raise SystemExit("a call on a destroyed context succeeded")
    except dm.DMError as e:
        assert e.status == dm.DM_ERR_INVALID_ARG, e
{order}
torch.cuda.synchronize()
print("lifetime ok")
"""

ORDERS = {
    "plans_then_batch": "dm.dm_plan_destroy(p1)\ndm.dm_plan_destroy(p2)\ndm.dm_batch_destroy(b)",
    "batch_then_plans": "dm.dm_batch_destroy(b)\ndm.dm_plan_destroy(p2)\ndm.dm_plan_destroy(p1)",
    "left_to_teardown": "pass",            # the finalizers at interpreter exit
}


@pytest.mark.parametrize("order", sorted(ORDERS))
def test_context_destroyed_before_its_children(dm, order):
    code = CHILD.format(root=ROOT, order=ORDERS[order])
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "lifetime ok" in r.stdout


def test_unpublished_predecessor_times_out(dm):
    ctx = dm.dm_create(0)
    dm.dm_set_wait_limit(ctx, 64)
    dm.dm_test_unpublished_wait(ctx)
    with pytest.raises(dm.DMError) as e:
        dm.dm_sync(ctx)
    assert e.value.status == dm.DM_ERR_TIMEOUT
    dm.dm_sync(ctx)                          # the error word was cleared
    dm.dm_set_wait_limit(ctx, 0)             # back to the default
    # the same context computes a correct product afterwards
    X, Z = inputs.workload_mixture_f32(n=20011, d=8, k=5)
    plan = dm.dm_prepare(ctx, "l1", torch.from_numpy(X).cuda())
    out = dm.dm_matmat(plan, torch.from_numpy(Z).cuda())
    dm.dm_sync(ctx)
    assert oracle.relative_error(out.cpu().numpy(), oracle.l1_sort(X, Z)) <= 1e-5


def test_wait_limit_argument_checks(dm):
    lib = dm.load()
    assert lib.dm_set_wait_limit(None, 5) == dm.DM_ERR_INVALID_ARG
    assert lib.dm_test_unpublished_wait(None) == dm.DM_ERR_INVALID_ARG


def test_tensor_core_kernels_give_up_cleanly(dm):
    ctx = dm.dm_create(0)
    X, Z = inputs.workload_mixture_f32(n=300007, d=32, k=16)
    Xd, Zd = torch.from_numpy(X).cuda(), torch.from_numpy(Z).cuda()
    want = oracle.l2sq_identity(X, Z)
    plan = dm.dm_prepare(ctx, "l2sq", Xd)
    dm.dm_sync(ctx)
    dm.dm_set_wait_limit(ctx, 1)
    outcomes = []
    for _ in range(5):
        out = dm.dm_matmat(plan, Zd)
        try:
            dm.dm_sync(ctx)
            outcomes.append("ok")
            assert oracle.relative_error(out.cpu().numpy(), want) <= 1e-5
        except dm.DMError as e:
            assert e.status == dm.DM_ERR_TIMEOUT
            outcomes.append("timeout")
    dm.dm_set_wait_limit(ctx, 0)
    for _ in range(2):
        out = dm.dm_matmat(plan, Zd)
        dm.dm_sync(ctx)
        assert oracle.relative_error(out.cpu().numpy(), want) <= 1e-5
    print("outcomes at a one-round wait limit:", outcomes)
