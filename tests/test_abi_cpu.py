"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, and exports every entry point declared in include/dm.h; status
strings and argument checks work without touching a device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "dm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(dm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2210_15114_gb300 import build, binding
    build.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dm_create", "dm_destroy", "dm_prepare", "dm_plan_destroy", "dm_matvec_l1",
                     "dm_matvec_l2sq", "dm_matmat", "dm_sync", "dm_status_string",
                     "dm_bruteforce", "dm_matmat_host", "dm_matmat_host_async", "dm_matmat_host_multi", "dm_plan_export", "dm_grad",
                     "dm_batch_create", "dm_batch_run", "dm_batch_lanes", "dm_batch_destroy",
                     "dm_prepare_lpp", "dm_prepare_l2_embed", "dm_l2sq_matmat_noalloc",
                     "dm_set_deterministic", "dm_set_engine"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2210_15114_gb300 import binding
    out = subprocess.run(["nm", "-D", "--defined-only", binding.lib_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(dm_\w+)$", out, flags=re.M))
    for name in declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_build_flags_target_sm103a():
    from paper_2210_15114_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings(lib):
    from paper_2210_15114_gb300 import binding
    assert binding.dm_status_string(0) == "DM_OK"
    assert binding.dm_status_string(6) == "DM_ERR_TIMEOUT"
    assert binding.dm_status_string(99) == "DM_ERR_UNKNOWN"


def test_argument_checks_without_device(lib):
    P = ctypes.c_void_p
    h = P()
    assert lib.dm_create(None, 0, None) == 1                     # null out pointer
    assert lib.dm_prepare(None, 0, 0, None, 1, 1, 1, ctypes.byref(h)) == 1
    assert lib.dm_matmat(None, None, 1, 1, None, 1) == 1
    assert lib.dm_sync(None) == 1
    assert lib.dm_set_engine(None, 0) == 1
    assert lib.dm_matvec_l1(None, None, None) == 1
    assert lib.dm_bruteforce(None, 0, 0, None, 1, 1, 1, None, 1, 1, None, 1) == 1
    assert lib.dm_grad(None, None, 1, None, 1, 1, None, 1) == 1
    assert lib.dm_prepare_lpp(None, 0, None, 1, 1, 1, 4, ctypes.byref(h)) == 1
    assert lib.dm_prepare_l2_embed(None, 0, None, 1, 1, 1, None, 8, ctypes.byref(h)) == 1
    assert lib.dm_batch_create(None, 0, 0, 1, None, None, None, None, None, None, None, None, None,
                               0, ctypes.byref(h)) == 1
    assert lib.dm_batch_run(None) == 1
    assert lib.dm_batch_lanes(None) == 0
    lib.dm_batch_destroy(None)                                     # no-op
    # the no-alloc entry checks its arguments before touching the device
    dummy = P(16)
    assert lib.dm_l2sq_matmat_noalloc(0, None, 10, 2, 2, dummy, 1, 1, dummy, 1, None) == 1
    assert lib.dm_l2sq_matmat_noalloc(0, dummy, 0, 2, 2, dummy, 1, 1, dummy, 1, None) == 1
    assert lib.dm_l2sq_matmat_noalloc(0, dummy, 10, 33, 33, dummy, 1, 1, dummy, 1, None) == 2
    assert lib.dm_l2sq_matmat_noalloc(0, dummy, 10, 2, 2, dummy, 33, 33, dummy, 33, None) == 2
    # ||.||_p^p plans: p = 2..16 even, 3..15 odd; the power is checked before
    # the context is used (a dummy context pointer is never dereferenced)
    for pw in (-3, 0, 1, 17, 18, 19):
        assert lib.dm_prepare_lpp(dummy, 0, dummy, 10, 2, 2, pw, ctypes.byref(h)) == 1, pw
        assert not h.value


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.dm_create(ctypes.byref(h), 0, None) in (1, 5)
    assert not h.value


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2210_15114_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB", str(tmp_path / "absent.so"))
    with pytest.raises(binding.DMError):
        binding.load()


def test_leading_dimension_of_views():
    # row-major views: the column stride of a single-column view is ignored,
    # any other non-unit column stride is rejected
    import torch
    from paper_2210_15114_gb300 import binding
    a = np.arange(12, dtype=np.int32)[:, None]                 # strides (4, 0)
    assert binding._ld(a) == 1
    assert binding._ld(torch.from_numpy(a)) == 1
    assert binding._ld(torch.zeros(5, 7)[:, :3]) == 7           # a column slice keeps ld
    assert binding._ld(np.zeros((5, 7), dtype=np.float32)[1:, 2:]) == 7
    with pytest.raises(binding.DMError):
        binding._ld(torch.zeros(4, 6)[:, ::2])
    with pytest.raises(binding.DMError):
        binding._ld(np.zeros((4, 6))[:, ::2])
