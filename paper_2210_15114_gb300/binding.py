"""ctypes binding of libdm's C ABI (include/dm.h).

Each function here has the name of the C entry point it calls and does only
argument marshalling: torch CUDA tensors become device pointers, numpy arrays
become host pointers, the current torch stream becomes the context's stream.
All computation happens in the CUDA kernels of libdm.  A missing or unloadable
library raises ``DMError`` at once: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .build import LIB, up_to_date

DM_OK = 0
DM_ERR_INVALID_ARG = 1
DM_ERR_UNSUPPORTED = 2
DM_ERR_NONFINITE = 3
DM_ERR_OOM = 4
DM_ERR_CUDA = 5
DM_ERR_TIMEOUT = 6
DM_ERR_INTERNAL = 7

DM_F32, DM_F64, DM_I32 = 0, 1, 2
DM_L1, DM_L2SQ = 0, 1

METRICS = {"l1": DM_L1, "l2sq": DM_L2SQ, "tv": 2}
DM_LPP, DM_L2_EMBED = 3, 4

_lock = threading.Lock()
_lib = None


class DMError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        name = dm_status_string(status) if _lib is not None else str(status)
        super().__init__(f"{where}: {name}")


def lib_path() -> str:
    return LIB


def load() -> ctypes.CDLL:
    """Load libdm.so (built in-tree by build.build()).  Raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB):
            raise DMError(-1, f"libdm not built ({LIB} missing); run "
                              "paper_2210_15114_gb300.build.build()")
        if not up_to_date():
            raise DMError(-1, "libdm.so is older than its sources; rebuild it")
        lib = ctypes.CDLL(LIB)
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        sigs = {
            "dm_create": ([ctypes.POINTER(P), I32, P], I32),
            "dm_destroy": ([P], None),
            "dm_set_stream": ([P, P], I32),
            "dm_set_deterministic": ([P, I32], I32),
            "dm_set_engine": ([P, I32], I32),
            "dm_prepare": ([P, I32, I32, P, I64, I64, I64, ctypes.POINTER(P)], I32),
            "dm_plan_destroy": ([P], None),
            "dm_matvec_l1": ([P, P, P], I32),
            "dm_matvec_l2sq": ([P, P, P], I32),
            "dm_matmat": ([P, P, I64, I64, P, I64], I32),
            "dm_grad": ([P, P, I64, P, I64, I64, P, I64], I32),
            "dm_prepare_lpp": ([P, I32, P, I64, I64, I64, I32, P], I32),
            "dm_prepare_l2_embed": ([P, I32, P, I64, I64, I64, P, I64, P], I32),
            "dm_batch_create": ([P, I32, I32, I64, P, P, P, P, P, P, P, P, P, I32, P], I32),
            "dm_batch_run": ([P], I32),
            "dm_batch_lanes": ([P], I32),
            "dm_batch_destroy": ([P], None),
            "dm_sync": ([P], I32),
            "dm_status_string": ([I32], ctypes.c_char_p),
            "dm_plan_export": ([P, P, P], I32),
            "dm_bruteforce": ([P, I32, I32, P, I64, I64, I64, P, I64, I64, P, I64], I32),
            "dm_matmat_host": ([P, I32, I32, P, I64, I64, I64, P, I64, I64, P, I64], I32),
            "dm_matmat_host_async": ([P, I32, I32, P, I64, I64, I64, P, I64, I64, P, I64], I32),
            "dm_matmat_host_multi": ([P, I32, P, I32, P, I64, I64, I64, P, I64, I64, P, I64], I32),
            "dm_launch_count": ([P], I64),
            "dm_profile_enable": ([P, I32], I32),
            "dm_profile_read": ([P, I32, ctypes.POINTER(ctypes.c_int), P, P, P], I32),
            "dm_l2sq_matmat_noalloc": ([I32, P, I64, I64, I64, P, I64, I64, P, I64, P], I32),
            "dm_set_wait_limit": ([P, ctypes.c_uint32], I32),
            "dm_dense_tn": ([P, P, I64, I64, I64, P, I64, I64, P, I64, ctypes.c_float], I32),
            "dm_dense_nn": ([P, P, I64, I64, I64, P, I64, I64, P, I64, ctypes.c_float, ctypes.c_float], I32),
            "dm_test_unpublished_wait": ([P], I32),
        }
        for name, (args, res) in sigs.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != DM_OK:
        raise DMError(status, where)


# ----------------------------------------------------------- dtype helpers
def dtype_code(t) -> int:
    """Map a torch or numpy dtype of the points to dm_dtype."""
    import torch
    table = {torch.float32: DM_F32, torch.float64: DM_F64, torch.int32: DM_I32,
             np.dtype(np.float32): DM_F32, np.dtype(np.float64): DM_F64,
             np.dtype(np.int32): DM_I32}
    key = t if isinstance(t, torch.dtype) else np.dtype(t)
    if key not in table:
        raise DMError(DM_ERR_UNSUPPORTED, f"element type {t}")
    return table[key]


def out_torch_dtype(code: int):
    import torch
    return {DM_F32: torch.float32, DM_F64: torch.float64, DM_I32: torch.int64}[code]


def out_numpy_dtype(code: int):
    return {DM_F32: np.float32, DM_F64: np.float64, DM_I32: np.int64}[code]


def _ld(t) -> int:
    """Leading dimension (elements) of a row-major 2-D tensor/array view.  The
    column stride of a single-column view (x[:, None]) is irrelevant."""
    if t.ndim == 1:
        return 1
    if hasattr(t, "stride") and callable(t.stride):
        st = t.stride()
        if st[1] != 1 and t.shape[1] != 1:
            raise DMError(DM_ERR_INVALID_ARG, "matrix rows must be contiguous")
        return st[0]
    st = t.strides
    if st[1] != t.itemsize and t.shape[1] != 1:
        raise DMError(DM_ERR_INVALID_ARG, "matrix rows must be contiguous")
    return st[0] // t.itemsize


def _dev_ptr(t) -> int:
    if not t.is_cuda:
        raise DMError(DM_ERR_INVALID_ARG, "expected a CUDA tensor")
    return t.data_ptr()


# ----------------------------------------------------------- entry points
class Context:
    """Owner of a dm_ctx handle (device, stream, scratch arena)."""

    def __init__(self, handle: int, device: int, stream: int = 0):
        self.handle = handle
        self.device = device
        self.stream = stream          # the stream work is issued on (cudaStream_t)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.dm_destroy(self.handle)
            self.handle = None


class Plan:
    """Owner of a dm_plan handle."""

    def __init__(self, handle: int, ctx: Context, metric: int, dtype: int, n: int, d: int):
        self.handle = handle
        self.ctx = ctx
        self.metric = metric
        self.dtype = dtype
        self.n = n
        self.d = d

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.dm_plan_destroy(self.handle)
            self.handle = None


def dm_create(device: int = 0, stream=None) -> Context:
    """dm_create on `device`; the stream defaults to torch's current stream."""
    import torch
    lib = load()
    if stream is None:
        stream = torch.cuda.current_stream(device).cuda_stream
    h = ctypes.c_void_p()
    _check(lib.dm_create(ctypes.byref(h), int(device), ctypes.c_void_p(stream)), "dm_create")
    return Context(h.value, int(device), stream)


def dm_destroy(ctx: Context) -> None:
    if ctx.handle:
        load().dm_destroy(ctx.handle)
        ctx.handle = None


def dm_set_stream(ctx: Context, stream) -> None:
    _check(load().dm_set_stream(ctx.handle, ctypes.c_void_p(stream)), "dm_set_stream")
    ctx.stream = stream


def dm_set_deterministic(ctx: Context, on: bool = True) -> None:
    _check(load().dm_set_deterministic(ctx.handle, 1 if on else 0), "dm_set_deterministic")


ENGINES = {"auto": 0, "cuda": 1, "tensor": 2}


def dm_set_engine(ctx: Context, engine: str = "auto") -> None:
    """dm_set_engine: units of the squared-l2 contraction ("auto", "cuda" for
    the CUDA cores, "tensor" for the tensor cores where the shape allows)."""
    if engine not in ENGINES:
        raise DMError(DM_ERR_INVALID_ARG, f"engine must be one of {sorted(ENGINES)}")
    _check(load().dm_set_engine(ctx.handle, ENGINES[engine]), "dm_set_engine")


def dm_prepare(ctx: Context, metric, X) -> Plan:
    """dm_prepare on a CUDA tensor X (n x d, rows contiguous)."""
    lib = load()
    m = METRICS[metric] if isinstance(metric, str) else int(metric)
    if X.ndim == 1:
        X = X.reshape(-1, 1)
    code = dtype_code(X.dtype)
    n, d = X.shape
    h = ctypes.c_void_p()
    _check(lib.dm_prepare(ctx.handle, m, code, ctypes.c_void_p(_dev_ptr(X)), n, d, _ld(X),
                          ctypes.byref(h)), "dm_prepare")
    plan = Plan(h.value, ctx, m, code, n, d)
    plan.X = X if m == DM_L2SQ else None   # the squared-l2 plan borrows X
    return plan


def dm_prepare_lpp(ctx: Context, X, p: int) -> Plan:
    """dm_prepare_lpp: ||x - y||_p^p plan on a CUDA tensor X (n x d): even p
    2..16 through moments of the centred coordinates, odd p 3..15 through
    the sorted coordinates."""
    if X.ndim == 1:
        X = X.reshape(-1, 1)
    code = dtype_code(X.dtype)
    n, d = X.shape
    h = ctypes.c_void_p()
    _check(load().dm_prepare_lpp(ctx.handle, code, ctypes.c_void_p(_dev_ptr(X)), n, d, _ld(X), int(p),
                                 ctypes.byref(h)), "dm_prepare_lpp")
    plan = Plan(h.value, ctx, DM_LPP, code, n, d)
    plan.X = X
    return plan


def dm_prepare_l2_embed(ctx: Context, X, G) -> Plan:
    """dm_prepare_l2_embed: approximate l2 plan through the map
    T(x) = G x / (beta m), G an m x d CUDA tensor of N(0, 1) entries."""
    if X.ndim == 1:
        X = X.reshape(-1, 1)
    code = dtype_code(X.dtype)
    if dtype_code(G.dtype) != code or G.ndim != 2 or G.shape[1] != X.shape[1]:
        raise DMError(DM_ERR_INVALID_ARG, "G must be m x d with the points' element type")
    G = G.contiguous()
    n, d = X.shape
    m = G.shape[0]
    h = ctypes.c_void_p()
    _check(load().dm_prepare_l2_embed(ctx.handle, code, ctypes.c_void_p(_dev_ptr(X)), n, d, _ld(X),
                                      ctypes.c_void_p(_dev_ptr(G)), m, ctypes.byref(h)),
           "dm_prepare_l2_embed")
    return Plan(h.value, ctx, DM_L2_EMBED, code, n, m)


def dm_plan_destroy(plan: Plan) -> None:
    if plan.handle:
        load().dm_plan_destroy(plan.handle)
        plan.handle = None


def _as2d(t):
    """A 1-D tensor as its n x 1 view (the stride of the elements becomes the
    leading dimension); 2-D tensors unchanged."""
    if t.ndim == 1:
        return t.reshape(-1, 1)
    if t.ndim != 2:
        raise DMError(DM_ERR_INVALID_ARG, "expected a vector or a matrix")
    return t


def _on_device(device: int, *ts):
    for t in ts:
        if not t.is_cuda or t.device.index != device:
            raise DMError(DM_ERR_INVALID_ARG, f"tensors must be on cuda:{device}")


def _query_args(plan: Plan, Z, out):
    """Checks of a query block Z (n or n x k, the plan's element type, on the
    plan's device) and of its result `out` (allocated when None: the shape of
    Z, the plan's result type).  Returns (out, Z as n x k, out as n x k)."""
    import torch
    if dtype_code(Z.dtype) != plan.dtype:
        raise DMError(DM_ERR_INVALID_ARG, "Z element type differs from the plan's")
    Z2 = _as2d(Z)
    if Z2.shape[0] != plan.n:
        raise DMError(DM_ERR_INVALID_ARG, f"Z has {Z2.shape[0]} rows, the plan {plan.n} points")
    shape = (plan.n,) if Z.ndim == 1 else (plan.n, Z2.shape[1])
    if out is None:
        out = torch.empty(shape, dtype=out_torch_dtype(plan.dtype), device=Z.device)
    elif tuple(out.shape) != shape or out.dtype != out_torch_dtype(plan.dtype):
        raise DMError(DM_ERR_INVALID_ARG, f"out must be {shape} of {out_torch_dtype(plan.dtype)}")
    _on_device(plan.ctx.device, Z, out)
    return out, Z2, _as2d(out)


def _matvec(name: str, plan: Plan, z, out):
    if z.ndim != 1:
        raise DMError(DM_ERR_INVALID_ARG, f"{name} takes one query vector of n elements")
    out, _, _ = _query_args(plan, z, out)
    if not out.is_contiguous():
        raise DMError(DM_ERR_INVALID_ARG, f"{name} writes a contiguous result vector")
    z = z.contiguous()                # the entry point reads n consecutive elements
    _check(getattr(load(), name)(plan.handle, ctypes.c_void_p(_dev_ptr(z)),
                                 ctypes.c_void_p(_dev_ptr(out))), name)
    return out


def dm_matvec_l1(plan: Plan, z, out=None):
    return _matvec("dm_matvec_l1", plan, z, out)


def dm_matvec_l2sq(plan: Plan, z, out=None):
    return _matvec("dm_matvec_l2sq", plan, z, out)


def dm_matmat(plan: Plan, Z, out=None):
    out, Z2, o2 = _query_args(plan, Z, out)
    _check(load().dm_matmat(plan.handle, ctypes.c_void_p(_dev_ptr(Z2)), Z2.shape[1], _ld(Z2),
                            ctypes.c_void_p(_dev_ptr(o2)), _ld(o2)), "dm_matmat")
    return out


def dm_grad(plan: Plan, W, Z, out=None):
    """dm_grad: G = d(sum_q w_q^T A(X) z_q)/dX, n x d (W and Z: n or n x k)."""
    import torch
    if dtype_code(W.dtype) != plan.dtype or dtype_code(Z.dtype) != plan.dtype:
        raise DMError(DM_ERR_INVALID_ARG, "W / Z element type differs from the plan's")
    W2, Z2 = _as2d(W), _as2d(Z)
    if W2.shape != Z2.shape:
        raise DMError(DM_ERR_INVALID_ARG, "W and Z must have the same shape")
    if W2.shape[0] != plan.n:
        raise DMError(DM_ERR_INVALID_ARG, f"W and Z have {W2.shape[0]} rows, the plan {plan.n} points")
    if out is None:
        out = torch.empty((plan.n, plan.d), dtype=out_torch_dtype(plan.dtype), device=W.device)
    elif tuple(out.shape) != (plan.n, plan.d) or out.dtype != out_torch_dtype(plan.dtype):
        raise DMError(DM_ERR_INVALID_ARG, f"out must be ({plan.n}, {plan.d}) of {out_torch_dtype(plan.dtype)}")
    _on_device(plan.ctx.device, W2, Z2, out)
    _check(load().dm_grad(plan.handle, ctypes.c_void_p(_dev_ptr(W2)), _ld(W2),
                          ctypes.c_void_p(_dev_ptr(Z2)), _ld(Z2), W2.shape[1],
                          ctypes.c_void_p(_dev_ptr(out)), _ld(out)), "dm_grad")
    return out


class Batch:
    """Owner of a dm_batch handle; keeps the set tensors alive (the graph
    reads them by address)."""

    def __init__(self, handle, ctx, Xs, Zs, outs):
        self.handle = handle
        self.ctx = ctx
        self.Xs, self.Zs, self.outs = Xs, Zs, outs

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.dm_batch_destroy(self.handle)
            self.handle = None


def dm_batch_create(ctx: Context, metric, Xs, Zs, outs=None, lanes: int = 0) -> Batch:
    """dm_batch_create over lists of device tensors (X_s: n_s x d_s, Z_s:
    n_s x k_s or n_s); outputs are allocated when `outs` is None."""
    import torch
    ns = len(Xs)
    if ns != len(Zs) or ns < 1:
        raise DMError(DM_ERR_INVALID_ARG, "Xs and Zs must be non-empty lists of equal length")
    code = dtype_code(Xs[0].dtype)
    X2 = [x.reshape(-1, 1) if x.ndim == 1 else x for x in Xs]
    Z2 = [z.reshape(-1, 1) if z.ndim == 1 else z for z in Zs]
    for x, z in zip(X2, Z2):
        if dtype_code(x.dtype) != code or dtype_code(z.dtype) != code:
            raise DMError(DM_ERR_INVALID_ARG, "all sets must share one element type")
    if outs is None:
        outs = [torch.empty((x.shape[0], z.shape[1]), dtype=out_torch_dtype(code), device=x.device)
                for x, z in zip(X2, Z2)]
    O2 = [o.reshape(-1, 1) if o.ndim == 1 else o for o in outs]
    I64a = ctypes.c_int64 * ns
    Pa = ctypes.c_void_p * ns
    n = I64a(*[x.shape[0] for x in X2])
    d = I64a(*[x.shape[1] for x in X2])
    k = I64a(*[z.shape[1] for z in Z2])
    ldx = I64a(*[_ld(x) for x in X2])
    ldz = I64a(*[_ld(z) for z in Z2])
    ldo = I64a(*[_ld(o) for o in O2])
    xp = Pa(*[_dev_ptr(x) for x in X2])
    zp = Pa(*[_dev_ptr(z) for z in Z2])
    op = Pa(*[_dev_ptr(o) for o in O2])
    h = ctypes.c_void_p()
    _check(load().dm_batch_create(ctx.handle, METRICS[metric] if isinstance(metric, str) else int(metric), code, ns, n, d, xp, ldx, k, zp, ldz,
                                  op, ldo, int(lanes), ctypes.byref(h)), "dm_batch_create")
    return Batch(h.value, ctx, Xs, Zs, outs)


def dm_batch_run(batch: Batch):
    _check(load().dm_batch_run(batch.handle), "dm_batch_run")
    return batch.outs


def dm_batch_lanes(batch: Batch) -> int:
    return int(load().dm_batch_lanes(batch.handle))


def dm_batch_destroy(batch: Batch) -> None:
    if batch.handle:
        load().dm_batch_destroy(batch.handle)
        batch.handle = None


def dm_sync(ctx: Context) -> None:
    _check(load().dm_sync(ctx.handle), "dm_sync")


def _dense_operand(t, device: int, what: str):
    import torch
    if t.dtype != torch.float32 or t.ndim != 2:
        raise DMError(DM_ERR_INVALID_ARG, f"{what} must be a 2-D FP32 tensor")
    _on_device(device, t)
    return t, _ld(t)


def dm_dense_tn(ctx: Context, A, B, alpha: float = 1.0, out=None):
    """dm_dense_tn: alpha A^T B for FP32 blocks A (n x m) and B (n x k)."""
    import torch
    A, lda = _dense_operand(A, ctx.device, "A")
    B, ldb = _dense_operand(B, ctx.device, "B")
    n, m = A.shape
    if B.shape[0] != n:
        raise DMError(DM_ERR_INVALID_ARG, "A and B must have the same number of rows")
    k = B.shape[1]
    if out is None:
        out = torch.empty((m, k), dtype=torch.float32, device=A.device)
    out, ldc = _dense_operand(out, ctx.device, "out")
    if tuple(out.shape) != (m, k):
        raise DMError(DM_ERR_INVALID_ARG, f"out must be ({m}, {k})")
    _check(load().dm_dense_tn(ctx.handle, ctypes.c_void_p(A.data_ptr()), n, m, lda,
                              ctypes.c_void_p(B.data_ptr()), k, ldb, ctypes.c_void_p(out.data_ptr()), ldc,
                              float(alpha)), "dm_dense_tn")
    return out


def dm_dense_nn(ctx: Context, A, T, out=None, alpha: float = 1.0, beta: float = 0.0):
    """dm_dense_nn: beta out + alpha A T for FP32 blocks A (n x m), T (m x k);
    out is allocated (and beta ignored) when None."""
    import torch
    A, lda = _dense_operand(A, ctx.device, "A")
    T, ldt = _dense_operand(T, ctx.device, "T")
    n, m = A.shape
    if T.shape[0] != m:
        raise DMError(DM_ERR_INVALID_ARG, "T must have as many rows as A has columns")
    k = T.shape[1]
    if out is None:
        out = torch.empty((n, k), dtype=torch.float32, device=A.device)
        beta = 0.0
    out, ldc = _dense_operand(out, ctx.device, "out")
    if tuple(out.shape) != (n, k):
        raise DMError(DM_ERR_INVALID_ARG, f"out must be ({n}, {k})")
    _check(load().dm_dense_nn(ctx.handle, ctypes.c_void_p(A.data_ptr()), n, m, lda,
                              ctypes.c_void_p(T.data_ptr()), k, ldt, ctypes.c_void_p(out.data_ptr()), ldc,
                              float(alpha), float(beta)), "dm_dense_nn")
    return out


def dm_set_wait_limit(ctx: Context, rounds: int = 0) -> None:
    """dm_set_wait_limit: rounds a device-side wait may spin (0: default)."""
    _check(load().dm_set_wait_limit(ctx.handle, int(rounds)), "dm_set_wait_limit")


def dm_test_unpublished_wait(ctx: Context) -> None:
    """dm_test_unpublished_wait: one radix-pass CTA whose predecessor never
    publishes (a test of the bounded wait; dm_sync then reports it)."""
    _check(load().dm_test_unpublished_wait(ctx.handle), "dm_test_unpublished_wait")


def dm_status_string(status: int) -> str:
    return load().dm_status_string(int(status)).decode()


def dm_plan_export(plan: Plan):
    """Sorted coordinates (d x n) and permutation (d x n int32) of an l1 plan."""
    import torch
    tdt = {DM_F32: torch.float32, DM_F64: torch.float64, DM_I32: torch.int32}[plan.dtype]
    dev = torch.device("cuda", plan.ctx.device)
    vals = torch.empty((plan.d, plan.n), dtype=tdt, device=dev)
    perm = torch.empty((plan.d, plan.n), dtype=torch.int32, device=dev)
    _check(load().dm_plan_export(plan.handle, ctypes.c_void_p(vals.data_ptr()),
                                 ctypes.c_void_p(perm.data_ptr())), "dm_plan_export")
    return vals, perm


def dm_bruteforce(ctx: Context, metric, X, Z, out=None):
    import torch
    m = METRICS[metric] if isinstance(metric, str) else int(metric)
    X = _as2d(X)
    code = dtype_code(X.dtype)
    squeeze = Z.ndim == 1
    Z2 = _as2d(Z)
    n, d = X.shape
    k = Z2.shape[1]
    if dtype_code(Z2.dtype) != code or Z2.shape[0] != n:
        raise DMError(DM_ERR_INVALID_ARG, "Z must have n rows of the points' element type")
    if out is None:
        out = torch.empty((n, k), dtype=out_torch_dtype(code), device=X.device)
    o2 = _as2d(out)
    if tuple(o2.shape) != (n, k) or out.dtype != out_torch_dtype(code):
        raise DMError(DM_ERR_INVALID_ARG, f"out must be ({n}, {k}) of {out_torch_dtype(code)}")
    _on_device(X.device.index if X.is_cuda else -1, X, Z2, o2)
    _check(load().dm_bruteforce(ctx.handle, m, code, ctypes.c_void_p(_dev_ptr(X)), n, d, _ld(X),
                                ctypes.c_void_p(_dev_ptr(Z2)), k, _ld(Z2),
                                ctypes.c_void_p(_dev_ptr(o2)), _ld(o2)), "dm_bruteforce")
    return out.reshape(-1) if squeeze else out


def _host_args(X, Z):
    """Host (numpy) points and queries as 2-D arrays, checked against each
    other: the library copies n x d and n x k elements from them."""
    if not isinstance(X, np.ndarray) or not isinstance(Z, np.ndarray):
        raise DMError(DM_ERR_INVALID_ARG, "host calls take numpy arrays")
    if X.ndim == 1:
        X = X.reshape(-1, 1)
    squeeze = Z.ndim == 1
    Z2 = Z.reshape(-1, 1) if squeeze else Z
    if X.ndim != 2 or Z2.ndim != 2:
        raise DMError(DM_ERR_INVALID_ARG, "X and Z must be 1-D or 2-D")
    code = dtype_code(X.dtype)
    if Z2.dtype != X.dtype or Z2.shape[0] != X.shape[0]:
        raise DMError(DM_ERR_INVALID_ARG, "Z must have n rows of the points' element type")
    return X, Z2, squeeze, code


def _host_out(out, n, k, code):
    """A host result buffer of the right type and shape: (n, k), or (n,) when
    k == 1 (the library writes n rows of k elements at its leading dimension)."""
    want = out_numpy_dtype(code)
    if out is None:
        return np.empty((n, k), dtype=want)
    if not isinstance(out, np.ndarray) or out.dtype != want:
        raise DMError(DM_ERR_INVALID_ARG, f"out must be a numpy array of {np.dtype(want).name}")
    if out.shape == (n,) and k == 1:
        return out.reshape(n, 1)
    if out.shape != (n, k):
        raise DMError(DM_ERR_INVALID_ARG, f"out must have shape ({n}, {k})")
    return out


def _host_call(fn_name, ctx: Context, metric, X: np.ndarray, Z: np.ndarray, out):
    m = METRICS[metric] if isinstance(metric, str) else int(metric)
    X, Z2, squeeze, code = _host_args(X, Z)
    n, d = X.shape
    k = Z2.shape[1]
    out = _host_out(out, n, k, code)
    _check(getattr(load(), fn_name)(ctx.handle, m, code, ctypes.c_void_p(X.ctypes.data), n, d, _ld(X),
                                    ctypes.c_void_p(Z2.ctypes.data), k, _ld(Z2),
                                    ctypes.c_void_p(out.ctypes.data), _ld(out)), fn_name)
    return out.reshape(-1) if squeeze else out


def dm_matmat_host(ctx: Context, metric, X: np.ndarray, Z: np.ndarray, out: np.ndarray = None):
    """End to end with host (numpy) buffers; returns the numpy result."""
    return _host_call("dm_matmat_host", ctx, metric, X, Z, out)


def dm_matmat_host_async(ctx: Context, metric, X: np.ndarray, Z: np.ndarray, out: np.ndarray = None):
    """dm_matmat_host without the final wait: returns the numpy array the
    result lands in after the next dm_sync(ctx).  X, Z and the returned array
    must stay alive (and X, Z unchanged) until then."""
    return _host_call("dm_matmat_host_async", ctx, metric, X, Z, out)


def dm_matmat_host_multi(ctx: Context, metrics, X: np.ndarray, Z: np.ndarray, outs=None):
    """Products of several metrics for the same host (numpy) X and Z, X and Z
    copied to the device once; returns the list of numpy results."""
    codes = [METRICS[m] if isinstance(m, str) else int(m) for m in metrics]
    X, Z2, squeeze, code = _host_args(X, Z)
    n, d = X.shape
    k = Z2.shape[1]
    if outs is None:
        outs = [np.empty((n, k), dtype=out_numpy_dtype(code)) for _ in codes]
    if len(outs) != len(codes):
        raise DMError(DM_ERR_INVALID_ARG, "one output per metric")
    if any(not isinstance(o, np.ndarray) or o.dtype != out_numpy_dtype(code) or o.size != n * k
           or not o.flags.c_contiguous for o in outs):
        raise DMError(DM_ERR_INVALID_ARG, "outputs must be contiguous n x k arrays of the output type")
    marr = (ctypes.c_int32 * max(len(codes), 1))(*codes)
    oarr = (ctypes.c_void_p * max(len(outs), 1))(*[o.ctypes.data for o in outs])
    _check(load().dm_matmat_host_multi(ctx.handle, len(codes), ctypes.cast(marr, ctypes.c_void_p), code,
                                       ctypes.c_void_p(X.ctypes.data), n, d, _ld(X),
                                       ctypes.c_void_p(Z2.ctypes.data), k, _ld(Z2),
                                       ctypes.cast(oarr, ctypes.c_void_p), k), "dm_matmat_host_multi")
    return [o.reshape(-1) if squeeze else o for o in outs]


def dm_launch_count(ctx: Context) -> int:
    return int(load().dm_launch_count(ctx.handle))


def dm_profile_enable(ctx: Context, enable: bool = True) -> None:
    _check(load().dm_profile_enable(ctx.handle, 1 if enable else 0), "dm_profile_enable")


def dm_profile_read(ctx: Context, max_groups: int = 32) -> dict:
    """{group name: (launches, total device ms)} collected since enabling."""
    names = ctypes.create_string_buffer(32 * max_groups)
    launches = (ctypes.c_int64 * max_groups)()
    total = (ctypes.c_double * max_groups)()
    count = ctypes.c_int()
    _check(load().dm_profile_read(ctx.handle, max_groups, ctypes.byref(count),
                                  ctypes.cast(names, ctypes.c_void_p),
                                  ctypes.cast(launches, ctypes.c_void_p),
                                  ctypes.cast(total, ctypes.c_void_p)), "dm_profile_read")
    out = {}
    for i in range(count.value):
        name = names.raw[32 * i:32 * (i + 1)].split(b"\0", 1)[0].decode()
        out[name] = (int(launches[i]), float(total[i]))
    return out


def dm_l2sq_matmat_noalloc(X, Z, out, stream=None) -> None:
    """dm_l2sq_matmat_noalloc: the squared-l2 product A Z into the caller's
    `out` without any allocation by the library (its scratch is a fixed
    device array; see include/dm.h for the limits and the sharing rules)."""
    import torch
    X = _as2d(X)
    Z2, o2 = _as2d(Z), _as2d(out)
    n, d = X.shape
    k = Z2.shape[1]
    code = dtype_code(X.dtype)
    if dtype_code(Z2.dtype) != code or Z2.shape[0] != n:
        raise DMError(DM_ERR_INVALID_ARG, "Z must have n rows of the points' element type")
    if tuple(o2.shape) != (n, k) or out.dtype != out_torch_dtype(code):
        raise DMError(DM_ERR_INVALID_ARG, f"out must be ({n}, {k}) of {out_torch_dtype(code)}")
    _on_device(X.device.index if X.is_cuda else -1, X, Z2, o2)
    if stream is None:
        stream = torch.cuda.current_stream(X.device).cuda_stream
    _check(load().dm_l2sq_matmat_noalloc(dtype_code(X.dtype), ctypes.c_void_p(_dev_ptr(X)), n, d,
                                         _ld(X), ctypes.c_void_p(_dev_ptr(Z2)), k, _ld(Z2),
                                         ctypes.c_void_p(_dev_ptr(o2)), _ld(o2),
                                         ctypes.c_void_p(stream)), "dm_l2sq_matmat_noalloc")
