"""CPU oracle for the implicit distance-matrix product of Indyk & Silwal,
"Faster Linear Algebra for Distance Matrices" (arXiv 2210.15114).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package's ``smoke()`` check and
the benchmark's CPU-baseline leg use this module; the library never imports
it, and it imports nothing from the library.  It shares no code with the CUDA
path.

Three forms, all plain and slow on purpose:

* ``l1_rows`` / ``l2sq_rows`` -- the definition ``(AZ)[r,:] = sum_j f(x_r, x_j)
  Z[j,:]`` written out as a double loop in C (``dm_oracle.c``), FP64 or exact
  int64, for all rows or a sample of rows.  f is the l1 distance of Section 2
  or the squared l2 distance of Appendix A.
* ``l1_sort`` -- Algorithm 1 (Preprocessing: sort each coordinate) followed by
  Algorithm 2 (Query for p = 1: prefix sums B_i of y_j x_j(i) and C_i of y_j
  in sorted order, then z(k) += x_k(i)(S3 - S4) + S2 - S1), in numpy.
* ``l1_grad_rows`` / ``l2sq_grad_rows`` (C), ``l1_grad_sort`` and
  ``l2sq_grad_closed`` (numpy) -- the gradient of w^T A(X) z with respect to
  X, which the paper does not state: the chain rule on the definition, and
  the same through the sorted order (l1) or the Gram decomposition (squared
  l2).
* ``block_krylov`` -- the randomized block Krylov iteration that the
  paper's application section uses (through products A Z only) for the top
  singular values and a low-rank approximation.
* ``tv_rows``, ``lpp_rows`` / ``lpp_even_expansion``, ``l2_embed`` /
  ``l2_approx`` -- the variants of Appendix A: total variation (half the l1
  product), ||x - y||_p^p by definition and by the even-p expansion, and the
  approximate l2 product through the Gaussian l2 -> l1 embedding; odd p
  through the sorted order (``lpp_odd_sort``).
* ``l2sq_identity`` -- the p = 2 query of Appendix A (Theorem
  "l2_squared_upper_bound"), with the typos of the printed algorithm read as
  the proof's Gram decomposition (Section 1.2): (Ay)_k = ||x_k||^2 sum_j y_j
  + sum_j y_j ||x_j||^2 - 2 <x_k, sum_j y_j x_j>.

Floating-point inputs are promoted to FP64 (FP32 data are compared on the same
FP32 values, promoted); integer inputs are computed in int64, whose
wrap-around arithmetic is exact whenever the true result fits in int64.

The sort order is ascending and stable (ties keep index order).  Any order of
equal values gives the same exact product, because tied pairs contribute
|0| = 0 on either side of the split.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_lib = None


def _lib_path() -> str:
    with open(_SRC, "rb") as f:
        tag = hashlib.sha1(f.read()).hexdigest()[:12]
    return os.path.join(_BUILD, f"liboracle_{tag}.so")


def build() -> str:
    """Compile ``dm_oracle.c`` with gcc (no fused multiply-add contraction, so
    x86 and Arm hosts round identically).  Returns the library path."""
    path = _lib_path()
    if os.path.exists(path):
        return path
    os.makedirs(_BUILD, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math",
                           "-shared", "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, path)
    return path


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p = ctypes.c_void_p
            i64 = ctypes.c_int64
            for name in ("oracle_l1_rows_f64", "oracle_l2sq_rows_f64",
                         "oracle_l1_rows_i64", "oracle_l2sq_rows_i64"):
                fn = getattr(lib, name)
                fn.argtypes = [p, i64, i64, p, i64, p, i64, p]
                fn.restype = None
            for name in ("oracle_l1_grad_rows_f64", "oracle_l2sq_grad_rows_f64",
                         "oracle_l1_grad_rows_i64", "oracle_l2sq_grad_rows_i64"):
                fn = getattr(lib, name)
                fn.argtypes = [p, i64, i64, p, p, i64, p, i64, p]
                fn.restype = None
            _lib = lib
    return _lib


def _is_int(a: np.ndarray) -> bool:
    return np.issubdtype(a.dtype, np.integer)


def _prep(X, Z):
    X = np.asarray(X)
    Z = np.asarray(Z)
    if X.ndim == 1:
        X = X[:, None]
    squeeze = Z.ndim == 1
    if squeeze:
        Z = Z[:, None]
    if X.shape[0] != Z.shape[0]:
        raise ValueError("X and Z must have the same number of rows")
    integer = _is_int(X) and _is_int(Z)
    dt = np.int64 if integer else np.float64
    return (np.ascontiguousarray(X, dtype=dt), np.ascontiguousarray(Z, dtype=dt),
            squeeze, integer)


def _rows_call(kind: str, X, Z, rows):
    X, Z, squeeze, integer = _prep(X, Z)
    n, d = X.shape
    k = Z.shape[1]
    if rows is None:
        rows = np.arange(n, dtype=np.int64)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    if rows.size and (rows.min() < 0 or rows.max() >= n):
        raise IndexError("row index out of range")
    out = np.zeros((rows.size, k), dtype=X.dtype)
    fn = getattr(_load(), f"oracle_{kind}_rows_{'i64' if integer else 'f64'}")
    fn(X.ctypes.data, n, d, Z.ctypes.data, k, rows.ctypes.data, rows.size,
       out.ctypes.data)
    return out[:, 0] if squeeze else out


def l1_rows(X, Z, rows=None) -> np.ndarray:
    """Definition of the l1 product (Section 2: A_ij = ||x_i - x_j||_1) for
    the given rows (all rows when ``rows`` is None).  O(n d k) per row."""
    return _rows_call("l1", X, Z, rows)


def l2sq_rows(X, Z, rows=None) -> np.ndarray:
    """Definition of the squared-l2 product (Appendix A: A_ij =
    ||x_i - x_j||_2^2) for the given rows.  O(n d k) per row."""
    return _rows_call("l2sq", X, Z, rows)


def preprocessing_order(column) -> np.ndarray:
    """Algorithm 1 for one coordinate: the order pi^i that sorts the i-th
    coordinates ascending (stable; ties keep index order)."""
    return np.argsort(np.asarray(column), kind="stable")


def l1_sort(X, Z) -> np.ndarray:
    """Algorithms 1 and 2 (Section 2) for the l1 product of every row.

    For each coordinate i: sort (Algorithm 1), then form the prefix arrays
    B_i (partial sums of y_j x_j(i)) and C_i (partial sums of y_j) in the
    sorted order, with B_i[q] / C_i[q] the sums over the q points that come
    strictly before position q -- the sets {j : pi(j) < pi(k)} of the proof of
    Theorem "p=1".  For every point k at position q:
        S1 = B_i[q], S2 = B_i[n] - B_i[q], S3 = C_i[q], S4 = C_i[n] - C_i[q],
        z(k) += x_k(i) (S3 - S4) + S2 - S1.
    Each column of a block Z is an independent query (Lemma "matrixmult").
    """
    X, Z, squeeze, _ = _prep(X, Z)
    n, d = X.shape
    out = np.zeros(Z.shape, dtype=X.dtype)
    zero_row = np.zeros((1, Z.shape[1]), dtype=X.dtype)
    for i in range(d):
        order = preprocessing_order(X[:, i])                 # Algorithm 1
        xs = X[order, i]
        ys = Z[order]
        B = np.concatenate([zero_row, np.cumsum(xs[:, None] * ys, axis=0)])
        C = np.concatenate([zero_row, np.cumsum(ys, axis=0)])
        q = np.empty(n, dtype=np.int64)
        q[order] = np.arange(n)                               # position of x_k(i)
        S1 = B[q]
        S2 = B[n] - B[q]
        S3 = C[q]
        S4 = C[n] - C[q]
        out += X[:, i, None] * (S3 - S4) + S2 - S1
    return out[:, 0] if squeeze else out


def l2sq_identity(X, Z) -> np.ndarray:
    """Query for p = 2 (Appendix A), every row:
        v  = sum_j y_j x_j          (d x k)
        S1 = sum_j y_j              (k)
        S2 = sum_j y_j ||x_j||^2    (k)
        z(k) = S1 ||x_k||^2 + S2 - 2 <x_k, v>.
    The printed algorithm squares y_j in S1 and S2; the proof's Gram
    decomposition (Section 1.2) fixes the reading used here."""
    X, Z, squeeze, _ = _prep(X, Z)
    sq = np.einsum("ij,ij->i", X, X)
    v = X.T @ Z
    S1 = Z.sum(axis=0)
    S2 = sq @ Z
    out = sq[:, None] * S1[None, :] + S2[None, :] - 2 * (X @ v)
    return out[:, 0] if squeeze else out


def _prep_grad(X, W, Z):
    X = np.asarray(X)
    if X.ndim == 1:
        X = X[:, None]
    W = np.asarray(W)
    Z = np.asarray(Z)
    if W.ndim == 1:
        W = W[:, None]
    if Z.ndim == 1:
        Z = Z[:, None]
    if not (X.shape[0] == W.shape[0] == Z.shape[0]) or W.shape != Z.shape:
        raise ValueError("X, W and Z must have n rows; W and Z the same shape")
    integer = _is_int(X) and _is_int(W) and _is_int(Z)
    dt = np.int64 if integer else np.float64
    return (np.ascontiguousarray(X, dtype=dt), np.ascontiguousarray(W, dtype=dt),
            np.ascontiguousarray(Z, dtype=dt), integer)


def _grad_rows_call(kind: str, X, W, Z, rows):
    X, W, Z, integer = _prep_grad(X, W, Z)
    n, d = X.shape
    k = W.shape[1]
    if rows is None:
        rows = np.arange(n, dtype=np.int64)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    if rows.size and (rows.min() < 0 or rows.max() >= n):
        raise IndexError("row index out of range")
    G = np.zeros((rows.size, d), dtype=X.dtype)
    fn = getattr(_load(), f"oracle_{kind}_grad_rows_{'i64' if integer else 'f64'}")
    fn(X.ctypes.data, n, d, W.ctypes.data, Z.ctypes.data, k, rows.ctypes.data, rows.size,
       G.ctypes.data)
    return G


def l1_grad_rows(X, W, Z, rows=None) -> np.ndarray:
    """Gradient of L = sum_q w_q^T A(X) z_q with respect to X for the l1
    matrix (the paper states none: the chain rule on the definition, with the
    symmetric subgradient sgn(0) = 0):
        dL/dx_i(c) = sum_q sum_j (w_iq z_jq + z_iq w_jq) sgn(x_i(c) - x_j(c)).
    Rows ``rows`` of the n x d gradient (all when None); O(n d k) per row."""
    return _grad_rows_call("l1", X, W, Z, rows)


def l2sq_grad_rows(X, W, Z, rows=None) -> np.ndarray:
    """Gradient of L = sum_q w_q^T A(X) z_q for the squared-l2 matrix:
        dL/dx_i(c) = sum_q sum_j (w_iq z_jq + z_iq w_jq) 2 (x_i(c) - x_j(c))."""
    return _grad_rows_call("l2sq", X, W, Z, rows)


def l1_grad_sort(X, W, Z) -> np.ndarray:
    """The l1 gradient of every row through the sorted order of each
    coordinate (Algorithm 1's sort, with prefix sums as in Algorithm 2).

    For a point at sorted position r whose value is shared by the tie group of
    positions a..b, sum_j y_j sgn(x_r - x_j) is the sum of y over the strictly
    smaller values minus the sum over the strictly larger ones:
        S_y(r) = E_y[a] - (T_y - I_y[b]),
    with E the exclusive and I the inclusive prefix sum of y in sorted order
    and T the total.  Then dL/dx_i(c) = sum_q w_iq S_z(r) + z_iq S_w(r).
    Integer inputs are computed in int64; others in FP64."""
    X, W, Z, _ = _prep_grad(X, W, Z)
    n, d = X.shape
    G = np.zeros((n, d), dtype=X.dtype)
    for c in range(d):
        order = preprocessing_order(X[:, c])
        xs = X[order, c]
        head = np.ones(n, dtype=bool)
        head[1:] = xs[1:] != xs[:-1]
        gid = np.cumsum(head) - 1                  # tie group of each position
        first = np.flatnonzero(head)               # a of each group
        last = np.append(first[1:] - 1, n - 1)     # b of each group
        a = first[gid]
        b = last[gid]
        for Y, other in ((Z, W), (W, Z)):
            ys = Y[order]
            inc = np.cumsum(ys, axis=0)
            exc = inc - ys
            S = exc[a] - (inc[-1][None, :] - inc[b])
            G[order, c] += (other[order] * S).sum(axis=1)
    return G


def l2sq_grad_closed(X, W, Z) -> np.ndarray:
    """The squared-l2 gradient in closed form, from the Gram decomposition of
    Section 1.2 (sum over j of the definition, expanded):
        dL/dx_i = 2 sum_q [ x_i (w_iq 1^T z_q + z_iq 1^T w_q)
                            - w_iq X^T z_q - z_iq X^T w_q ]."""
    X, W, Z, _ = _prep_grad(X, W, Z)
    sz = Z.sum(axis=0)
    sw = W.sum(axis=0)
    XtZ = X.T @ Z                                   # d x k
    XtW = X.T @ W
    coef = W @ sz + Z @ sw                          # n
    return 2 * (X * coef[:, None] - W @ XtZ.T - Z @ XtW.T)


def block_krylov(product, Pi, q: int, rank: int):
    """Randomized block Krylov iteration for the top `rank` singular values
    and a rank-`rank` approximation of a symmetric matrix A that is reached
    only through products Y = A Z (the application of Appendix C, Theorems
    "musco" and "singular_values_system").  FP64, numpy.

    Steps (for symmetric A the Krylov space of A^T A A Pi, ... is spanned
    by powers of A): Q_1 = orth(A Pi); for i = 1..q: W = A Q_i, and -- while
    i < q -- Q_{i+1} = orth(W minus its projections on Q_1..Q_i).  The
    projections are removed twice, the block is orthonormalized (QR), and
    the projections are removed twice more before a final QR: when A has
    low rank the new block can be pure rounding noise, whose normalized
    directions lean on the earlier blocks until they are projected out
    again.  Then the Rayleigh-Ritz step M = Q^T (A Q)
    on Q = [Q_1 .. Q_q] (the products A Q_i are reused), its eigenpairs
    (theta, V), and the `rank` pairs of largest |theta|: singular values
    |theta| and A ~ U diag(theta) U^T with U = Q V.
    Returns (theta, U) ordered by decreasing |theta|."""
    Pi = np.asarray(Pi, dtype=np.float64)
    W = np.asarray(product(Pi), dtype=np.float64)
    blocks, products = [], []
    for i in range(q):
        for _ in range(2):
            for _ in range(2):
                for B in blocks:
                    W = W - B @ (B.T @ W)
            W, _ = np.linalg.qr(W)
        Qi = W
        blocks.append(Qi)
        W = np.asarray(product(Qi), dtype=np.float64)
        products.append(W)
    Q = np.concatenate(blocks, axis=1)
    AQ = np.concatenate(products, axis=1)
    M = Q.T @ AQ
    M = 0.5 * (M + M.T)
    theta, V = np.linalg.eigh(M)
    order = np.argsort(-np.abs(theta))[:rank]
    return theta[order], Q @ V[:, order]


def tv_rows(X, Z, rows=None) -> np.ndarray:
    """Total variation distance of distributions x_i over d outcomes
    (Appendix A, "Distances for Distributions", Theorem "tv"):
    TV(x, y) = (1/2) ||x - y||_1, so the product is half the l1 product."""
    return 0.5 * l1_rows(X, Z, rows)


def lpp_rows(X, Z, p: int, rows=None) -> np.ndarray:
    """Definition of the product for f(x, y) = ||x - y||_p^p (Appendix A,
    "General p"), any integer p >= 1: a direct double loop in numpy, FP64
    (int64 for integer inputs, exact when the result fits)."""
    X = np.asarray(X)
    Z = np.asarray(Z)
    if X.ndim == 1:
        X = X[:, None]
    squeeze = Z.ndim == 1
    if squeeze:
        Z = Z[:, None]
    integer = _is_int(X) and _is_int(Z)
    dt = np.int64 if integer else np.float64
    X = X.astype(dt)
    Z = Z.astype(dt)
    if rows is None:
        rows = np.arange(len(X))
    out = np.zeros((len(rows), Z.shape[1]), dtype=dt)
    for r, i in enumerate(np.asarray(rows)):
        diff = np.abs(X[i][None, :] - X)
        dist = (diff ** p).sum(axis=1)
        out[r] = dist @ Z
    return out[:, 0] if squeeze else out


def lpp_even_expansion(X, Z, p: int) -> np.ndarray:
    """The query for even p of Appendix A in its corrected reading: with
    S_{i,t} = C(p, t) sum_j y_j (-x_j(i))^(p-t) for t = 0..p,
    (Ay)(k) = sum_i sum_t x_k(i)^t S_{i,t}.  (The printed algorithm omits
    y_j and the binomial coefficients and starts t at 1.)  FP64 / int64."""
    if p % 2:
        raise ValueError("p must be even")
    X = np.asarray(X)
    Z = np.asarray(Z)
    if X.ndim == 1:
        X = X[:, None]
    squeeze = Z.ndim == 1
    if squeeze:
        Z = Z[:, None]
    integer = _is_int(X) and _is_int(Z)
    dt = np.int64 if integer else np.float64
    X = X.astype(dt)
    Z = Z.astype(dt)
    out = np.zeros((len(X), Z.shape[1]), dtype=dt)
    from math import comb
    for i in range(X.shape[1]):
        x = X[:, i]
        for t in range(p + 1):
            S = comb(p, t) * (((-x) ** (p - t))[None, :] @ Z)      # 1 x k
            out += (x ** t)[:, None] * S
    return out[:, 0] if squeeze else out


def lpp_odd_sort(X, Z, p: int) -> np.ndarray:
    """||x - y||_p^p for odd p through the sorted order (Theorem "odd_p":
    the p = 1 technique with p + 1 prefix sums per coordinate).  For the
    point at sorted position r of coordinate i, inside the tie group a..b,
    with sums over the strictly smaller (L) and strictly larger (R) values,
        sum_j y_j |x - x_j|^p = sum_t C(p, t) x^t (L_{p-t} - R_{p-t}),
        L_s = sum_{x_j < x} y_j (-x_j)^s,  R_s = sum_{x_j > x} y_j (-x_j)^s
    (ties contribute |0|^p = 0).  FP64 / int64."""
    if p % 2 == 0:
        raise ValueError("p must be odd")
    from math import comb
    X = np.asarray(X)
    Z = np.asarray(Z)
    if X.ndim == 1:
        X = X[:, None]
    squeeze = Z.ndim == 1
    if squeeze:
        Z = Z[:, None]
    integer = _is_int(X) and _is_int(Z)
    dt = np.int64 if integer else np.float64
    X = X.astype(dt)
    Z = Z.astype(dt)
    n, d = X.shape
    out = np.zeros((n, Z.shape[1]), dtype=dt)
    for i in range(d):
        order = preprocessing_order(X[:, i])
        xs = X[order, i]
        head = np.ones(n, dtype=bool)
        head[1:] = xs[1:] != xs[:-1]
        gid = np.cumsum(head) - 1
        first = np.flatnonzero(head)
        last = np.append(first[1:] - 1, n - 1)
        a, b = first[gid], last[gid]
        ys = Z[order]
        acc = np.zeros_like(ys)
        for t in range(p + 1):
            w = ys * ((-xs) ** (p - t))[:, None]
            inc = np.cumsum(w, axis=0)
            exc = inc - w
            S = exc[a] - (inc[-1][None, :] - inc[b])
            acc += comb(p, t) * (xs ** t)[:, None] * S
        out[order] += acc
    return out[:, 0] if squeeze else out


L2_EMBED_BETA = float(np.sqrt(2.0 / np.pi))


def l2_embed(X, G) -> np.ndarray:
    """The linear map of Theorem "l2embed": T(x)_i = (1/(beta m)) sum_j
    G_ij x_j with beta = sqrt(2/pi) and G an m x d matrix of N(0, 1)
    entries, applied to every point (rows of X); FP64."""
    X = np.asarray(X, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    return X @ G.T / (L2_EMBED_BETA * G.shape[0])


def l2_approx(X, G, Z) -> np.ndarray:
    """Approximate l2 product of Appendix A ("Approximate Matrix-Vector Query
    for l2"): the l1 product (Algorithms 1 and 2) of the embedded points."""
    return l1_sort(l2_embed(X, G), Z)


def relative_error(got, want) -> float:
    """Frobenius relative error ||got - want|| / ||want|| over the whole block
    (0 when both are zero)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    den = np.linalg.norm(want)
    num = np.linalg.norm(got - want)
    if den == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return float(num / den)
