"""Randomized block Krylov iteration over the library's distance-matrix
products: the top singular values and a low-rank approximation of A, the
application the paper draws from fast products (Appendix C, Theorems "musco"
and "singular_values_system").

Every product A Z is one dm_matmat call on a prepared plan (the library's
kernels).  The steps between products -- block Gram-Schmidt against the
earlier blocks, QR of an n x k block, the small Rayleigh-Ritz eigenproblem --
are dense linear algebra on tall-skinny blocks and go to torch (cuBLAS /
cuSOLVER); they never touch A.

For symmetric A the Krylov space of the iteration is spanned by powers of A:
Q_1 = orth(A Pi); W = A Q_i; Q_{i+1} = orth(W minus its projections on
Q_1..Q_i), the projections removed twice before and twice after an
orthonormalization (a low-rank A makes late blocks rounding noise, whose
normalized directions must be projected out again; one pass each leaves
the basis far from orthonormal in FP32).  Orthonormalization is
Cholesky QR applied twice (Gram matrix W^T W, its Cholesky factor R in
FP64, W R^-1): two skinny matrix products instead of a Householder QR of a
tall block, with Householder QR as the fallback when the block is
numerically rank deficient.  The Rayleigh-Ritz matrix M = Q^T (A Q) reuses the
products A Q_i.  Its eigenpairs (theta, V) of largest |theta| give the
singular values |theta| and A ~ U diag(theta) U^T with U = Q V.
"""
from __future__ import annotations

import torch

from . import binding


def block_krylov(plan, Pi: torch.Tensor, q: int, rank: int):
    """Run q Krylov blocks of width k = Pi.shape[1] on `plan` (q + 1 calls
    of dm_matmat with k columns).  Returns (theta, U): the `rank` Ritz values
    of largest modulus (FP64, decreasing |theta|) and their Ritz vectors
    (n x rank, Pi's dtype)."""
    if Pi.ndim != 2:
        raise ValueError("Pi must be n x k")
    n, k = Pi.shape
    if rank > q * k:
        raise ValueError("rank exceeds the Krylov dimension q * k")
    dev, dt = Pi.device, Pi.dtype
    Q = torch.empty((n, q * k), dtype=dt, device=dev)
    AQ = torch.empty((n, q * k), dtype=dt, device=dev)
    W = binding.dm_matmat(plan, Pi.contiguous())
    for i in range(q):
        prev = Q[:, : i * k]
        for _ in range(2):
            if i:
                for _ in range(2):
                    W = W - prev @ (prev.T @ W)
            W = _orthonormalize(W)
        Q[:, i * k:(i + 1) * k] = W
        binding.dm_matmat(plan, Q[:, i * k:(i + 1) * k], out=AQ[:, i * k:(i + 1) * k])
        W = AQ[:, i * k:(i + 1) * k].clone()
    M = (Q.T @ AQ).double()
    M = 0.5 * (M + M.T)
    theta, V = torch.linalg.eigh(M)
    order = torch.argsort(theta.abs(), descending=True)[:rank]
    U = Q @ V[:, order].to(dt)
    return theta[order], U


def _orthonormalize(W: torch.Tensor) -> torch.Tensor:
    """Orthonormal basis of the columns of a tall block W (n x k): Cholesky
    QR twice, or Householder QR when W is (numerically) rank deficient -- a
    Gram matrix that is not positive definite, or a Cholesky diagonal spread
    beyond 1e3, past which a Gram matrix formed in the block's precision no
    longer resolves the smallest direction."""
    Q = W
    for _ in range(2):
        G = (Q.T @ Q).double()
        R, info = torch.linalg.cholesky_ex(G, upper=True)
        dg = torch.diagonal(R).abs()
        if int(info.item()) != 0 or float(dg.min()) < 1e-3 * float(dg.max()):
            return torch.linalg.qr(W).Q
        Rinv = torch.linalg.solve_triangular(R, torch.eye(R.shape[0], dtype=R.dtype, device=R.device),
                                             upper=True)
        Q = Q @ Rinv.to(Q.dtype)
    return Q

