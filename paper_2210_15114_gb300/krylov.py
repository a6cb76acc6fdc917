"""Randomized block Krylov iteration over the library's distance-matrix
products: the top singular values and a low-rank approximation of A, the
application the paper draws from fast products (Appendix C, Theorems "musco"
and "singular_values_system").

Every product A Z is one dm_matmat call on a prepared plan (the library's
kernels).  The steps between products -- block Gram-Schmidt against the
earlier blocks, Cholesky QR of an n x k block, the Rayleigh-Ritz matrix and
the Ritz vectors -- are dense products on tall-skinny FP32 blocks, done by
the library's dm_dense_tn (P^T W, Gram matrices, Q^T (A Q)) and dm_dense_nn
(W - P T, W R^-1, Q V); only the k x k and (qk) x (qk) factorizations
(Cholesky, triangular inverse, symmetric eigenproblems) go to torch, and
blocks of another element type use torch's matrix products.  None of these
steps touches A.

For symmetric A the Krylov space of the iteration is spanned by powers of A:
Q_1 = orth(A Pi); W = A Q_i; Q_{i+1} = orth(W minus its projections on
Q_1..Q_i), the projections removed twice before an orthonormalization and
then checked: the coefficients Q^T W of the orthonormalized block are formed
once more, and where one exceeds _REORTH_TOL (a low-rank A makes late blocks
rounding noise, whose normalized directions lie largely in the span of the
basis) they are removed and the block is orthonormalized again.  Orthonormalization is
Cholesky QR applied twice (Gram matrix W^T W, its Cholesky factor R in
FP64, W R^-1): two skinny matrix products instead of a Householder QR of a
tall block.  A numerically rank-deficient block (A of rank below the Krylov
dimension: squared l2 has rank d + 2) keeps its well-resolved directions --
W V_r diag(lambda_r)^-1/2 from the FP64 eigendecomposition of its Gram
matrix -- and is filled up to k columns with seeded Gaussian columns, which
are projected off the basis and orthonormalized the same way: the basis
stays orthonormal, and the filled directions carry Ritz values at rounding
level.  The Rayleigh-Ritz matrix M = Q^T (A Q) reuses the
products A Q_i.  Its eigenpairs (theta, V) of largest |theta| give the
singular values |theta| and A ~ U diag(theta) U^T with U = Q V.
"""
from __future__ import annotations

import torch

from . import binding

# Gram eigenvalues below this fraction of the largest are rounding noise of an
# FP32 block; Cholesky factors with a diagonal spread beyond 1e3 (eigenvalue
# ratios near 1e-6) mark the block as rank deficient.
_RANK_TOL = 1e-5
_SPREAD = 1e3
# Cosine between an orthonormalized block and the basis above which the
# block is projected and orthonormalized once more (FP32 Cholesky QR leaves
# cosines near 1e-7 when the block is well resolved).
_REORTH_TOL = 1e-5
_FILL_SEED = 0x5EED


def _tn(ctx, A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    """A^T B (dm_dense_tn for FP32 blocks)."""
    if A.dtype == torch.float32 and B.dtype == torch.float32:
        return binding.dm_dense_tn(ctx, A, B)
    return A.T @ B


def _nn(ctx, A: torch.Tensor, T: torch.Tensor, out=None, alpha: float = 1.0, beta: float = 0.0):
    """beta out + alpha A T (dm_dense_nn for FP32 blocks and T up to 64
    columns); out is allocated when None."""
    if A.dtype == torch.float32 and T.dtype == torch.float32 and T.shape[1] <= 64:
        return binding.dm_dense_nn(ctx, A, T.contiguous(), out=out, alpha=alpha, beta=beta)
    r = alpha * (A @ T)
    if out is None:
        return r
    out.mul_(beta).add_(r)
    return out


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
    gen = torch.Generator(device=dev)
    gen.manual_seed(_FILL_SEED)
    ctx = plan.ctx
    W = binding.dm_matmat(plan, Pi.contiguous())
    for i in range(q):
        prev = Q[:, : i * k]
        W = _project_out(ctx, W, prev)
        W = _orthonormalize(ctx, W, prev, gen)
        if prev.shape[1]:
            C = _tn(ctx, prev, W)
            if float(C.abs().max()) > _REORTH_TOL:
                W = _nn(ctx, prev, C, out=W, alpha=-1.0, beta=1.0)
                W = _orthonormalize(ctx, W, prev, gen)
        Q[:, i * k:(i + 1) * k] = W
        binding.dm_matmat(plan, Q[:, i * k:(i + 1) * k], out=AQ[:, i * k:(i + 1) * k])
        W = AQ[:, i * k:(i + 1) * k].clone()
    # Rayleigh-Ritz matrix Q^T (A Q): symmetric, so only the block columns'
    # upper parts are formed (block column j: blocks 0..j), and the strict
    # upper triangle is mirrored
    M = torch.zeros((q * k, q * k), dtype=torch.float64, device=dev)
    for j in range(q):
        M[: (j + 1) * k, j * k:(j + 1) * k] = _tn(ctx, Q[:, : (j + 1) * k], AQ[:, j * k:(j + 1) * k]).double()
    upper = torch.triu(M, diagonal=1)
    M = upper + upper.T + torch.diag(torch.diagonal(M))
    theta, V = torch.linalg.eigh(M)
    order = torch.argsort(theta.abs(), descending=True)[:rank]
    U = _nn(ctx, Q, V[:, order].to(dt))
    # the eigensolver has synchronized already: surface any device-side error
    # of the products (a bounded wait that ran out) instead of returning
    binding.dm_sync(plan.ctx)
    return theta[order], U


def _project_out(ctx, W: torch.Tensor, prev: torch.Tensor) -> torch.Tensor:
    """W minus its projections on the orthonormal columns of prev, removed
    twice (block classical Gram-Schmidt with one reorthogonalization); W is
    updated in place."""
    if prev.shape[1] == 0:
        return W
    for _ in range(2):
        W = _nn(ctx, prev, _tn(ctx, prev, W), out=W, alpha=-1.0, beta=1.0)
    return W


def _cholqr2(ctx, W: torch.Tensor):
    """Cholesky QR applied twice, or None when W is numerically rank
    deficient (a Gram matrix that is not positive definite, or a Cholesky
    diagonal spread beyond _SPREAD, past which a Gram matrix formed in the
    block's precision no longer resolves the smallest direction)."""
    Q = W
    for _ in range(2):
        G = _tn(ctx, Q, Q).double()
        R, info = torch.linalg.cholesky_ex(G, upper=True)
        dg = torch.diagonal(R).abs()
        if int(info.item()) != 0 or float(dg.min()) * _SPREAD < float(dg.max()):
            return None
        Rinv = torch.linalg.solve_triangular(R, torch.eye(R.shape[0], dtype=R.dtype, device=R.device),
                                             upper=True)
        Q = _nn(ctx, Q, Rinv.to(Q.dtype))
    return Q


def _orthonormalize(ctx, W: torch.Tensor, prev: torch.Tensor, gen: torch.Generator) -> torch.Tensor:
    """Orthonormal basis of a tall block W (n x k) whose columns are already
    orthogonal to prev: Cholesky QR twice; for a rank-deficient W, its
    resolved directions plus seeded Gaussian fill (projected off prev),
    Householder QR only if that block is still deficient."""
    Q = _cholqr2(ctx, W)
    if Q is not None:
        return Q
    # k x k eigenproblem on the host (a small dense solve; the block stays on the device)
    lam, V = torch.linalg.eigh(_tn(ctx, W, W).double().cpu())    # ascending
    top = float(lam[-1]) if lam.numel() else 0.0
    keep = lam > max(_RANK_TOL * top, 0.0)
    r = int(keep.sum().item())
    good = _nn(ctx, W, (V[:, keep] / lam[keep].sqrt()).to(device=W.device, dtype=W.dtype))
    # unit-norm Gaussian columns, on the scale of the resolved ones
    fill = torch.randn((W.shape[0], W.shape[1] - r), generator=gen, device=W.device, dtype=W.dtype)
    fill /= W.shape[0] ** 0.5
    Wf = _project_out(ctx, torch.cat([good, fill], dim=1), prev)
    Q = _cholqr2(ctx, Wf)
    return Q if Q is not None else torch.linalg.qr(Wf).Q.contiguous()
