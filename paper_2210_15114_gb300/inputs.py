"""Seeded synthetic inputs for the distance-matrix product.

This module only draws numbers; it holds none of the method's arithmetic.
Both the CUDA path (through the tests and the benchmark) and the CPU oracle
receive the very same arrays from here.  Every generator uses numpy's PCG64
``default_rng(seed)``, draws in FP64 and casts at the end, so a FP32 input is
the FP64 draw rounded once.

Workload shapes follow the paper's own experiments (Section 4: points from a
mixture of spherical Gaussians; query vectors with Gaussian entries) and the
sizes the library is benchmarked on:

* ``uniform_points``   -- coordinates uniform in [lo, hi).
* ``gaussian_mixture`` -- ``clusters`` spherical Gaussians, cluster means drawn
  N(0, mean_sd^2) per coordinate, within-cluster sd ``sd``, cluster chosen
  uniformly per point.
* ``integer_points``   -- integer coordinates uniform in [lo, hi).
* ``gaussian_queries`` -- query block Z with N(0, 1) entries.
* ``integer_queries``  -- integer query block uniform in [lo, hi].
* ``grid_1d``          -- the 1-D grid x_i = i.
"""
from __future__ import annotations

import numpy as np

SEED_X = 0
SEED_Z = 1


def uniform_points(n: int, d: int, seed: int = SEED_X, lo: float = 0.0,
                   hi: float = 1.0, dtype=np.float64) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n, d)).astype(dtype)


def gaussian_mixture(n: int, d: int, clusters: int, seed: int = SEED_X,
                     mean_sd: float = 10.0, sd: float = 1.0,
                     dtype=np.float32) -> np.ndarray:
    rng = np.random.default_rng(seed)
    means = rng.normal(0.0, mean_sd, size=(clusters, d))
    label = rng.integers(0, clusters, size=n)
    pts = means[label] + rng.normal(0.0, sd, size=(n, d))
    return pts.astype(dtype)


def integer_points(n: int, d: int, seed: int = SEED_X, lo: int = 0,
                   hi: int = 1 << 16, dtype=np.int32) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi, size=(n, d)).astype(dtype)


def gaussian_queries(n: int, k: int, seed: int = SEED_Z,
                     dtype=np.float32) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 1.0, size=(n, k)).astype(dtype)


def integer_queries(n: int, k: int, seed: int = SEED_Z, lo: int = -100,
                    hi: int = 100, dtype=np.int32) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(n, k)).astype(dtype)


def grid_1d(n: int, dtype=np.float64) -> np.ndarray:
    return np.arange(n, dtype=np.float64).reshape(n, 1).astype(dtype)


def sample_rows(n: int, count: int, seed: int = 7) -> np.ndarray:
    """Row indices for sampled checks: the first and last rows plus a seeded
    uniform sample, sorted and unique."""
    rng = np.random.default_rng(seed)
    rows = np.concatenate([[0, n - 1], rng.integers(0, n, size=max(0, count - 2))])
    return np.unique(rows.astype(np.int64))


# The workloads the library is measured and checked on.
def workload_small_f64():
    """n = 4096 points, d = 8, coordinates uniform [0, 1) in FP64; one FP64
    Gaussian query."""
    X = uniform_points(4096, 8, SEED_X, dtype=np.float64)
    z = gaussian_queries(4096, 1, SEED_Z, dtype=np.float64)
    return X, z


def workload_mixture_f32(n: int = 1 << 20, d: int = 32, k: int = 16):
    """16-cluster Gaussian mixture (means N(0, 10^2), sd 1), FP32 points and an
    FP32 N(0, 1) query block of k columns."""
    X = gaussian_mixture(n, d, 16, SEED_X, 10.0, 1.0, dtype=np.float32)
    Z = gaussian_queries(n, k, SEED_Z, dtype=np.float32)
    return X, Z


def workload_integer(n: int = 1 << 20, d: int = 32, k: int = 16):
    """int32 coordinates uniform in [0, 2^16), int32 query entries uniform in
    [-100, 100]."""
    X = integer_points(n, d, SEED_X, 0, 1 << 16)
    Z = integer_queries(n, k, SEED_Z, -100, 100)
    return X, Z


SEED_W = 1     # the gradient's left vector w
SEED_ZG = 2    # the gradient's right vector z


def workload_gradient(n: int = 1 << 21, d: int = 64, k: int = 1, tie_heavy: bool = False):
    """Points for the gradient of w^T A(X) z: FP32 coordinates uniform in
    [0, 1), or -- the tie-heavy variant -- integers uniform in [0, 1023]
    stored as FP32 (about n / 1024 points share each value of a coordinate);
    w and z are FP32 N(0, 1) columns (k of each)."""
    rng = np.random.default_rng(SEED_X)
    if tie_heavy:
        X = rng.integers(0, 1024, size=(n, d)).astype(np.float32)
    else:
        X = rng.uniform(0.0, 1.0, size=(n, d)).astype(np.float32)
    W = gaussian_queries(n, k, SEED_W, dtype=np.float32)
    Z = gaussian_queries(n, k, SEED_ZG, dtype=np.float32)
    return X, W, Z



SEED_PI = 3    # the Gaussian start block of the Krylov iteration


def workload_krylov(n: int = 1 << 22, d: int = 16, k: int = 40, clusters: int = 10):
    """Points for the block Krylov row: a `clusters`-cluster Gaussian mixture
    (means N(0, 10^2), sd 1) in FP32, and the FP32 N(0, 1) start block Pi
    (n x k)."""
    X = gaussian_mixture(n, d, clusters, SEED_X, 10.0, 1.0, dtype=np.float32)
    Pi = gaussian_queries(n, k, SEED_PI, dtype=np.float32)
    return X, Pi


def workload_batch(nsets: int = 512, n_lo: int = 1024, n_hi: int = 262144, d_lo: int = 2,
                   d_hi: int = 64, k_lo: int = 1, k_hi: int = 32, seed0: int = 1000,
                   dtype=np.float32):
    """Independent point sets of uneven size: set s draws from seed seed0 + s
    its n (log-uniform in [n_lo, n_hi], rounded), d (uniform in
    {d_lo..d_hi}), k (uniform in {k_lo..k_hi}), coordinates uniform in
    [-1, 1) and queries N(0, 1).  Integer dtype: coordinates uniform in
    [0, 2^16), queries in [-100, 100].  Returns a list of (X, Z)."""
    out = []
    for s in range(nsets):
        rng = np.random.default_rng(seed0 + s)
        n = int(round(float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))))
        d = int(rng.integers(d_lo, d_hi + 1))
        k = int(rng.integers(k_lo, k_hi + 1))
        if np.issubdtype(np.dtype(dtype), np.integer):
            X = rng.integers(0, 1 << 16, size=(n, d)).astype(dtype)
            Z = rng.integers(-100, 101, size=(n, k)).astype(dtype)
        else:
            X = rng.uniform(-1.0, 1.0, size=(n, d)).astype(dtype)
            Z = rng.normal(0.0, 1.0, size=(n, k)).astype(dtype)
        out.append((X, Z))
    return out


SEED_G = 4     # the Gaussian matrix of the l2 -> l1 embedding


def embedding_matrix(m: int, d: int, dtype=np.float32) -> np.ndarray:
    """The m x d N(0, 1) matrix G of the l2 -> l1 embedding (seed 4)."""
    return np.random.default_rng(SEED_G).normal(0.0, 1.0, size=(m, d)).astype(dtype)


def simplex_points(n: int, d: int, seed: int = SEED_X, dtype=np.float32) -> np.ndarray:
    """Discrete distributions over d outcomes (Dirichlet(1, ..., 1) rows),
    the inputs of the total-variation product."""
    return np.random.default_rng(seed).dirichlet(np.ones(d), size=n).astype(dtype)


def workload_offset_mixture(n: int, d: int, k: int, offset: float = 1000.0):
    """The 16-cluster mixture shifted by `offset` in every coordinate, FP32
    (the shift costs the FP32 coordinates about log2(offset / 10) bits of the
    spread), with an N(0, 1) query block of k columns (mixed signs)."""
    X = (gaussian_mixture(n, d, 16, SEED_X, 10.0, 1.0, dtype=np.float64) + offset).astype(np.float32)
    Z = gaussian_queries(n, k, SEED_Z, dtype=np.float32)
    return X, Z

