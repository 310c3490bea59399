"""Seeded synthetic inputs for msMINRES-CIQ workloads.

This module is shared by the FP64 oracle (``oracle/``), the CUDA library's
tests and ``bench.py``.  It holds no arithmetic of the method itself: only a
counter-based random generator and the recipes that turn a seed into the
points ``X``, the right-hand sides ``B`` and the Lanczos start vector.

Generator: splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014; the finaliser constants are the ones of
Vigna's public-domain ``splitmix64.c``).  Output ``i`` of stream ``seed`` is
the finaliser applied to ``seed + (i + 1) * 0x9E3779B97F4A7C15 (mod 2^64)``,
which is exactly the i-th output of the sequential generator started at
``seed``.  Uniforms take the top 53 bits: ``u = (z >> 11) * 2^-53`` in [0, 1).
Normals use Box-Muller on consecutive uniform pairs.

Workload recipes (the paper's datasets are not available, so these stand in
for their shapes; Sec. 4 and App. E-F of the paper give the sizes):

* ``X ~ U[0,1]^d`` row-major ``N x d``;
* ``B ~ N(0, I)`` stored as ``T x N`` (row ``c`` is right-hand side ``c``);
* the Lanczos start vector is ``2u - 1`` per entry (a random start; the paper
  only asks for a random initial vector, Sec. B.2).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream offsets so that X, B and the start vector of one seed never overlap.
STREAM_X = 1
STREAM_B = 2
STREAM_START = 3


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of splitmix64 started at ``seed``."""
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_seed(seed: int, stream: int) -> int:
    """Derive an independent stream seed (one splitmix64 draw keyed by stream)."""
    return int(splitmix64(seed ^ (stream * 0x632BE59BD9B4E019), 1)[0])


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """53-bit uniforms in [0, 1) (float64)."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on uniform pairs (float64)."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def points(seed: int, n: int, d: int) -> np.ndarray:
    """``X ~ U[0,1]^d``, shape (n, d), float64."""
    return uniform(stream_seed(seed, STREAM_X), n * d).reshape(n, d)


def rhs(seed: int, n: int, t: int) -> np.ndarray:
    """``B ~ N(0, I)``, shape (t, n): row c is right-hand side c."""
    return normal(stream_seed(seed, STREAM_B), n * t).reshape(t, n)


STREAM_ORTHO = 4


def orthogonal(seed: int, n: int) -> np.ndarray:
    """A Haar-distributed n x n orthogonal matrix (FP64): the Q factor of a
    seeded Gaussian matrix with the signs of R's diagonal moved into Q."""
    G = normal(stream_seed(seed, STREAM_ORTHO), n * n).reshape(n, n)
    Qm, R = np.linalg.qr(G)
    return Qm * np.sign(np.diag(R))[None, :]


SPECTRA = ("inv_sqrt", "inv_square")


def spectrum(kind: str, n: int) -> np.ndarray:
    """Eigenvalues of the synthetic matrices of the Q-sweep study (Sec. 5,
    Fig. quad_error): lambda_t = 1/sqrt(t) or 1/t^2, t = 1..n, descending."""
    t = np.arange(1, n + 1, dtype=np.float64)
    if kind == "inv_sqrt":
        return 1.0 / np.sqrt(t)
    if kind == "inv_square":
        return 1.0 / t ** 2
    raise ValueError(kind)


def spectrum_matrix(seed: int, n: int, kind: str):
    """(K, lam, U): K = U diag(lam) U^T in FP64 with U = orthogonal(seed, n)."""
    lam = spectrum(kind, n)
    U = orthogonal(seed, n)
    K = (U * lam[None, :]) @ U.T
    return 0.5 * (K + K.T), lam, U


def start_vector(seed: int, n: int) -> np.ndarray:
    """Lanczos start vector with entries ``2u - 1`` (float64).

    The CUDA library draws the same vector on the device from the same
    definition when no start vector is passed in.
    """
    return 2.0 * uniform(seed, n) - 1.0


@dataclasses.dataclass(frozen=True)
class Workload:
    """One GP problem: kernel, hyperparameters and solve settings."""
    name: str
    n: int
    d: int
    kernel: str          # "rbf" or "matern52"
    lengthscale: float
    outputscale: float
    noise: float         # sigma^2 added to the diagonal
    t: int               # right-hand sides
    q: int               # quadrature points
    tol: float
    max_iter: int
    op: str              # "sqrt" or "invsqrt"
    seed: int

    def make(self, n: int | None = None):
        """Return (X, B) as float64 arrays, optionally on the first ``n`` points."""
        n = self.n if n is None else n
        X = points(self.seed, self.n, self.d)[:n]
        B = rhs(self.seed, self.n, self.t)[:, :n]
        return X, B


# Workloads shaped like the paper's experiments (seed = 20201106 + index).
PLAIN_FP64_1K = Workload("matern52_n1024_d3_t1_q8", 1024, 3, "matern52", 0.2, 1.0, 1e-2,
                         1, 8, 1e-6, 200, "both", 20201106)
THOMPSON_50K = Workload("rbf_n50000_d6_t64_q12", 50_000, 6, "rbf", 0.3, 1.0, 1e-3,
                        64, 12, 1e-4, 2000, "sqrt", 20201107)
PRECISION_200K = Workload("matern52_n200000_d4_t256_q15", 200_000, 4, "matern52", 0.1, 1.0,
                          1e-2, 256, 15, 1e-4, 2000, "invsqrt", 20201108)


def batched_problems(seed: int, count: int = 512, t: int = 8):
    """Uneven independent GPs: N log-uniform in [256, 8192], d in {2..12},
    kernel RBF or Matern-5/2, lengthscale log-uniform in [0.05, 1],
    sigma^2 log-uniform in [1e-4, 1e-1], outputscale 1, ``t`` N(0,I) RHS each.

    Returns a list of dicts with the problem description and arrays.
    """
    u = uniform(stream_seed(seed, 7), 5 * count).reshape(count, 5)
    probs = []
    for p in range(count):
        n = int(math.floor(math.exp(math.log(256) + u[p, 0] * (math.log(8192) - math.log(256)))))
        n = min(max(n, 256), 8192)
        d = 2 + int(u[p, 1] * 11)
        kern = "rbf" if u[p, 2] < 0.5 else "matern52"
        ls = math.exp(math.log(0.05) + u[p, 3] * (math.log(1.0) - math.log(0.05)))
        noise = math.exp(math.log(1e-4) + u[p, 4] * (math.log(1e-1) - math.log(1e-4)))
        ps = seed * 1000003 + p
        probs.append(dict(n=n, d=d, kernel=kern, lengthscale=ls, outputscale=1.0, noise=noise,
                          X=points(ps, n, d), B=rhs(ps, n, t)))
    return probs
