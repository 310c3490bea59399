"""Per-column relative errors for the parity tests.

Right-hand sides travel as the rows of a (T, N) array: row c is column c of
the C layout.  The tolerance of the method's results is a relative 2-norm per
right-hand side, so every comparison takes each row's error on its own and
gates on the largest one (a single bad column cannot hide inside a norm over
all of them).  A 1-D array is one column.
"""
import numpy as np


def colrel(a, b):
    """Relative 2-norm error of each row of ``a`` against the same row of ``b``."""
    a = np.atleast_2d(np.asarray(a, dtype=np.float64))
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    assert a.shape == b.shape, (a.shape, b.shape)
    num = np.linalg.norm(a - b, axis=1)
    den = np.linalg.norm(b, axis=1)
    zero = den == 0.0
    return np.where(zero, np.where(num == 0.0, 0.0, np.inf), num / np.where(zero, 1.0, den))


def rel(a, b):
    """Largest per-row relative error (see ``colrel``)."""
    return float(colrel(a, b).max())


def fp32_gate(run, K, ref, factor=15.0, least=1e-5):
    """Tolerance of an FP32 solve against the FP64 oracle at equal nodes and J.

    ``run(Km)`` returns the oracle's result (rows = right-hand sides) for the
    matrix ``Km``; ``ref`` is that result for ``K`` itself.  The oracle run on
    K rounded entry by entry to FP32 is what exact arithmetic makes of the
    best kernel entries an FP32 path can hold: its distance from ``ref`` is a
    floor no FP32 evaluation of K can go below.  K^{-1/2}b is sensitive to it
    (at kappa ~ 1e4 the floor alone is 4e-6 to 7e-6).  The FP32 path adds the
    rounding of its Lanczos vectors, of each MVM result and up to 2 ulp per
    kernel entry (expf, FP32 distances): emulated on the CPU that came to 4-6
    times the floor, measured on the GPU 9-11 times.  The gate is
    ``max(least, factor * floor)``.
    """
    K32 = np.asarray(K, dtype=np.float64).astype(np.float32).astype(np.float64)
    floor = rel(run(K32), ref)
    return max(least, factor * floor), floor
