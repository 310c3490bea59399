"""FP64 CPU oracle for msMINRES-CIQ (Pleiss et al., "Fast Matrix Square Roots
with Applications to Gaussian Processes and Bayesian Optimization", 2020).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg may import it.  The CUDA library never
calls it, and it shares no code with the CUDA library: the only module both
sides use is ``ciq_inputs`` (seeded random inputs, no method arithmetic).

Two parts:

* O1 ``eig``      -- the definition: K^{+-1/2} b = V diag(lambda^{+-1/2}) V^T b
                     through a dense symmetric eigendecomposition.
* O2 ``ciq``      -- plain serial msMINRES-CIQ in FP64, step by step:
                     Lanczos bounds (App. B.2), Hale-Higham-Trefethen nodes
                     (Eq. quad_points_and_locations, Eq. contour_integral_quad_4,
                     Algorithm "quadrature"), multi-shift MINRES (App. C,
                     Eq. minres_qr_shifted) and the CIQ sum
                     (Eq. contour_integral_quad, Algorithm "ciq").

Every function cites the passage it follows.  Pins (tests marked
``not gpu``) tie each part to closed forms, library routines (SciPy, LAPACK)
and brute force rather than to the oracle itself.  The lambda_min reading
for sigma^2 = 0 (theta_min / 100), which the paper leaves open, is pinned on
the matrices it is used for (it lies below LAPACK's smallest eigenvalue there);
it is not a bound in general.
"""
