"""Explicit-matrix solves (ciq_sqrt_dense / ciq_invsqrt_dense) against the
FP64 oracle and the eigendecomposition, on the synthetic spectra of the
Q-sweep study (Sec. 5, Fig. quad_error: lambda_t = 1/sqrt(t), 1/t^2, and a
one-dimensional Matern kernel matrix on random points)."""
import numpy as np
import pytest
import torch

import ciq_inputs as ci
import paper_2006_11267_b300 as P
from oracle import ciq as O
from oracle import eig, kernels
from relerr import fp32_gate, rel

pytestmark = pytest.mark.gpu



def matrix(kind, n, seed):
    if kind == "matern1d":
        # sigma^2 = 1e-4 keeps the FP32 matrix positive definite
        X = ci.points(seed, n, 1)
        return kernels.dense_K(X, "matern52", 0.2, 1.0, 1e-4)
    return ci.spectrum_matrix(seed, n, kind)[0]


@pytest.mark.parametrize("op", ["sqrt", "invsqrt"])
@pytest.mark.parametrize("krylov", ["recurrence", "basis"])
def test_dense_solve_matches_oracle_at_equal_nodes_and_J(op, krylov):
    n, T, Q, J = 1000, 5, 10, 150
    K32 = matrix("inv_sqrt", n, 3).astype(np.float32)
    K = K32.astype(np.float64)
    B = ci.rhs(4, n, T).astype(np.float32)
    lam = np.linalg.eigvalsh(K)
    nodes = O.quad_nodes(lam[0], lam[-1], Q)
    ref, info_o = O.ciq_apply(O.dense_mvm(K), B.astype(np.float64), Q, op, max_iter=J, nodes=nodes,
                              lmin=lam[0], lmax=lam[-1])
    fn = P.ciq_sqrt_dense if op == "sqrt" else P.ciq_invsqrt_dense
    out, info = fn(torch.from_numpy(K32).cuda(), torch.from_numpy(B).cuda(), Q, 0.0, max_iter=J,
                   nodes=nodes, lmin=lam[0], lmax=lam[-1], krylov=krylov)
    assert info["iters"] == J and info["krylov"] == krylov
    # The matrix is given in FP32, so the oracle already sees the rounded
    # entries: the gate is 1e-5, or 15 times the change that rounding them
    # once more would cause (relerr.fp32_gate) when that is larger.
    tol, floor = fp32_gate(
        lambda Km: O.ciq_apply(O.dense_mvm(Km), B.astype(np.float64), Q, op, max_iter=J, nodes=nodes,
                               lmin=lam[0], lmax=lam[-1])[0], K, ref)
    err = rel(out.cpu().numpy(), ref)
    assert err < tol, (err, tol, floor)


@pytest.mark.parametrize("kind", ["inv_sqrt", "inv_square", "matern1d"])
def test_q_sweep_on_the_studys_matrices(kind):
    # The study's setting: Lanczos bounds, relative residual 1e-4 or J = 400.
    # Error against the eigendecomposition of the FP32 matrix.  Q = 8 meets
    # 1e-4 on the well-conditioned 1/sqrt(t) spectrum; the ill-conditioned
    # ones (kappa ~ 1e6: the lower bound is theta_min / 100 without a noise
    # term) need Q = 12 for 1e-3 here.  The error falls with Q up to the
    # solve's own level.
    n, T = 1024, 4
    K32 = matrix(kind, n, 11).astype(np.float32)
    B = ci.rhs(12, n, T).astype(np.float32)
    exact = eig.sqrt_apply(K32.astype(np.float64), B.T.astype(np.float64)).T
    errs = {}
    for q in (4, 8, 12):
        out, info = P.ciq_sqrt_dense(K32, B, q, 1e-4, max_iter=400, stop_rule="residual")   # host arrays
        assert info["status"] in (0, 4)
        errs[q] = (np.linalg.norm(out - exact, axis=1) / np.linalg.norm(exact, axis=1)).max()
    assert errs[4] > errs[8] > 0 and errs[12] < 1.5 * errs[8]
    if kind == "inv_sqrt":
        assert errs[8] < 1e-4
    else:
        assert errs[12] < 1e-3, errs


def test_dense_identity_and_scaled_identity():
    # K = c I: K^{1/2} b = sqrt(c) b and K^{-1/2} b = b / sqrt(c) (one Lanczos step).
    K = (4.0 * np.eye(300)).astype(np.float32)
    B = ci.rhs(2, 300, 3).astype(np.float32)
    out, info = P.ciq_sqrt_dense(torch.from_numpy(K).cuda(), torch.from_numpy(B).cuda(), 8, 1e-6,
                                 lmin=4.0, lmax=4.0)
    assert rel(out.cpu().numpy(), 2.0 * B) < 1e-6 and info["iters"] <= 2
    out, _ = P.ciq_invsqrt_dense(torch.from_numpy(K).cuda(), torch.from_numpy(B).cuda(), 8, 1e-6,
                                 lmin=4.0, lmax=4.0)
    assert rel(out.cpu().numpy(), 0.5 * B) < 1e-6


def test_dense_wide_block_and_tiny_matrix():
    # T = 70 (two column groups) and N = 1
    K32 = matrix("inv_sqrt", 600, 5).astype(np.float32)
    B = ci.rhs(6, 600, 70).astype(np.float32)
    exact = eig.invsqrt_apply(K32.astype(np.float64), B.T.astype(np.float64)).T
    out, info = P.ciq_invsqrt_dense(torch.from_numpy(K32).cuda(), torch.from_numpy(B).cuda(), 10, 1e-7,
                                    max_iter=300)
    assert rel(out.cpu().numpy(), exact) < 1e-4
    one = np.array([[2.25]], np.float32)
    out, _ = P.ciq_sqrt_dense(one, np.array([[3.0]], np.float32), 6, 1e-8, lmin=2.25, lmax=2.25)
    assert abs(out[0, 0] - 4.5) < 1e-5
