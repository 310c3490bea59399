"""Preconditioned msMINRES-CIQ (App. "Preconditioning msMINRES-CIQ", Eq.
precond_sqrt, Eq. precond_sqrt_inverse) through the C ABI against the FP64
oracle (oracle/precond.py, pinned in tests/test_oracle_precond.py).

The preconditioner's factor for the parity cases is the oracle's own pivoted
Cholesky factor, rounded to FP32 and handed to both sides, so that both solve
with the same P = L L^T + sigma^2 I; the device's pivoted Cholesky is checked
against the oracle's separately.  Errors are relative 2-norms per right-hand
side (tests/relerr.py)."""
import numpy as np
import pytest
import scipy.linalg
import torch

import ciq_inputs as ci
import paper_2006_11267_b300 as P
from oracle import kernels
from oracle import precond as PC
from oracle.quadrature import quad_nodes
from relerr import colrel, fp32_gate, rel

pytestmark = pytest.mark.gpu


def case(n, d, t, seed, kind="matern52", ls=0.25, noise=1e-2):
    X = ci.points(seed, n, d).astype(np.float32)
    B = ci.rhs(seed + 1, n, t).astype(np.float32)
    X64 = X.astype(np.float64)
    Kxx = kernels.kernel_matrix(X64, X64, kind, ls, 1.0)
    return X, B, Kxx, Kxx + noise * np.eye(n), P.Kernel(kind, ls, 1.0, noise)


def oracle_factor(Kxx, rank):
    """The oracle's pivoted Cholesky factor rounded to FP32 (both sides use
    it): (L of shape (n, rank) for the oracle, its transpose (rank, n) -- row m
    is column m -- for the library, pivots)."""
    L, piv = PC.pivoted_cholesky(np.diag(Kxx), lambda i: Kxx[:, i], rank)
    L32 = L.astype(np.float32)
    return L32, np.ascontiguousarray(L32.T), piv


@pytest.mark.parametrize("kind,n,d,rank", [("rbf", 700, 3, 40), ("matern52", 1000, 5, 64), ("rbf", 129, 2, 129)])
def test_pivoted_cholesky_matches_oracle(kind, n, d, rank):
    X, _, Kxx, _, k = case(n, d, 1, 30 + n, kind, ls=0.3)
    L_o, piv_o = PC.pivoted_cholesky(np.diag(Kxx), lambda i: Kxx[:, i], rank)
    L, piv, got = P.ciq_pivoted_cholesky(torch.from_numpy(X).cuda(), k, rank)
    L = L.cpu().numpy().astype(np.float64)
    piv = piv.cpu().numpy()
    # Pivots are index work: equal while the oracle's choice is not a near
    # tie.  The device's residual diagonal s - sum_m l_im^2 carries FP32
    # kernel values (relative error ~1e-7 in each l_im), so two candidates
    # are told apart when their residuals differ by more than 1e-5 times the
    # part already removed from the diagonal.  Step 0 is an exact tie (every
    # diagonal entry is the outputscale) that both sides break by the first index.
    m = 0
    s = 1.0
    for j in range(got):
        dres = s - np.sum(L_o[:, :j] ** 2, axis=1)
        order = np.argsort(-dres, kind="stable")
        a, b = order[0], order[1]
        if j > 0 and dres[a] - dres[b] < 1e-5 * max(s - dres[b], 1e-12) + 1e-12:
            break
        assert piv[j] == piv_o[j], j
        m = j + 1
    assert m >= min(rank, 20)
    err = colrel(L[:m], L_o[:, :m].T)
    assert err.max() < 1e-3, err.max()
    # Valid in any case: L L^T below K_XX (the residual is positive semidefinite
    # up to FP32 rounding) and exact zeros above the diagonal in pivot order.
    E = Kxx - L.T @ L
    assert np.linalg.eigvalsh(E).min() > -1e-5 * np.abs(Kxx).max()
    Lp = L[:got][:, piv[:got]]
    assert np.abs(np.tril(Lp, -1)).max() == 0.0


def _nodes_of_A(K, Pm, Q):
    lam = scipy.linalg.eigh(K, Pm, eigvals_only=True)
    return quad_nodes(1.0, 1.05 * lam[-1], Q), lam


@pytest.mark.parametrize("krylov", ["basis", "recurrence"])
@pytest.mark.parametrize("op,form", [("sqrt", "identity"), ("sqrt", "mvm"), ("invsqrt", "identity")])
def test_precond_fp32_solve_matches_oracle_at_equal_nodes_and_J(op, form, krylov):
    # The identity form of R b is P^{1/2} applied to the estimate of A^{1/2} b:
    # FP32 errors of the solve in the space of A reach the result scaled by up
    # to ||P^{1/2}||, so that form is compared where the solve runs, after
    # P^{-1/2} (FP64, both sides).  The printed form K (R' b) is compared
    # after K^{-1} (FP64, both sides), i.e. as the solve's R' b; its last MVM
    # is the kernel MVM checked on its own elsewhere.  R' b as it is.
    n, d, t, Q, J, rank = 900, 3, 5, 10, 300, 30
    X, B, Kxx, K, k = case(n, d, t, 71)
    L32, Lrows, _ = oracle_factor(Kxx, rank)
    pre = PC.Preconditioner(L32.astype(np.float64), k.noise)
    Pm = pre.dense()
    (w, tq), lam = _nodes_of_A(K, Pm, Q)
    lp, Vp = np.linalg.eigh(Pm)
    if op == "invsqrt":
        to_a = np.eye(n)
    elif form == "identity":
        to_a = (Vp * lp ** -0.5) @ Vp.T
    else:
        to_a = np.linalg.inv(K)
    run = lambda Km: PC.ciq_precond_apply(lambda V: Km @ V, pre, B.astype(np.float64), Q, op, max_iter=J,
                                          nodes=(w, tq), lmin=1.0, sqrt_form=form)[0] @ to_a
    ref, info_o = PC.ciq_precond_apply(lambda V: K @ V, pre, B.astype(np.float64), Q, op, max_iter=J,
                                       nodes=(w, tq), lmin=1.0, sqrt_form=form)
    assert np.max(info_o["errbound"]) < 1e-9 * np.linalg.norm(B, axis=1).min()       # converged
    fn = P.ciq_sqrt_precond if op == "sqrt" else P.ciq_invsqrt_precond
    out, info = fn(torch.from_numpy(X).cuda(), k, torch.from_numpy(B).cuda(), Q, 0.0, L=torch.from_numpy(Lrows).cuda(),
                   max_iter=J, nodes=(w, tq), lmin=1.0, krylov=krylov, sqrt_form=form)
    assert info["iters"] == J and info["krylov"] == krylov and info["precond_rank"] == rank
    tol, floor = fp32_gate(run, K, ref @ to_a)
    err = rel(out.cpu().numpy().astype(np.float64) @ to_a, ref @ to_a)
    assert err < tol, (err, tol, floor)


@pytest.mark.parametrize("op", ["sqrt", "invsqrt"])
def test_precond_device_prepass_bounds_and_host_factor(op):
    # Pre-pass on A on the device (lambda_min = 1), the factor passed as host
    # memory, the error-bound stop (tight, 1e-6, in the space of A): every
    # column within 1e-3 of the exact rotated root (O1 of the preconditioned
    # problem) and lambda_max used within the margin of the true one.
    n, d, t, rank = 1100, 4, 6, 50
    X, B, Kxx, K, k = case(n, d, t, 81, "rbf", ls=0.3, noise=1e-3)
    L32, Lrows, _ = oracle_factor(Kxx, rank)
    Pm = PC.Preconditioner(L32.astype(np.float64), k.noise).dense()
    Rb, Rpb = PC.rotated_roots_exact(K, Pm, B.astype(np.float64))
    lam = scipy.linalg.eigh(K, Pm, eigvals_only=True)
    fn = P.ciq_sqrt_precond if op == "sqrt" else P.ciq_invsqrt_precond
    out, info = fn(torch.from_numpy(X).cuda(), k, torch.from_numpy(B).cuda(), 12, 1e-6, L=Lrows, max_iter=2000,
                   stop_rule="errbound")
    assert info["status"] == 0 and info["lmin_used"] == 1.0
    assert lam[-1] <= info["lmax_used"] <= 1.06 * lam[-1]
    exact = Rb if op == "sqrt" else Rpb
    assert rel(out.cpu().numpy(), exact) < 1e-3


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_precond_with_the_device_factor_gives_a_root_of_K(prec):
    # The device's own factor: R R^T = K and R' R'^T = K^{-1}, checked on
    # all N columns of the identity (dense R), and R = K^{1/2} Omega with
    # Omega orthogonal -- properties that hold for whichever factor the
    # device chose.
    n, d, rank = 300, 3, 25
    X, _, Kxx, K, k = case(n, d, 1, 91, "rbf", ls=0.35, noise=1e-2)
    I = np.eye(n, dtype=np.float32)
    Xd, Id = torch.from_numpy(X).cuda(), torch.from_numpy(I).cuda()
    R, info = P.ciq_sqrt_precond(Xd, k, Id, 15, 1e-7, rank=rank, max_iter=2000, stop_rule="errbound",
                                 precision=prec)
    assert info["status"] == 0 and info["precond_rank"] == rank
    Rp, _ = P.ciq_invsqrt_precond(Xd, k, Id, 15, 1e-7, rank=rank, max_iter=2000, stop_rule="errbound",
                                  precision=prec)
    R = R.cpu().numpy().astype(np.float64).T            # column c = R e_c
    Rp = Rp.cpu().numpy().astype(np.float64).T
    tol = 2e-4 if prec == "fp32" else 2e-3
    assert np.linalg.norm(R @ R.T - K) / np.linalg.norm(K) < tol
    Kinv = np.linalg.inv(K)
    assert np.linalg.norm(Rp @ Rp.T - Kinv) / np.linalg.norm(Kinv) < tol
    Om = np.linalg.solve(np.real(scipy.linalg.sqrtm(K)), R)
    assert np.abs(Om.T @ Om - np.eye(n)).max() < 10 * tol


@pytest.mark.parametrize("op", ["sqrt", "invsqrt"])
def test_precond_fp16_tensor_core_matches_fp32(op):
    # Tensor-core split tiles under the preconditioner, 64 right-hand sides
    # and a ragged N, R b in the printed form K (R' b): the result agrees with
    # the FP32 path's within the tensor-core MVM's accuracy, and the solve
    # takes fewer iterations than the unpreconditioned K^{-1/2} b solve.
    n, d, t, rank = 3001, 6, 64, 100
    X, B, Kxx, K, k = case(n, d, t, 101, "rbf", ls=0.3, noise=1e-3)
    _, Lrows, _ = oracle_factor(Kxx, rank)
    Xd, Bd, Ld = torch.from_numpy(X).cuda(), torch.from_numpy(B).cuda(), torch.from_numpy(Lrows).cuda()
    fn = P.ciq_sqrt_precond if op == "sqrt" else P.ciq_invsqrt_precond
    kw = dict(stop_rule="errbound", max_iter=3000, sqrt_form="mvm")
    a32, i32 = fn(Xd, k, Bd, 12, 1e-5, L=Ld, precision="fp32", **kw)
    a16, i16 = fn(Xd, k, Bd, 12, 1e-5, L=Ld, precision="fp16", **kw)
    assert i32["status"] == 0 and i16["status"] == 0
    # K (R' b) multiplies R' b's error (FP16-split MVMs inside the solve) by K.
    assert rel(a16.cpu().numpy(), a32.cpu().numpy()) < (1e-3 if op == "invsqrt" else 2e-3)
    # Both preconditioned forms stop on R' b's rule: compare with K^{-1/2} b's solve.
    _, i0 = P.ciq_invsqrt(Xd, k, Bd, 12, 1e-5, precision="fp16", stop_rule="errbound", max_iter=3000)
    assert i16["iters"] < i0["iters"], (i16["iters"], i0["iters"])
