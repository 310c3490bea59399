"""Parity of the CUDA path against the FP64 oracle, through the C ABI.

Inputs are seeded (ciq_inputs) and rounded to FP32 before both sides see
them, so differences come from arithmetic only.  Every error is a relative
2-norm per right-hand side, gated on the largest (tests/relerr.py).
Tolerances:
  * FP32 kernel MVM: 2e-6 relative -- FP32 rounding of d-term
    distances, expf/sqrtf (<= 2 ulp) and compensated N-term sums;
  * FP32 solves vs the serial FP64 oracle at equal nodes and J, once both
    have converged: within 1e-5, or within 15 times the oracle's own change
    when K's entries are rounded to FP32 if that is larger (relerr.fp32_gate:
    at kappa ~ 1e4 the rounding of the entries alone moves K^{-1/2}b by 4e-6
    to 7e-6, so 1e-5 is out of reach of any FP32 kernel evaluation there;
    the GPU's FP32 path measured 9-11 times that floor);
  * FP64 solves: 1e-11 once converged.  Before convergence two correct FP64
    implementations differ by far more than rounding (finite-precision
    Lanczos is chaotic there: a 1e-16 change of K moves the J = 200 iterate
    of the 1024-point Matern problem by 1e-6), so the unconverged FP64
    case is compared through its error against the eigendecomposition.
"""
import numpy as np
import pytest
import torch

import ciq_inputs as ci
import paper_2006_11267_b300 as P
from oracle import ciq as O
from oracle import eig, kernels
from oracle.lanczos import lanczos, ritz_extremes
from relerr import colrel, fp32_gate, rel

pytestmark = pytest.mark.gpu

DEV = "cuda"


def f32(a):
    return np.asarray(a, dtype=np.float32)


def problem(n, d, t, seed, kind="matern52", ls=0.2, s=1.0, noise=1e-2):
    X = f32(ci.points(seed, n, d))
    B = f32(ci.rhs(seed, n, t))
    return X, B, P.Kernel(kind, ls, s, noise)


def dense_K(X, k):
    return kernels.dense_K(X.astype(np.float64), k.type, k.lengthscale, k.outputscale, k.noise)


# --------------------------------------------------------------------- MVM ----
@pytest.mark.parametrize("kind", ["rbf", "matern52"])
@pytest.mark.parametrize("n,d,t", [(1, 1, 1), (129, 3, 1), (1000, 6, 3), (777, 12, 8), (1000, 16, 17),
                                   (1300, 4, 64), (900, 2, 70)])
def test_kernel_mvm_fp32_matches_oracle(kind, n, d, t):
    X, V, k = problem(n, d, t, 100 + n + d + t, kind, ls=0.3, s=1.3, noise=1e-3)
    out = P.ciq_kernel_mvm(torch.from_numpy(X).to(DEV), k, torch.from_numpy(V).to(DEV))
    ref = dense_K(X, k) @ V.T.astype(np.float64)
    assert rel(out.cpu().numpy(), ref.T) < 2e-6


@pytest.mark.parametrize("kind", ["rbf", "matern52"])
def test_kernel_mvm_fp64_matches_oracle(kind):
    X, V, k = problem(700, 5, 2, 7, kind)
    X = X.astype(np.float64)
    V = V.astype(np.float64)
    out = P.ciq_kernel_mvm_f64(torch.from_numpy(X).to(DEV), k, torch.from_numpy(V).to(DEV))
    ref = dense_K(X, k) @ V.T
    assert rel(out.cpu().numpy(), ref.T) < 1e-13


# ------------------------------------------------------------ pre-pass ----
def test_lanczos_bounds_match_oracle_and_device_start_vector():
    X, _, k = problem(1500, 3, 1, 11)
    start = f32(ci.start_vector(77, 1500))
    Xd = torch.from_numpy(X).to(DEV)
    b1 = P.ciq_lanczos_bounds(Xd, k, iters=10, start=torch.from_numpy(start).to(DEV))
    b2 = P.ciq_lanczos_bounds(Xd, k, iters=10, seed=77)            # drawn on the device
    assert b1 == b2                                                  # same generator, bit for bit
    K = dense_K(X, k)
    a, bt = lanczos(lambda v: K @ v, start.astype(np.float64), 10)
    tmin, tmax = ritz_extremes(a, bt)
    assert abs(b1["ritz_max"] - tmax) / tmax < 1e-5
    assert abs(b1["ritz_min"] - tmin) / tmin < 1e-3
    assert b1["lmin_used"] == k.noise
    assert abs(b1["lmax_used"] - 1.05 * b1["ritz_max"]) < 1e-12 * b1["lmax_used"]


# -------------------------------------------------------------- solves ----
def _oracle(op, X, k, B, Q, J, nodes, tol=0.0, stop_rule="residual"):
    K = dense_K(X, k)
    return O.ciq_apply(O.dense_mvm(K), B.astype(np.float64), Q, op, tol=tol, max_iter=J,
                       stop_rule=stop_rule, nodes=nodes, lmin=k.noise, lmax=None)


def fp32_tol(op, K, ref, run, factor=15.0):
    """1e-5, or `factor` times the change that rounding K's entries to FP32
    alone makes to the oracle's result when that is larger (relerr.fp32_gate)."""
    return fp32_gate(run, K, ref, factor=factor)


@pytest.mark.parametrize("krylov", ["recurrence", "basis"])
@pytest.mark.parametrize("op", ["sqrt", "invsqrt"])
@pytest.mark.parametrize("kind,n,d,t,Q,J", [("matern52", 777, 3, 3, 8, 800), ("rbf", 1025, 6, 17, 12, 600),
                                             ("matern52", 300, 2, 64, 15, 600), ("rbf", 2000, 4, 8, 10, 900)])
def test_fp32_solve_matches_serial_oracle_at_equal_nodes_and_J(op, kind, n, d, t, Q, J, krylov):
    X, B, k = problem(n, d, t, 200 + n, kind, ls=0.25)
    K = dense_K(X, k)
    lam = np.linalg.eigvalsh(K)
    nodes = O.quad_nodes(k.noise, 1.05 * lam[-1], Q)
    ref, info_o = _oracle(op, X, k, B, Q, J, nodes)
    assert np.max(info_o["errbound"] / np.linalg.norm(ref, axis=1)) < 1e-9      # oracle converged
    fn = P.ciq_sqrt if op == "sqrt" else P.ciq_invsqrt
    out, info = fn(torch.from_numpy(X).to(DEV), k, torch.from_numpy(B).to(DEV), Q, 0.0,
                   max_iter=J, nodes=nodes, lmin=k.noise, krylov=krylov)
    assert info["iters"] == J and info["krylov"] == krylov
    # Both forms keep the Lanczos p as a float pair (measured 6-10x the floor
    # for K^{-1/2}b in either, against 9-11x with FP32 p); the recurrence's
    # identity-form K^{1/2}b adds its FP32 direction updates (9-14x): 12x for
    # the stored basis and 15x for the recurrence.
    tol, floor = fp32_tol(op, K, ref, lambda Km: O.ciq_apply(O.dense_mvm(Km), B.astype(np.float64), Q, op,
                                                             max_iter=J, nodes=nodes, lmin=k.noise)[0],
                          factor=12.0 if krylov == "basis" else 15.0)
    err = rel(out.cpu().numpy(), ref)
    assert err < tol, (err, tol, floor)


@pytest.mark.parametrize("op,form", [("sqrt", "identity"), ("sqrt", "mvm"), ("invsqrt", "identity")])
def test_basis_errbound_stop_matches_oracle_scalar_norm_rule(op, form):
    # The stored-basis error-bound rule (||b|| sqrt(alpha_1), Gauss rule) at equal
    # nodes: the true error stays <= tol, the result agrees with the oracle's
    # errbound_norm="scalar" run, and the stop comes within a few steps of the
    # direction recurrence's (same FP32 Lanczos; FP32 needs more steps than the
    # FP64 oracle, whose stop is therefore not compared).
    X, B, k = problem(1500, 3, 8, 31, "matern52", ls=0.25)
    K = dense_K(X, k)
    lam = np.linalg.eigvalsh(K)
    nodes = O.quad_nodes(k.noise, 1.05 * lam[-1], 12)
    tol = 1e-4
    ref, info_o = O.ciq_apply(O.dense_mvm(K), B.astype(np.float64), 12, op, tol=tol, max_iter=1500,
                              stop_rule="errbound", nodes=nodes, lmin=k.noise, lmax=1.05 * lam[-1],
                              sqrt_form=form, errbound_norm="scalar")
    fn = P.ciq_sqrt if op == "sqrt" else P.ciq_invsqrt
    out, info = fn(torch.from_numpy(X).to(DEV), k, torch.from_numpy(B).to(DEV), 12, tol, max_iter=1500,
                   nodes=nodes, lmin=k.noise, lmax=1.05 * lam[-1], stop_rule="errbound", sqrt_form=form)
    assert info["status"] == 0 and info["krylov"] == "basis"              # the default for FP32
    if form == "identity":                 # the MVM form's recurrence rule is on y, not on K y
        _, info_r = fn(torch.from_numpy(X).to(DEV), k, torch.from_numpy(B).to(DEV), 12, tol, max_iter=1500,
                       nodes=nodes, lmin=k.noise, lmax=1.05 * lam[-1], stop_rule="errbound",
                       krylov="recurrence")
        assert abs(info["iters"] - info_r["iters"]) <= max(3, int(0.02 * info["iters"]))
    exact = (eig.sqrt_apply if op == "sqrt" else eig.invsqrt_apply)(K, B.T.astype(np.float64)).T
    err = np.linalg.norm(out.cpu().numpy() - exact, axis=1) / np.linalg.norm(exact, axis=1)
    assert err.max() <= 1.05 * tol
    assert rel(out.cpu().numpy(), ref) < 10 * tol


@pytest.mark.parametrize("op", ["sqrt", "invsqrt"])
def test_fp64_solve_matches_serial_oracle_converged(op):
    X, B, k = problem(1024, 3, 2, 20201106)
    X64, B64 = X.astype(np.float64), B.astype(np.float64)
    start = ci.start_vector(5, 1024)
    K = dense_K(X64, k)
    ref, info_o = O.ciq_apply(O.dense_mvm(K), B64, 8, op, tol=0.0, max_iter=800, noise=k.noise,
                              start=start)
    fn = P.ciq_sqrt_f64 if op == "sqrt" else P.ciq_invsqrt_f64
    out, info = fn(torch.from_numpy(X64).to(DEV), k, torch.from_numpy(B64).to(DEV), 8, 0.0,
                   max_iter=800, lanczos_start=torch.from_numpy(start).to(DEV))
    assert abs(info["ritz_max"] - info_o["ritz_max"]) < 1e-10 * info_o["ritz_max"]
    assert abs(info["ritz_min"] - info_o["ritz_min"]) < 1e-8 * info_o["ritz_min"]
    np.testing.assert_allclose(info["w"], info_o["w"], rtol=1e-10)
    np.testing.assert_allclose(info["t"], info_o["t"], rtol=1e-10)
    assert rel(out.cpu().numpy(), ref) < 1e-11


@pytest.mark.parametrize("op", ["sqrt", "invsqrt"])
def test_fp64_plain_msminres_ciq_1024_point_matern(op):
    # N = 1024 in [0,1]^3, Matern-5/2, l = 0.2, s = 1, sigma^2 = 1e-2, one RHS,
    # Q = 8, relative residual 1e-6 capped at 200 iterations (the cap binds).
    X, B, k = problem(1024, 3, 1, 20201106)
    X64, B64 = X.astype(np.float64), B.astype(np.float64)
    start = ci.start_vector(5, 1024)
    K = dense_K(X64, k)
    truth = (eig.sqrt_apply if op == "sqrt" else eig.invsqrt_apply)(K, B64.T).T
    ref, info_o = O.ciq_apply(O.dense_mvm(K), B64, 8, op, tol=1e-6, max_iter=200, noise=k.noise,
                              start=start)
    fn = P.ciq_sqrt_f64 if op == "sqrt" else P.ciq_invsqrt_f64
    out, info = fn(torch.from_numpy(X64).to(DEV), k, torch.from_numpy(B64).to(DEV), 8, 1e-6,
                   max_iter=200, lanczos_start=torch.from_numpy(start).to(DEV))
    assert info["iters"] == int(info_o["iters"][0]) == 200
    assert info["status"] == 4                                  # the cap binds, as in the oracle
    e_gpu, e_orc = rel(out.cpu().numpy(), truth), rel(ref, truth)
    # Unconverged: both are equally far from the truth, not bitwise equal.
    assert abs(e_gpu - e_orc) <= 0.25 * e_orc
    r_orc = np.max(np.abs(info_o["phibar"])) / np.linalg.norm(B64)
    assert abs(info["resid_max"] - r_orc) <= 0.25 * r_orc and min(info["resid_max"], r_orc) > 1e-6


@pytest.mark.parametrize("op", ["sqrt", "invsqrt"])
def test_fp32_against_eig_oracle_q15(op):
    X, B, k = problem(1024, 3, 2, 20201106)
    K = dense_K(X, k)
    ref = (eig.sqrt_apply if op == "sqrt" else eig.invsqrt_apply)(K, B.T.astype(np.float64)).T
    fn = P.ciq_sqrt if op == "sqrt" else P.ciq_invsqrt
    out, info = fn(torch.from_numpy(X).to(DEV), k, torch.from_numpy(B).to(DEV), 15, 1e-4, max_iter=1000)
    assert info["status"] == 0
    assert rel(out.cpu().numpy(), ref) < 1e-3


def test_host_buffers_equal_device_buffers():
    X, B, k = problem(600, 4, 5, 31, "rbf", ls=0.4)
    o_dev, i_dev = P.ciq_invsqrt(torch.from_numpy(X).to(DEV), k, torch.from_numpy(B).to(DEV), 8, 1e-5,
                                 max_iter=300, seed=3)
    o_host, i_host = P.ciq_invsqrt(X, k, B, 8, 1e-5, max_iter=300, seed=3)
    assert isinstance(o_host, np.ndarray)
    np.testing.assert_array_equal(o_dev.cpu().numpy(), o_host)
    assert i_dev["iters"] == i_host["iters"]


def test_sqrt_forms_agree():
    X, B, k = problem(800, 3, 4, 41)
    Xd, Bd = torch.from_numpy(X).to(DEV), torch.from_numpy(B).to(DEV)
    a1, _ = P.ciq_sqrt(Xd, k, Bd, 12, 1e-6, max_iter=600, sqrt_form="identity")
    a2, _ = P.ciq_sqrt(Xd, k, Bd, 12, 1e-6, max_iter=600, sqrt_form="mvm")
    assert rel(a1.cpu().numpy(), a2.cpu().numpy()) < 1e-4


def test_edge_cases_tiny_sizes_zero_column_and_duplicates():
    k = P.Kernel("rbf", 0.5, 1.0, 0.1)
    # N = 1: K = s + sigma^2, exact after one step.
    X = f32([[0.3, 0.7]])
    B = f32([[2.0], [-1.0]])
    out, info = P.ciq_invsqrt(torch.from_numpy(X).to(DEV), k, torch.from_numpy(B).to(DEV), 8, 1e-6)
    np.testing.assert_allclose(out.cpu().numpy(), B / np.sqrt(1.1), rtol=1e-5)
    # Zero right-hand side gives zero; duplicate points keep K SPD through sigma^2.
    X = f32(np.repeat(ci.points(3, 50, 2), 2, axis=0))
    B = f32(ci.rhs(4, 100, 3))
    B[1] = 0.0
    out, info = P.ciq_sqrt(torch.from_numpy(X).to(DEV), k, torch.from_numpy(B).to(DEV), 10, 1e-6, max_iter=400)
    o = out.cpu().numpy()
    assert np.all(o[1] == 0.0)
    ref = eig.sqrt_apply(dense_K(X, k), B.T.astype(np.float64)).T
    assert rel(o, ref) < 1e-4
    # Ragged sizes around the 128-row padding.
    for n in [2, 127, 129, 255]:
        X, B, kk = problem(n, 3, 2, n)
        out, info = P.ciq_invsqrt(torch.from_numpy(X).to(DEV), kk, torch.from_numpy(B).to(DEV), 8, 1e-7,
                                  max_iter=600)
        ref = eig.invsqrt_apply(dense_K(X, kk), B.T.astype(np.float64)).T
        assert rel(out.cpu().numpy(), ref) < 2e-4, n


def test_stop_rules_report_and_iteration_cap():
    X, B, k = problem(900, 3, 4, 51)
    Xd, Bd = torch.from_numpy(X).to(DEV), torch.from_numpy(B).to(DEV)
    _, info = P.ciq_sqrt(Xd, k, Bd, 8, 1e-12, max_iter=5)
    assert info["status"] == 4 and info["iters"] == 5                 # not converged, capped
    _, info = P.ciq_sqrt(Xd, k, Bd, 8, 1e-3, max_iter=500, stop_rule="errbound")
    assert info["status"] == 0 and info["errbound_max"] <= 1e-3
    _, info = P.ciq_sqrt(Xd, k, Bd, 8, 1e-4, max_iter=500, stop_rule="residual")
    assert info["status"] == 0 and info["resid_max"] <= 1e-4


# ------------------------------------------------------------ stored K ----
def _npad(n):
    return (n + 127) // 128 * 128


@pytest.mark.parametrize("kind", ["rbf", "matern52"])
def test_kernel_matrix_matches_oracle_with_zero_padding(kind):
    n, d = 300, 5
    X, _, k = problem(n, d, 1, 61, kind, ls=0.3, s=1.7, noise=2e-3)
    npad = _npad(n)
    Kd = torch.full((npad, npad + 4), float("nan"), device=DEV)
    P.ciq_kernel_matrix(torch.from_numpy(X).to(DEV), k, Kd)
    Km = Kd.cpu().numpy().astype(np.float64)
    ref = dense_K(X, k)
    assert rel(Km[:n, :n], ref) < 3e-7                   # per row of K
    assert np.all(Km[n:npad, :npad] == 0) and np.all(Km[:npad, n:npad] == 0)


@pytest.mark.parametrize("n,t", [(1, 1), (300, 1), (777, 5), (1000, 17), (1300, 64), (513, 70)])
def test_stored_mvm_matches_oracle(n, t):
    X, V, k = problem(n, 4, t, 70 + n + t, "rbf", ls=0.3, s=1.3, noise=1e-3)
    npad = _npad(n)
    Kd = torch.empty((npad, npad), device=DEV)
    P.ciq_kernel_matrix(torch.from_numpy(X).to(DEV), k, Kd)
    out = P.ciq_stored_mvm(Kd, torch.from_numpy(V).to(DEV), n=n)
    ref = dense_K(X, k) @ V.T.astype(np.float64)
    assert rel(out.cpu().numpy(), ref.T) < 2e-6


@pytest.mark.parametrize("prec,tol", [("fp16", 2e-5), ("bf16", 1e-4)])
@pytest.mark.parametrize("n,t", [(1, 1), (300, 8), (777, 5), (1000, 17), (3001, 64), (513, 70), (2000, 128)])
def test_stored_mvm_tensor_cores_matches_oracle(prec, tol, n, t):
    # K streamed by TMA (ragged edges are the stored matrix's zero padding),
    # scaled by a power of two and split into two 16-bit parts, as is V:
    # per column the FP16 split keeps about 22 significant bits (the on-the-fly
    # tensor-core MVM's 2e-5 gate), BF16 about 16 (1e-4).
    X, V, k = problem(n, 4, t, 170 + n + t, "rbf", ls=0.3, s=1.3, noise=1e-3)
    npad = _npad(n)
    Kd = torch.empty((npad, npad), device=DEV)
    P.ciq_kernel_matrix(torch.from_numpy(X).to(DEV), k, Kd)
    out = P.ciq_stored_mvm(Kd, torch.from_numpy(V).to(DEV), n=n, precision=prec)
    ref = dense_K(X, k) @ V.T.astype(np.float64)
    assert rel(out.cpu().numpy(), ref.T) < tol


def test_stored_mvm_tensor_cores_general_psd_matrix_and_pitch():
    # A caller's positive definite matrix with a prescribed spectrum (not a
    # kernel matrix: entries of both signs, diagonal far from 1) in a pitched
    # layout (ldk > Npad): the scale taken from the diagonal keeps every
    # entry in range.
    n, t = 1500, 24
    rng = np.random.default_rng(5)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1e-2, 3e3, n)
    K = (Qm * lam) @ Qm.T
    npad = _npad(n)
    Kp = np.zeros((npad, npad + 8), np.float32)
    Kp[:n, :n] = K
    V = rng.standard_normal((t, n)).astype(np.float32)
    out = P.ciq_stored_mvm(torch.from_numpy(Kp).to(DEV), torch.from_numpy(V).to(DEV), n=n, precision="fp16")
    K32 = K.astype(np.float32).astype(np.float64)
    V64 = V.T.astype(np.float64)
    ref = K32 @ V64
    # Each split entry is within 2^-22 of the FP32 value and the three
    # products are exact in FP32: per column the error is a few 2^-22
    # || |K| |V| || (entries of both signs cancel in K V) plus the FP32
    # accumulation (about 1e-6 of the result, folded every 1,536 columns).
    bound = 8 * 2.0 ** -22 * np.linalg.norm(np.abs(K32) @ np.abs(V64), axis=0) / np.linalg.norm(ref, axis=0) + 2e-6
    err = colrel(out.cpu().numpy(), ref.T)
    assert np.all(err < bound), (err.max(), bound.min())


@pytest.mark.parametrize("op", ["sqrt", "invsqrt"])
def test_stored_k_tensor_core_solve_matches_on_the_fly_tensor_core_solve(op):
    # The same FP16-split arithmetic on K's entries either way (stored K is
    # formed with the accurate exponential, the on-the-fly tile from the
    # split distances): both solves agree within the FP16-split MVM error.
    X, B, k = problem(2500, 3, 16, 991, "matern52", ls=0.25)
    fn = P.ciq_sqrt if op == "sqrt" else P.ciq_invsqrt
    Xd, Bd = torch.from_numpy(X).to(DEV), torch.from_numpy(B).to(DEV)
    a, ia = fn(Xd, k, Bd, 10, 1e-6, max_iter=1500, precision="fp16", mvm="stored", stop_rule="errbound")
    b, ib = fn(Xd, k, Bd, 10, 1e-6, max_iter=1500, precision="fp16", stop_rule="errbound")
    assert ia["status"] == 0 and ib["status"] == 0
    # Both are within the FP16-split mode's 1e-3 of the exact root; their
    # MVMs differ by a few 1e-6 (accurate expf against ex2.approx of the
    # split distances), amplified by the root's conditioning.
    assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-3


@pytest.mark.parametrize("op", ["sqrt", "invsqrt"])
def test_stored_k_solve_matches_serial_oracle(op):
    X, B, k = problem(777, 3, 3, 977, "matern52", ls=0.25)
    K = dense_K(X, k)
    lam = np.linalg.eigvalsh(K)
    nodes = O.quad_nodes(k.noise, 1.05 * lam[-1], 8)
    ref, _ = _oracle(op, X, k, B, 8, 800, nodes)
    fn = P.ciq_sqrt if op == "sqrt" else P.ciq_invsqrt
    out, info = fn(torch.from_numpy(X).to(DEV), k, torch.from_numpy(B).to(DEV), 8, 0.0, max_iter=800,
                   nodes=nodes, lmin=k.noise, mvm="stored")
    assert info["iters"] == 800
    tol, floor = fp32_tol(op, K, ref, lambda Km: O.ciq_apply(O.dense_mvm(Km), B.astype(np.float64), 8, op,
                                                             max_iter=800, nodes=nodes, lmin=k.noise)[0])
    err = rel(out.cpu().numpy(), ref)
    assert err < tol, (err, tol, floor)
