"""Tensor-core (tcgen05) MVM and solves against the FP64 oracle, through the C ABI.

Precision modes split every 16-bit operand into a leading and a trailing part
(three products: hi*hi + hi*lo + lo*hi).  With FP16 parts that keeps about 22
significant bits; with BF16 parts 16 bits, which the norm expansion of the
distance (terms of size |x/l|^2 that cancel) turns into larger absolute
errors for small lengthscales.  The tensor core accumulates in FP32 with a
bias that grows with the number of accumulation steps, so O is accumulated in
chunks of 1,024 points and folded into a compensated sum; the 50,000-point
check below guards that.

Tolerances (relative, Frobenius): FP16 MVM 2e-5 (measured 2-7e-6); BF16 MVM
1e-4 at lengthscale >= 0.2 (measured 1-3e-5); FP16 solves against the
eigendecomposition 1e-3, the accuracy target of the mixed-precision mode.
"""
import numpy as np
import pytest
import torch

import ciq_inputs as ci
import paper_2006_11267_b300 as P
from oracle import eig, kernels
from relerr import colrel, rel

pytestmark = pytest.mark.gpu


def f32(a):
    return np.asarray(a, dtype=np.float32)


@pytest.mark.parametrize("prec,tol", [("fp16", 2e-5), ("bf16", 1e-4)])
@pytest.mark.parametrize("n,d,t,kind,ls", [(1000, 3, 8, "rbf", 0.3), (1000, 3, 16, "matern52", 0.3),
                                           (1300, 6, 64, "rbf", 0.3), (2000, 12, 33, "matern52", 0.5),
                                           (777, 2, 128, "rbf", 0.2), (5000, 6, 200, "rbf", 0.3),
                                           (513, 5, 256, "matern52", 0.25), (129, 14, 1, "rbf", 1.0)])
def test_tc_mvm_matches_oracle(prec, tol, n, d, t, kind, ls):
    X = f32(ci.points(n + d, n, d))
    V = f32(ci.rhs(n + t, n, t))
    k = P.Kernel(kind, ls, 1.3, 1e-3)
    ref = kernels.dense_K(X.astype(np.float64), kind, ls, 1.3, 1e-3) @ V.T.astype(np.float64)
    out = P.ciq_kernel_mvm(torch.from_numpy(X).cuda(), k, torch.from_numpy(V).cuda(), precision=prec)
    assert rel(out.cpu().numpy(), ref.T) < tol


@pytest.mark.parametrize("n,d,t,kind,ls", [(1000, 3, 8, "rbf", 0.3), (1300, 6, 64, "rbf", 0.3),
                                           (2000, 12, 33, "matern52", 0.5), (3001, 6, 100, "matern52", 0.2),
                                           (129, 14, 1, "rbf", 1.0)])
def test_tc_mvm_tf32_matches_oracle_within_the_rounding_bound(n, d, t, kind, ls):
    # TF32 tiles: P and V rounded to TF32 (unit roundoff u = 2^-11), one
    # product, FP32 accumulation.  Each term P_ij V_j carries a relative error
    # of at most 2u + u^2, so row i of O is off by at most 2^-10 sum_j |K_ij| |V_j|
    # (the sigma^2 V term is added unrounded): per column, ||err|| <= 2^-10
    # || |K| |V| ||.  The distance tile (FP16 split, ~22 bits) and the FP32
    # accumulation add about 1e-5 (the FP16-split mode's gate).
    X = f32(ci.points(n + d + 7, n, d))
    V = f32(ci.rhs(n + t + 7, n, t))
    k = P.Kernel(kind, ls, 1.3, 1e-3)
    K = kernels.dense_K(X.astype(np.float64), kind, ls, 1.3, 1e-3)
    V64 = V.T.astype(np.float64)
    ref = K @ V64
    bound = 2.0 ** -10 * np.linalg.norm(np.abs(K) @ np.abs(V64), axis=0) / np.linalg.norm(ref, axis=0) + 1e-5
    out = P.ciq_kernel_mvm(torch.from_numpy(X).cuda(), k, torch.from_numpy(V).cuda(), precision="tf32")
    err = colrel(out.cpu().numpy(), ref.T)
    assert np.all(err < bound), (err.max(), bound.min())
    # TF32 is coarser than the FP16 split but far from noise: the error is
    # at least a few times the FP16-split mode's.
    assert err.max() > 1e-5


def test_tc_mvm_fp16_small_lengthscale():
    X = f32(ci.points(9, 900, 4))
    V = f32(ci.rhs(10, 900, 17))
    k = P.Kernel("matern52", 0.1, 1.0, 1e-2)
    ref = kernels.dense_K(X.astype(np.float64), "matern52", 0.1, 1.0, 1e-2) @ V.T.astype(np.float64)
    out = P.ciq_kernel_mvm(torch.from_numpy(X).cuda(), k, torch.from_numpy(V).cuda(), precision="fp16")
    assert rel(out.cpu().numpy(), ref.T) < 2e-5


def test_tc_mvm_accumulation_at_50k_points_sampled_rows():
    W = ci.THOMPSON_50K
    X = f32(ci.points(W.seed, W.n, W.d))
    V = f32(ci.rhs(W.seed, W.n, W.t))
    k = P.Kernel(W.kernel, W.lengthscale, W.outputscale, W.noise)
    out = P.ciq_kernel_mvm(torch.from_numpy(X).cuda(), k, torch.from_numpy(V).cuda(), precision="fp16")
    rows = np.concatenate([np.arange(0, 64), np.arange(W.n - 64, W.n), np.arange(20000, 20128)])
    Kr = kernels.kernel_matrix(X[rows].astype(np.float64), X.astype(np.float64), W.kernel, W.lengthscale,
                               W.outputscale)
    ref = Kr @ V.T.astype(np.float64) + W.noise * V.T[rows].astype(np.float64)
    assert rel(out.cpu().numpy()[:, rows], ref.T) < 2e-5


@pytest.mark.parametrize("t", [8, 64])
def test_stored_tc_mvm_at_50k_points_sampled_rows(t):
    # The bench's stored-K workload at full size (K of 10 GB formed once,
    # the tensor-core MVM in its timed launch shape: 391 row tiles x 3
    # splits): sampled rows (first, last and middle row tiles) against the
    # FP64 oracle, per column within the FP16-split mode's 2e-5.
    W = ci.THOMPSON_50K
    X = f32(ci.points(W.seed, W.n, W.d))
    V = f32(ci.rhs(W.seed + 3, W.n, t))
    k = P.Kernel(W.kernel, W.lengthscale, W.outputscale, W.noise)
    npad = -(-W.n // 128) * 128
    K = torch.empty((npad, npad), dtype=torch.float32, device="cuda")
    P.ciq_kernel_matrix(torch.from_numpy(X).cuda(), k, K)
    out = P.ciq_stored_mvm(K, torch.from_numpy(V).cuda(), n=W.n, precision="fp16")
    del K
    torch.cuda.empty_cache()
    rows = np.concatenate([np.arange(0, 64), np.arange(W.n - 64, W.n), np.arange(20000, 20128)])
    Kr = kernels.kernel_matrix(X[rows].astype(np.float64), X.astype(np.float64), W.kernel, W.lengthscale,
                               W.outputscale)
    ref = Kr @ V.T.astype(np.float64) + W.noise * V.T[rows].astype(np.float64)
    assert rel(out.cpu().numpy()[:, rows], ref.T) < 2e-5


@pytest.mark.parametrize("krylov", ["recurrence", "basis"])
@pytest.mark.parametrize("op", ["sqrt", "invsqrt"])
def test_tc_fp16_solve_against_eig_oracle(op, krylov):
    X = f32(ci.points(20201106, 2048, 3))
    B = f32(ci.rhs(20201106, 2048, 40))
    k = P.Kernel("matern52", 0.2, 1.0, 1e-2)
    K = kernels.dense_K(X.astype(np.float64), "matern52", 0.2, 1.0, 1e-2)
    ref = (eig.sqrt_apply if op == "sqrt" else eig.invsqrt_apply)(K, B.T.astype(np.float64)).T
    fn = P.ciq_sqrt if op == "sqrt" else P.ciq_invsqrt
    out, info = fn(torch.from_numpy(X).cuda(), k, torch.from_numpy(B).cuda(), 15, 1e-4, stop_rule="errbound",
                   max_iter=2000, precision="fp16", krylov=krylov)
    assert info["status"] == 0 and info["krylov"] == krylov
    err = np.linalg.norm(out.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() < 1e-3


def test_tc_fp16_full_size_square_root_property():
    # K^{1/2}(K^{1/2} b) = K b on the 50,000-point RBF workload (error bound 1e-3 per solve).
    W = ci.THOMPSON_50K
    X = torch.from_numpy(f32(ci.points(W.seed, W.n, W.d))).cuda()
    B = torch.from_numpy(f32(ci.rhs(W.seed, W.n, W.t))).cuda()
    k = P.Kernel(W.kernel, W.lengthscale, W.outputscale, W.noise)
    A, info = P.ciq_sqrt(X, k, B, W.q, 1e-3, stop_rule="errbound", max_iter=4000, precision="fp16")
    assert info["status"] == 0 and info["krylov"] == "basis"          # the stored basis (47.7 GiB) by default
    A2, _ = P.ciq_sqrt(X, k, A[:4].contiguous(), W.q, 1e-4, stop_rule="errbound", max_iter=4000, precision="fp16")
    KB = P.ciq_kernel_mvm(X, k, B[:4].contiguous(), precision="fp32")
    e = (torch.linalg.norm(A2 - KB, dim=1) / torch.linalg.norm(KB, dim=1)).cpu().numpy()
    assert e.max() < 3e-4
    # The same property against the FP64 oracle's K b on sampled rows (first,
    # middle and last row tiles), computed entry by entry on the host.
    rows = np.concatenate([np.arange(0, 64), np.arange(20000, 20128), np.arange(W.n - 64, W.n)])
    Xh = X.cpu().numpy().astype(np.float64)
    Bh = B[:4].cpu().numpy().astype(np.float64)
    Kr = kernels.kernel_matrix(Xh[rows], Xh, W.kernel, W.lengthscale, W.outputscale)
    ref = Kr @ Bh.T + W.noise * Bh.T[rows]                     # (rows, 4)
    got = A2.cpu().numpy().astype(np.float64)[:, rows].T
    e = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert e.max() < 3e-4, e.max()


def test_tc_split_k_changes_only_the_summation_order():
    # Splitting a row tile's 128-column steps over S CTAs adds S float-pair
    # partial sums in split order: only rounding changes, so each split is
    # reproducible bit for bit (deterministic centre, fixed order) and the
    # solves agree within the accuracy the stop rule leaves (relative
    # residual 1e-4: measured differences ~1e-4 between splits).
    X = torch.from_numpy(f32(ci.points(11, 9000, 5))).cuda()
    V = torch.from_numpy(f32(ci.rhs(12, 9000, 40))).cuda()
    k = P.Kernel("rbf", 0.4, 1.0, 1e-2)
    outs = {}
    for s in (1, 2, 5, 8):
        X2, V2 = X.clone(), V.clone()
        a = P.ciq_sqrt(X2, k, V2, 8, 1e-4, max_iter=600, precision="fp16", tc_split=s)[0]
        b = P.ciq_sqrt(X2, k, V2, 8, 1e-4, max_iter=600, precision="fp16", tc_split=s)[0]
        assert torch.equal(a, b), s
        outs[s] = a.cpu().numpy()
    for s in (2, 5, 8):
        assert rel(outs[s], outs[1]) < 1e-3, s


def test_tc_bounded_wait_runs_out_and_the_host_reads_the_status():
    # Failure detection without a fault: with fault_inject = 1, CTA 0 of the
    # first tensor-core MVM never receives its first point tile, so its
    # bounded waits (about 2 s) run out; the kernel records the error,
    # frees its tensor memory and returns, later MVMs of the call do no
    # work, and the call returns CIQ_ERR_TIMEOUT.  The device stays usable:
    # the same solve right after is correct.
    X = torch.from_numpy(f32(ci.points(31, 700, 3))).cuda()
    B = torch.from_numpy(f32(ci.rhs(32, 700, 4))).cuda()
    k = P.Kernel("rbf", 0.3, 1.0, 1e-2)
    with pytest.raises(P.CiqError) as e:
        P.ciq_sqrt(X, k, B, 8, 1e-4, max_iter=50, precision="fp16", fault_inject=1)
    assert e.value.status == P._ciq.CIQ_ERR_TIMEOUT
    probs = [dict(X=X, B=B, kernel=k), dict(X=X[:300].contiguous(), B=B[:, :300].contiguous(), kernel=k)]
    with pytest.raises(P.CiqError) as e:
        P.ciq_sqrt_batched(probs, 8, 1e-4, max_iter=50, precision="fp16", fault_inject=1)
    assert e.value.status == P._ciq.CIQ_ERR_TIMEOUT
    out, info = P.ciq_sqrt(X, k, B, 8, 1e-4, max_iter=500, precision="fp16")
    assert info["status"] == 0
    K = kernels.dense_K(X.cpu().numpy().astype(np.float64), "rbf", 0.3, 1.0, 1e-2)
    truth = eig.sqrt_apply(K, B.cpu().numpy().astype(np.float64).T).T
    assert rel(out.cpu().numpy(), truth) < 1e-3


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_nan_in_the_points_is_reported(prec):
    # A non-finite point makes a row and a column of K non-finite; the first
    # Lanczos coefficients are then NaN and the solve reports CIQ_ERR_NAN
    # (per column: status NaN) instead of returning numbers.
    X = f32(ci.points(41, 500, 3))
    X[17, 1] = np.nan
    Xd = torch.from_numpy(X).cuda()
    B = torch.from_numpy(f32(ci.rhs(42, 500, 4))).cuda()
    k = P.Kernel("rbf", 0.3, 1.0, 1e-2)
    with pytest.raises(P.CiqError) as e:
        P.ciq_sqrt(Xd, k, B, 8, 1e-4, max_iter=100, precision=prec, lmin=1e-2, lmax=400.0)
    assert e.value.status == P._ciq.CIQ_ERR_NAN


def test_basis_and_recurrence_forms_agree_at_full_size():
    # The 50,000-point workload in the bench's configuration: the stored-basis
    # form and the direction recurrence stop within a few steps of each other
    # (their error-bound denominators differ, R15) and agree to the 1e-3 target.
    W = ci.THOMPSON_50K
    X = torch.from_numpy(f32(ci.points(W.seed, W.n, W.d))).cuda()
    B = torch.from_numpy(f32(ci.rhs(W.seed, W.n, 16))).cuda()
    k = P.Kernel(W.kernel, W.lengthscale, W.outputscale, W.noise)
    outs, infos = {}, {}
    for form in ("basis", "recurrence"):
        outs[form], infos[form] = P.ciq_sqrt(X, k, B, W.q, 1e-3, stop_rule="errbound", max_iter=4000,
                                             precision="fp16", krylov=form)
        assert infos[form]["status"] == 0 and infos[form]["krylov"] == form
        assert infos[form]["errbound_max"] <= 1e-3
    assert abs(infos["basis"]["iters"] - infos["recurrence"]["iters"]) <= 0.02 * infos["recurrence"]["iters"]
    d = torch.linalg.norm(outs["basis"] - outs["recurrence"], dim=1) / torch.linalg.norm(outs["recurrence"], dim=1)
    assert d.max().item() < 2e-3
