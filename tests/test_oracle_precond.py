"""Pins for the preconditioned oracle (oracle/precond.py): App.
"Preconditioning msMINRES-CIQ", Eq. precond_sqrt and Eq. precond_sqrt_inverse.

Each check ties a part to something outside it: LAPACK/SciPy (Cholesky,
sqrtm, generalized eigenvalues, dense solves), brute force (the pivot rule
from explicit Schur complements), the unpreconditioned oracle run on the
explicit matrix P^{-1/2} K P^{-1/2}, and the identities that define the
rotated roots (R R^T = K, R' R'^T = K^{-1}, R = K^{1/2} Omega with Omega
orthogonal; rank 0 and full rank give the principal roots)."""
import numpy as np
import pytest
import scipy.linalg

import ciq_inputs as ci
from oracle import eig, kernels
from oracle import precond as PC
from oracle.lanczos import lanczos
from oracle.msminres import msminres
from oracle.quadrature import quad_nodes


def _kernel_case(n=120, d=3, kind="rbf", ls=0.35, noise=1e-2, seed=7):
    X = ci.points(seed, n, d)
    Kxx = kernels.kernel_matrix(X, X, kind, ls, 1.0)
    return Kxx, Kxx + noise * np.eye(n), noise


def _pre(Kxx, noise, rank):
    return PC.kernel_preconditioner(np.diag(Kxx), lambda i: Kxx[:, i], noise, rank)


def test_pivoted_cholesky_full_rank_reproduces_the_matrix_and_scipy_cholesky():
    Kxx, _, _ = _kernel_case(n=60, ls=0.6)
    K = Kxx + 1e-6 * np.eye(60)                      # strictly positive definite
    L, piv = PC.pivoted_cholesky(np.diag(K), lambda i: K[:, i], 60)
    assert sorted(piv.tolist()) == list(range(60))
    np.testing.assert_allclose(L @ L.T, K, rtol=0, atol=1e-12 * np.abs(K).max())
    # In pivot order the factor is the lower Cholesky factor of the permuted matrix.
    Lp = L[piv]
    assert np.abs(np.triu(Lp, 1)).max() == 0.0
    np.testing.assert_allclose(Lp, np.linalg.cholesky(K[np.ix_(piv, piv)]), rtol=1e-10, atol=1e-12)


def test_pivoted_cholesky_pivot_rule_and_schur_complement_by_brute_force():
    Kxx, _, _ = _kernel_case(n=90)
    L, piv = PC.pivoted_cholesky(np.diag(Kxx), lambda i: Kxx[:, i], 25)
    for k in range(25):
        S = Kxx - L[:, :k] @ L[:, :k].T                    # explicit Schur complement after k steps
        assert piv[k] == int(np.argmax(np.diag(S)))
    E = Kxx - L @ L.T
    assert np.linalg.eigvalsh(E).min() > -1e-12           # positive semidefinite residual
    assert np.abs(E[piv]).max() < 1e-12 and np.abs(E[:, piv]).max() < 1e-12
    # the trace of the residual falls with every step
    tr = [np.trace(Kxx - L[:, :k] @ L[:, :k].T) for k in range(26)]
    assert all(b < a for a, b in zip(tr, tr[1:]))


@pytest.mark.parametrize("rank", [0, 5, 40])
def test_preconditioner_inverse_and_root_match_dense_linear_algebra(rank):
    Kxx, K, noise = _kernel_case()
    pre, _ = _pre(Kxx, noise, rank)
    P = pre.dense()
    V = ci.rhs(3, K.shape[0], 4).T
    np.testing.assert_allclose(pre.matvec(V), P @ V, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(pre.solve(V), np.linalg.solve(P, V), rtol=1e-9, atol=1e-9 * np.abs(np.linalg.solve(P, V)).max())
    S = np.real(scipy.linalg.sqrtm(P))
    np.testing.assert_allclose(pre.sqrt(V), S @ V, rtol=0, atol=1e-9 * np.abs(S @ V).max())
    np.testing.assert_allclose(pre.sqrt(pre.sqrt(V)), P @ V, rtol=0, atol=1e-9 * np.abs(P @ V).max())


@pytest.mark.parametrize("rank", [0, 10, 60])
def test_spectrum_of_preconditioned_matrix_is_at_least_one(rank):
    # P = L L^T + sigma^2 I <= K because K_XX - L L^T is a Schur complement:
    # the generalized eigenvalues of (K, P) are >= 1 (the lambda_min reading).
    Kxx, K, noise = _kernel_case(noise=1e-3)
    pre, _ = _pre(Kxx, noise, rank)
    lam = scipy.linalg.eigh(K, pre.dense(), eigvals_only=True)
    assert lam.min() >= 1.0 - 1e-9
    if rank == 0:
        np.testing.assert_allclose(lam, np.linalg.eigvalsh(K) / noise, rtol=1e-9)


def test_preconditioned_lanczos_is_lanczos_on_the_explicit_operator():
    Kxx, K, noise = _kernel_case()
    pre, _ = _pre(Kxx, noise, 15)
    P = pre.dense()
    lp, Vp = np.linalg.eigh(P)
    Pmh = (Vp * lp ** -0.5) @ Vp.T
    A = Pmh @ K @ Pmh
    z = pre.sqrt(ci.start_vector(4, K.shape[0]))
    # 12 steps: before orthogonality is lost (after it two correct
    # implementations drift apart, finite-precision Lanczos being chaotic).
    a1, b1 = PC.precond_lanczos(lambda v: K @ v, pre.solve, z, 12)
    a2, b2 = lanczos(lambda v: A @ v, Pmh @ z, 12)
    np.testing.assert_allclose(a1, a2, rtol=1e-9)
    np.testing.assert_allclose(b1, b2, rtol=1e-9)


def test_preconditioned_msminres_against_explicit_operator_and_exact_solves():
    Kxx, K, noise = _kernel_case(n=80)
    n = K.shape[0]
    pre, _ = _pre(Kxx, noise, 12)
    P = pre.dense()
    lp, Vp = np.linalg.eigh(P)
    Pmh = (Vp * lp ** -0.5) @ Vp.T
    A = Pmh @ K @ Pmh
    Z = pre.sqrt(ci.rhs(5, n, 3).T)
    shifts = np.array([0.0, 0.3, 7.0])
    # equal J (12, before finite-precision drift): the iterates are P^{-1/2}
    # times those of plain msMINRES on A from P^{-1/2} z
    X1, i1 = PC.precond_msminres(lambda V: K @ V, pre.solve, Z, shifts, 12)
    Y2, i2 = msminres(lambda V: A @ V, Pmh @ Z, shifts, 12)
    np.testing.assert_allclose(X1, np.einsum("ij,qjc->qic", Pmh, Y2), rtol=0, atol=1e-8 * np.abs(X1).max())
    np.testing.assert_allclose(np.abs(i1["phibar"]), np.abs(i2["phibar"]), rtol=1e-7)
    # |phibar| is the P^{-1}-norm of the true residual of (K + tP) x = z
    for q, t in enumerate(shifts):
        r = Z - (K + t * P) @ X1[q]
        np.testing.assert_allclose(np.sqrt(np.einsum("ic,ic->c", r, np.linalg.solve(P, r))),
                                   np.abs(i1["phibar"][q]), rtol=1e-6)
    # J = n: the exact shifted solves
    Xn, _ = PC.precond_msminres(lambda V: K @ V, pre.solve, Z, shifts, n)
    for q, t in enumerate(shifts):
        np.testing.assert_allclose(Xn[q], np.linalg.solve(K + t * P, Z), rtol=0, atol=1e-7 * np.abs(Xn[q]).max())


def test_exact_rotated_roots_satisfy_their_defining_identities():
    Kxx, K, noise = _kernel_case(n=70)
    n = K.shape[0]
    pre, _ = _pre(Kxx, noise, 9)
    R, Rp = PC.rotated_roots_exact(K, pre.dense(), np.eye(n))      # rows: R e_i, i.e. R^T
    R, Rp = R.T, Rp.T
    np.testing.assert_allclose(R @ R.T, K, rtol=0, atol=1e-9 * np.abs(K).max())
    Kinv = np.linalg.inv(K)
    np.testing.assert_allclose(Rp @ Rp.T, Kinv, rtol=0, atol=1e-8 * np.abs(Kinv).max())
    Om = np.linalg.solve(np.real(scipy.linalg.sqrtm(K)), R)        # R = K^{1/2} Omega
    np.testing.assert_allclose(Om.T @ Om, np.eye(n), rtol=0, atol=1e-7)


@pytest.mark.parametrize("op", ["sqrt", "invsqrt"])
@pytest.mark.parametrize("rank", [0, 8, 70])
def test_preconditioned_ciq_converges_to_the_rotated_root(op, rank):
    # rank 0 (P = sigma^2 I) and full rank (P = K) give the principal roots.
    Kxx, K, noise = _kernel_case(n=70, noise=1e-2)
    n = K.shape[0]
    pre, _ = _pre(Kxx, noise, rank)
    B = ci.rhs(9, n, 3)
    Rb, Rpb = PC.rotated_roots_exact(K, pre.dense(), B)
    exact = Rb if op == "sqrt" else Rpb
    A, info = PC.ciq_precond_apply(lambda V: K @ V, pre, B, 20, op, tol=1e-12, max_iter=400, stop_rule="errbound",
                                   start=ci.start_vector(2, n))
    err = np.linalg.norm(A - exact, axis=1) / np.linalg.norm(exact, axis=1)
    assert err.max() < 1e-7, err
    assert info["lmin"] == 1.0
    if rank in (0, 70):
        prin = (eig.sqrt_apply if op == "sqrt" else eig.invsqrt_apply)(K, B.T).T
        assert (np.linalg.norm(exact - prin, axis=1) / np.linalg.norm(prin, axis=1)).max() < 1e-8


@pytest.mark.parametrize("op", ["sqrt", "invsqrt"])
def test_preconditioned_ciq_sqrt_forms_and_scalar_stop_rule(op):
    Kxx, K, noise = _kernel_case(n=150, noise=1e-3)
    n = K.shape[0]
    pre, _ = _pre(Kxx, noise, 20)
    B = ci.rhs(11, n, 4)
    kw = dict(tol=1e-4, max_iter=600, stop_rule="errbound", start=ci.start_vector(3, n))
    A1, i1 = PC.ciq_precond_apply(lambda V: K @ V, pre, B, 12, op, **kw)
    A2, i2 = PC.ciq_precond_apply(lambda V: K @ V, pre, B, 12, op, errbound_norm="scalar", **kw)
    # the scalar norms (||b|| sqrt(alpha_1), Gauss rule) stop within a few steps of the estimate's norm
    assert np.abs(i1["iters"] - i2["iters"]).max() <= 5
    if op == "sqrt":
        A3, _ = PC.ciq_precond_apply(lambda V: K @ V, pre, B, 12, op, sqrt_form="mvm", tol=0.0, max_iter=300,
                                     start=ci.start_vector(3, n))
        A4, _ = PC.ciq_precond_apply(lambda V: K @ V, pre, B, 12, op, tol=0.0, max_iter=300,
                                     start=ci.start_vector(3, n))
        assert (np.linalg.norm(A3 - A4, axis=1) / np.linalg.norm(A4, axis=1)).max() < 1e-6


def test_literal_sqrt_form_is_accurate_in_the_space_of_K():
    # Eq. precond_sqrt as printed, R b = K (R' b) with R' b's solve and stop
    # rule, against the identity form whose error in the space of K can exceed
    # the bound its A-space stop rule uses (kernel matrix with sigma^2 = 1e-3).
    X = ci.points(13, 600, 4)
    Kxx = kernels.kernel_matrix(X, X, "rbf", 0.3, 1.0)
    K = Kxx + 1e-3 * np.eye(600)
    pre, _ = _pre(Kxx, 1e-3, 30)
    B = ci.rhs(14, 600, 4)
    Rb, _ = PC.rotated_roots_exact(K, pre.dense(), B)
    kw = dict(tol=1e-3, max_iter=3000, stop_rule="errbound", start=ci.start_vector(5, 600))
    A_lit, i_lit = PC.ciq_precond_apply(lambda V: K @ V, pre, B, 12, "sqrt", sqrt_form="mvm", **kw)
    A_id, i_id = PC.ciq_precond_apply(lambda V: K @ V, pre, B, 12, "sqrt", **kw)
    e_lit = (np.linalg.norm(A_lit - Rb, axis=1) / np.linalg.norm(Rb, axis=1)).max()
    e_id = (np.linalg.norm(A_id - Rb, axis=1) / np.linalg.norm(Rb, axis=1)).max()
    assert e_lit < 1e-3 < e_id, (e_lit, e_id)
    assert i_lit["iters"].max() > i_id["iters"].max()
