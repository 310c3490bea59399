"""Posterior Thompson draws (Sec. 5, Eq. thompson_sample) through the C ABI
against the FP64 oracle (oracle/posterior.py, pinned in
tests/test_oracle_posterior.py): the draw against the eigendecomposition of
the dense posterior covariance (O1), and msMINRES-CIQ on that dense matrix
(O2) at equal nodes and J.  Errors are relative 2-norms per draw
(tests/relerr.py)."""
import numpy as np
import pytest
import torch

import ciq_inputs as ci
import paper_2006_11267_b300 as P
from oracle import ciq as O
from oracle import posterior as PO
from relerr import fp32_gate, rel

pytestmark = pytest.mark.gpu

LS = np.array([0.3, 0.2, 0.4, 0.25])
S, NOISE, JITTER, MEAN = 1.2, 1e-4, 1e-4, 0.1


def data(n, nc, t, seed, d=4):
    Xtr = ci.points(seed, n, d).astype(np.float32)
    Xc = ci.points(seed + 1, nc, d).astype(np.float32)
    y = np.sin(5.0 * Xtr.astype(np.float64) @ np.arange(1, d + 1) / d).astype(np.float32)
    eps = ci.rhs(seed + 2, nc, t).astype(np.float32)
    return Xtr, y, Xc, eps


def oracle(kind, Xtr, y, Xc):
    return PO.posterior(Xtr.astype(np.float64), y.astype(np.float64), Xc.astype(np.float64), kind, LS, S, NOISE,
                        JITTER, MEAN)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("kind", ["matern52", "rbf"])
def test_posterior_draws_against_eigendecomposition(kind, prec):
    Xtr, y, Xc, eps = data(150, 3000, 8, 11)
    mu, cov = oracle(kind, Xtr, y, Xc)
    exact = PO.thompson_draws(mu, cov, eps)
    dev = lambda a: torch.from_numpy(a).cuda()
    out, info = P.ciq_posterior_sample(dev(Xtr), dev(y), dev(Xc), kind, LS, S, NOISE, JITTER, MEAN, dev(eps), 15,
                                       1e-5, stop_rule="errbound", max_iter=3000, precision=prec)
    assert info["status"] == 0 and info["lmin_used"] == JITTER
    got = out.cpu().numpy().astype(np.float64)
    assert rel(got, exact) < 1e-3
    assert rel(got - mu[None, :], exact - mu[None, :]) < 1e-3          # the fluctuation part itself
    # eps = 0: the posterior mean alone
    zero = np.zeros((1, Xc.shape[0]), np.float32)
    m0, _ = P.ciq_posterior_sample(dev(Xtr), dev(y), dev(Xc), kind, LS, S, NOISE, JITTER, MEAN, dev(zero), 15, 1e-5,
                                   stop_rule="errbound", max_iter=3000)
    assert rel(m0.cpu().numpy()[0], mu) < 1e-5


@pytest.mark.parametrize("krylov", ["basis", "recurrence"])
def test_posterior_fp32_matches_serial_oracle_at_equal_nodes_and_J(krylov):
    Xtr, y, Xc, eps = data(100, 1500, 5, 21)
    mu, cov = oracle("matern52", Xtr, y, Xc)
    lam = np.linalg.eigvalsh(cov)
    Q, J = 12, 1500                     # kappa(COV*) ~ 1e5: converged well before J
    nodes = O.quad_nodes(JITTER, 1.05 * lam[-1], Q)
    run = lambda C: O.ciq_apply(O.dense_mvm(C), eps.astype(np.float64), Q, "sqrt", max_iter=J, nodes=nodes,
                                lmin=JITTER)[0]
    ref, info_o = O.ciq_apply(O.dense_mvm(cov), eps.astype(np.float64), Q, "sqrt", max_iter=J, nodes=nodes,
                              lmin=JITTER)
    assert np.max(info_o["errbound"] / np.linalg.norm(ref, axis=1)) < 1e-8            # converged
    out, info = P.ciq_posterior_sample(Xtr, y, Xc, "matern52", LS, S, NOISE, JITTER, MEAN, eps, Q, 0.0,
                                       max_iter=J, nodes=nodes, lmin=JITTER, krylov=krylov)
    assert info["iters"] == J and info["krylov"] == krylov
    tol, floor = fp32_gate(run, cov, ref)
    err = rel(out - mu[None, :].astype(np.float32), ref)
    assert err < tol, (err, tol, floor)


def test_prior_draws_without_training_data_and_interpolation():
    _, _, Xc, eps = data(1, 800, 3, 31)
    dev = lambda a: torch.from_numpy(a).cuda()
    out, info = P.ciq_posterior_sample(None, None, dev(Xc), "matern52", LS, S, NOISE, JITTER, MEAN, dev(eps), 15,
                                       1e-6, stop_rule="errbound", max_iter=2000)
    mu, cov = PO.posterior(np.zeros((0, 4)), np.zeros(0), Xc.astype(np.float64), "matern52", LS, S, NOISE, JITTER,
                           MEAN)
    assert rel(out.cpu().numpy(), PO.thompson_draws(mu, cov, eps)) < 1e-3
    # Candidates at the training points with nearly noise-free data: every
    # draw passes within a few sqrt(jitter) of the observations there.
    Xtr, y, Xc2, _ = data(60, 500, 1, 41)
    Xc2 = np.vstack([Xtr, Xc2]).astype(np.float32)
    eps2 = ci.rhs(42, Xc2.shape[0], 4).astype(np.float32)
    out, _ = P.ciq_posterior_sample(Xtr, y, Xc2, "matern52", LS, S, 1e-8, JITTER, MEAN, eps2, 15, 1e-6,
                                    stop_rule="errbound", max_iter=3000)
    assert np.abs(out[:, :60] - y[None, :]).max() < 6 * np.sqrt(JITTER)


@pytest.mark.parametrize("form", ["identity", "mvm"])
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_preconditioned_draws_use_a_root_of_the_posterior_covariance(prec, form):
    # opt.precond_rank: the device factors K** - C C^T (pivoted Cholesky
    # with the low-rank term in its columns and diagonal) and the draws use
    # the rotated root R (R R^T = COV*), the mean added after the map back
    # through P^{1/2} (identity form) or the final (K** - C C^T) MVM (printed
    # form).  Checked on all N* columns of the identity: (out - mu) holds R^T,
    # so R R^T against the dense covariance (a property of any valid root,
    # whichever pivots the device chose).  Gate: P^{1/2} and P^{-1/2} use the
    # FP32 basis Qh, whose orthonormality error (~1e-7) enters P^{1/2} P^{-1/2}
    # through g^+ g^- ~ sqrt(kappa(P)) (about 300 at jitter 1e-4): a few 1e-4
    # whatever the solve's precision (measured 3.0-3.3e-4; 4e-6 without the
    # preconditioner), below the mode's 1e-3.
    Xtr, y, Xc, _ = data(60, 700, 1, 21)
    mu, cov = oracle("matern52", Xtr, y, Xc)
    nc = Xc.shape[0]
    eye = np.eye(nc, dtype=np.float32)
    kw = dict(max_iter=3000, stop_rule="errbound", precision=prec, sqrt_form=form, precond_rank=40)
    out, info = P.ciq_posterior_sample(Xtr, y, Xc, "matern52", LS, S, NOISE, JITTER, MEAN, torch.from_numpy(eye).cuda(),
                                       15, 1e-7, **kw)
    assert info["status"] == 0 and info["precond_rank"] == 40
    R = (out.cpu().numpy().astype(np.float64) - mu[None, :]).T
    assert np.linalg.norm(R @ R.T - cov) / np.linalg.norm(cov) < 1e-3
    zero = torch.zeros((1, nc), device="cuda")
    m, _ = P.ciq_posterior_sample(Xtr, y, Xc, "matern52", LS, S, NOISE, JITTER, MEAN, zero, 15, 1e-7, **kw)
    assert rel(m.cpu().numpy(), mu[None, :]) < 1e-5


def test_unpreconditioned_printed_form_includes_the_low_rank_term():
    # sqrt_form "mvm" without a preconditioner: COV* (sum_q w_q x_q), the
    # final MVM with the -C C^T term: a root of COV* as well.
    Xtr, y, Xc, _ = data(60, 500, 1, 23)
    mu, cov = oracle("rbf", Xtr, y, Xc)
    nc = Xc.shape[0]
    eye = torch.eye(nc, device="cuda")
    out, info = P.ciq_posterior_sample(Xtr, y, Xc, "rbf", LS, S, NOISE, JITTER, MEAN, eye, 15, 1e-7, max_iter=3000,
                                       stop_rule="errbound", sqrt_form="mvm")
    assert info["status"] == 0
    R = (out.cpu().numpy().astype(np.float64) - mu[None, :]).T
    assert np.linalg.norm(R @ R.T - cov) / np.linalg.norm(cov) < 1e-4


def test_preconditioned_draws_need_fewer_iterations():
    # The posterior covariance at jitter 1e-4 is ill-conditioned; a rank-100
    # preconditioner takes its largest directions out of A, so the solve in
    # the space of A needs fewer iterations (measured 218 against 283 here;
    # the spectrum of this 4000-candidate covariance decays slowly past its
    # first 100 directions).
    Xtr, y, Xc, eps = data(100, 4000, 16, 31)
    Xd, ed = torch.from_numpy(Xc).cuda(), torch.from_numpy(eps).cuda()
    kw = dict(max_iter=4000, stop_rule="errbound", precision="fp16")
    _, i0 = P.ciq_posterior_sample(Xtr, y, Xd, "matern52", LS, S, NOISE, JITTER, MEAN, ed, 12, 1e-3, **kw)
    _, i1 = P.ciq_posterior_sample(Xtr, y, Xd, "matern52", LS, S, NOISE, JITTER, MEAN, ed, 12, 1e-3, precond_rank=100,
                                   **kw)
    assert i0["status"] == 0 and i1["status"] == 0 and i1["precond_rank"] == 100
    assert i1["iters"] < 0.9 * i0["iters"], (i1["iters"], i0["iters"])


def test_full_size_posterior_draws_on_sampled_candidates():
    # The bench's posterior workload at full size and in its launch shape
    # (50,000 candidates, 256 observations, Matern-5/2 ARD, 64 draws, error
    # bound 1e-3, FP16 split), checked where the oracle can compute outputs
    # one by one: the posterior mean (eps = 0) on sampled candidates, and the
    # root applied twice, R (R eps) = COV* eps, on the same candidates (rows
    # of COV* from the oracle's kernels and the exact inner solve).
    import bench
    from oracle import kernels as OK

    c = bench.POSTERIOR
    Xtr, y, Xc, eps = bench.posterior_inputs(c["n_cand"])
    ls = np.array(c["ls"])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    args = (dev(Xtr), dev(y), dev(Xc), c["kind"], ls, c["s"], c["noise"], c["jitter"], c["mean"])
    kw = dict(stop_rule="errbound", max_iter=4000, precision="fp16")
    zero = np.zeros((1, c["n_cand"]), np.float32)
    mu_d, _ = P.ciq_posterior_sample(*args, dev(zero), c["q"], 1e-3, **kw)
    f, info = P.ciq_posterior_sample(*args, dev(eps), c["q"], 1e-3, **kw)
    assert info["status"] == 0
    g = (f - mu_d).cpu().numpy()                                   # R eps
    f2, _ = P.ciq_posterior_sample(*args, dev(g), c["q"], 1e-3, **kw)
    h = (f2 - mu_d).cpu().numpy().astype(np.float64)               # R (R eps)
    n = c["n_cand"]
    rows = np.concatenate([np.arange(0, 64), np.arange(n - 64, n), np.arange(25000, 25128)])
    X64, Xtr64, E = Xc.astype(np.float64), Xtr.astype(np.float64), eps.astype(np.float64).T
    kern = lambda A, B: PO.kernel_ard(A, B, c["kind"], ls, c["s"])
    M = kern(Xtr64, Xtr64) + c["noise"] * np.eye(Xtr.shape[0])
    Kr = kern(X64[rows], Xtr64)                                    # K*X on the sampled rows
    mu_rows = c["mean"] + Kr @ np.linalg.solve(M, y.astype(np.float64) - c["mean"])
    assert np.linalg.norm(mu_d.cpu().numpy()[0, rows] - mu_rows) / np.linalg.norm(mu_rows) < 1e-5
    KxE = kern(Xtr64, X64) @ E                                     # K_X* eps, all candidates
    cov_e = kern(X64[rows], X64) @ E - Kr @ np.linalg.solve(M, KxE) + c["jitter"] * E[rows]
    err = np.linalg.norm(h[:, rows] - cov_e.T, axis=1) / np.linalg.norm(cov_e.T, axis=1)
    # Two applications of a root, each stopped at the 1e-3 bound: to first
    # order their relative errors add (measured 4.2e-4, median 3.4e-4).
    assert err.max() < 2e-3, err.max()
