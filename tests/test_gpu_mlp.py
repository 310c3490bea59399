"""The learned spectral-bound predictor on the GPU: feature, initialisation,
normaliser, gradient, Adam and inference kernels against the FP64 oracle
(oracle/mlp.py), and the learned batched pipeline against the pre-pass one.

Tolerances: the kernels compute in FP32 (tanhf, FP32 sums of at most 64
terms per neuron, FP64 totals over samples), so values match the FP64 oracle
to ~1e-6 relative and gradients to ~1e-5; BF16 inference rounds weights and
activations to 8 significant bits, so standardised outputs move by ~1e-2.
"""
import math

import numpy as np
import pytest
import torch

import ciq_inputs as ci
import paper_2006_11267_b300 as P
from paper_2006_11267_b300 import learned
from oracle import eig, kernels, mlp

pytestmark = pytest.mark.gpu

DEV = "cuda"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def small_batch(seed, count, nmax=2048, t=8):
    """The uneven-batch recipe with N log-uniform in [256, nmax]."""
    u = ci.uniform(ci.stream_seed(seed, 9), 5 * count).reshape(count, 5)
    out = []
    for p in range(count):
        n = int(math.exp(math.log(256) + u[p, 0] * (math.log(nmax) - math.log(256))))
        d = 2 + int(u[p, 1] * 11)
        kind = "rbf" if u[p, 2] < 0.5 else "matern52"
        ls = math.exp(math.log(0.05) + u[p, 3] * (math.log(1.0) - math.log(0.05)))
        noise = math.exp(math.log(1e-4) + u[p, 4] * (math.log(1e-1) - math.log(1e-4)))
        ps = seed * 1000003 + p
        out.append(dict(X=dev(ci.points(ps, n, d)), B=dev(ci.rhs(ps, n, t)), kernel=P.Kernel(kind, ls, 1.0, noise)))
    return out


def test_features_match_oracle():
    probs = small_batch(3, 6) + [dict(X=dev(ci.points(5, 1, 16)), B=dev(ci.rhs(5, 1, 1)),
                                      kernel=P.Kernel("rbf", 0.7, 2.0, 0.0))]
    F = P.ciq_mlp_features(probs).cpu().numpy()
    for pr, f in zip(probs, F):
        k = pr["kernel"]
        ref = mlp.features(pr["X"].cpu().numpy().astype(np.float64), k.type, k.lengthscale, k.outputscale, k.noise)
        np.testing.assert_allclose(f, ref, rtol=1e-5, atol=1e-6)


def test_init_and_normaliser_match_oracle():
    Fh = ci.normal(1, 300 * mlp.N_IN).reshape(300, mlp.N_IN) * 2.0 + 0.5
    Fh[:, 7] = 3.0
    Yh = ci.normal(2, 300 * mlp.N_OUT).reshape(300, mlp.N_OUT) - 4.0
    theta = torch.zeros(P.CIQ_MLP_PARAMS, device=DEV)
    P.ciq_mlp_normaliser(dev(Fh), dev(Yh), theta)
    P.ciq_mlp_init(theta, 1234)
    ref = mlp.init_params(1234, mlp.normaliser(Fh.astype(np.float32), Yh.astype(np.float32)))
    np.testing.assert_allclose(theta.cpu().numpy(), ref, rtol=2e-6, atol=1e-7)


@pytest.mark.parametrize("n", [1, 32, 77, 1000])
def test_loss_and_gradient_match_oracle(n):
    Fh = ci.normal(10 + n, n * mlp.N_IN).reshape(n, mlp.N_IN) * 1.5
    Yh = ci.normal(20 + n, n * mlp.N_OUT).reshape(n, mlp.N_OUT)
    th = mlp.init_params(3, mlp.normaliser(ci.normal(4, 50 * mlp.N_IN).reshape(50, mlp.N_IN),
                                           ci.normal(5, 50 * mlp.N_OUT).reshape(50, mlp.N_OUT)))
    th[mlp.OFF_B1:mlp.OFF_W2] = 0.2
    th32 = th.astype(np.float32)
    loss, g = P.ciq_mlp_loss_grad(dev(th32), dev(Fh), dev(Yh))
    rloss, rg = mlp.loss_and_grad(th32.astype(np.float64), Fh.astype(np.float32).astype(np.float64),
                                  Yh.astype(np.float32).astype(np.float64))
    assert loss == pytest.approx(rloss, rel=1e-5)
    g = g.cpu().numpy()
    assert np.linalg.norm(g - rg) <= 2e-5 * np.linalg.norm(rg)
    assert np.all(g[:mlp.OFF_W1] == 0)


def test_adam_training_tracks_oracle():
    n = 500
    Fh = ci.uniform(31, n * mlp.N_IN).reshape(n, mlp.N_IN) * 2.0 - 1.0
    Yh = np.stack([np.sin(2 * Fh[:, 0]) + Fh[:, 1] ** 2, Fh[:, 2] * Fh[:, 3], np.cos(Fh[:, 0] - Fh[:, 5])], axis=1)
    F, Y = dev(Fh), dev(Yh)
    theta = torch.zeros(P.CIQ_MLP_PARAMS, device=DEV)
    adam = torch.zeros(2 * P.CIQ_MLP_PARAMS, device=DEV)
    P.ciq_mlp_normaliser(F, Y, theta)
    P.ciq_mlp_init(theta, 77)
    th0 = theta.cpu().numpy().astype(np.float64)
    steps = 40
    losses = torch.zeros(steps, device=DEV)
    # two calls (20 + 20 steps) continue one run: moments and step count carry over
    P.ciq_mlp_train(theta, adam, F, Y, 20, 64, 1e-3, 99, 1, losses[:20])
    P.ciq_mlp_train(theta, adam, F, Y, 20, 64, 1e-3, 99, 21, losses[20:])
    ref, _, _, rlosses = mlp.train(th0, Fh.astype(np.float32).astype(np.float64),
                                   Yh.astype(np.float32).astype(np.float64), steps, 64, 1e-3, 99)
    got = theta.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) <= 2e-2 * np.linalg.norm(ref - th0)
    np.testing.assert_allclose(losses.cpu().numpy(), rlosses, rtol=2e-3)


def test_predict_fp32_and_bf16_against_oracle():
    n = 300
    Fh = ci.normal(41, n * mlp.N_IN).reshape(n, mlp.N_IN)
    th = mlp.init_params(9, mlp.normaliser(Fh, ci.normal(42, n * 3).reshape(n, 3)))
    th32 = th.astype(np.float32)
    ref_std = mlp.forward(th32.astype(np.float64), Fh.astype(np.float32).astype(np.float64))[3]
    ref = mlp.forward(th32.astype(np.float64), Fh.astype(np.float32).astype(np.float64))[4]
    out32 = P.ciq_mlp_predict(dev(th32), dev(Fh), bf16=False).cpu().numpy()
    np.testing.assert_allclose(out32, ref, rtol=1e-5, atol=1e-5)
    out16 = P.ciq_mlp_predict(dev(th32), dev(Fh), bf16=True).cpu().numpy()
    ysd = th32[79:82].astype(np.float64)
    ymu = th32[76:79].astype(np.float64)
    err_std = np.abs((out16 - ymu) / ysd - ref_std)
    assert err_std.max() < 0.1 and err_std.mean() < 0.02


def test_learned_batch_matches_prepass_batch_and_saves_work():
    Q, tol = 8, 1e-4
    opts = dict(max_iter=3000)
    train = small_batch(100, 1024)
    F, Y, _ = learned.label_problems(train, Q, tol, **opts)
    theta, losses = learned.train_predictor(F, Y, steps=3000, batch=128, lr=2e-3)
    losses = losses.cpu().numpy()
    assert losses[-200:].mean() < 0.2 * losses[:50].mean()
    val = small_batch(101, 256)
    Fv, Yv, _ = learned.label_problems(val, Q, tol, **opts)
    margin = learned.lmax_margin_from_validation(theta, Fv, Yv, 0.99)
    pred = P.ciq_mlp_predict(theta, Fv).cpu().numpy()
    rmse = float(np.sqrt(np.mean((pred[:, 1] - Yv[:, 1].cpu().numpy()) ** 2)))
    assert rmse < 0.3          # theta_max within ~30 % (log units) on held-out problems
    test = small_batch(102, 128, nmax=900)
    outs_l, infos_l = P.ciq_sqrt_batched_learned(test, Q, tol, theta, margin, **opts)
    outs_p, infos_p = P.ciq_sqrt_batched(test, Q, tol, **opts)
    fallbacks = sum(i["fallback"] for i in infos_l)
    assert fallbacks <= 0.1 * len(test)
    work_l = sum(i["iters"] + i["lanczos_iters"] for i in infos_l)
    work_p = sum(i["iters"] + i["lanczos_iters"] for i in infos_p)
    assert work_l < work_p
    # Judged by the oracle: both pipelines' errors against the eigendecomposition.
    worst_l = worst_p = 0.0
    for pr, ol, op in list(zip(test, outs_l, outs_p))[:24]:
        k = pr["kernel"]
        X = pr["X"].cpu().numpy().astype(np.float64)
        K = kernels.dense_K(X, k.type, k.lengthscale, k.outputscale, k.noise)
        B = pr["B"].cpu().numpy().astype(np.float64)
        truth = eig.sqrt_apply(K, B.T).T
        el = np.linalg.norm(ol.cpu().numpy() - truth) / np.linalg.norm(truth)
        ep = np.linalg.norm(op.cpu().numpy() - truth) / np.linalg.norm(truth)
        worst_l, worst_p = max(worst_l, el), max(worst_p, ep)
    assert worst_l <= max(2.0 * worst_p, 1e-3)


def test_learned_spectral_check_value_is_the_largest_ritz_value():
    # With learned bounds the solve records column 0's msMINRES tridiagonal
    # and reports its largest eigenvalue (warp multisection over Sturm
    # counts), which the spectral check compares with the lambda_max used.
    # After ~100 Lanczos steps the largest Ritz value equals lambda_max(K) to
    # within the FP16-split MVM's accuracy, so it is judged by the FP64
    # eigendecomposition of K.  An untrained network with a wide margin
    # (e^4) keeps the predicted bounds valid, so no problem falls back.
    probs = small_batch(55, 5, nmax=700)
    F, Y, _ = learned.label_problems(probs, 8, 1e-6, max_iter=1000)
    theta = torch.zeros(P.CIQ_MLP_PARAMS, device=DEV)
    P.ciq_mlp_normaliser(F, Y, theta)
    P.ciq_mlp_init(theta, 5)
    _, infos = P.ciq_sqrt_batched_learned(probs, 8, 1e-6, theta, 4.0, max_iter=1000)
    long_runs = 0
    for pr, info in zip(probs, infos):
        assert not info["fallback"]
        k = pr["kernel"]
        K = kernels.dense_K(pr["X"].cpu().numpy().astype(np.float64), k.type, k.lengthscale, k.outputscale, k.noise)
        lam = np.linalg.eigvalsh(K)[-1]
        # Ritz values lie in the spectrum; a short run (a well-conditioned
        # problem) need not have reached lambda_max yet.
        assert info["ritz_max_solve"] <= lam * (1 + 1e-5)
        assert info["ritz_max_solve"] <= info["lmax_used"]
        if info["iters"] >= 30:
            long_runs += 1
            assert abs(info["ritz_max_solve"] - lam) <= 1e-4 * lam, (info["ritz_max_solve"], lam)
    assert long_runs >= 2
