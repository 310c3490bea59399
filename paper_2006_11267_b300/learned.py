"""Training and use of the learned spectral-bound predictor (no counterpart in
the paper; see include/ciq.h, "learned spectral-bound predictor").

Everything numeric runs in libciq's kernels: features, labels (the batched
solve with its Lanczos pre-pass), normaliser, initialisation, Adam training
and BF16 inference.  This module only sequences those calls and takes the
logarithms of the labels the solve reports.
"""
from __future__ import annotations

import math

from . import _ciq


def label_problems(problems, Q, tol, **opts):
    """(F, Y, infos): network inputs and labels (log theta_min, log theta_max,
    log iterations) of each problem from a batched solve with the pre-pass.
    problems: dicts with X, B, kernel (device tensors); lmin/lmax are ignored."""
    import torch
    plain = [{k: v for k, v in p.items() if k not in ("lmin", "lmax")} for p in problems]
    _, infos = _ciq.ciq_sqrt_batched(plain, Q, tol, **opts)
    F = _ciq.ciq_mlp_features(plain)
    Y = torch.tensor([[math.log(max(i["ritz_min"], 1e-300)), math.log(max(i["ritz_max"], 1e-300)),
                       math.log(max(i["iters"], 1))] for i in infos], dtype=torch.float32, device=F.device)
    return F, Y, infos


def train_predictor(F, Y, steps=4000, batch=128, lr=2e-3, seed=0x5eed, init_seed=7):
    """A trained parameter vector (device) and the minibatch losses."""
    import torch
    theta = torch.zeros(_ciq.CIQ_MLP_PARAMS, dtype=torch.float32, device=F.device)
    adam = torch.zeros(2 * _ciq.CIQ_MLP_PARAMS, dtype=torch.float32, device=F.device)
    losses = torch.zeros(max(1, steps), dtype=torch.float32, device=F.device)
    _ciq.ciq_mlp_normaliser(F, Y, theta)
    _ciq.ciq_mlp_init(theta, init_seed)
    _ciq.ciq_mlp_train(theta, adam, F, Y, steps, batch, lr, seed, 1, losses)
    return theta, losses


def lmax_margin_from_validation(theta, F, Y, quantile=0.99):
    """Margin (in log units) to add to the predicted log theta_max so that the
    given fraction of validation problems is not under-predicted."""
    import torch
    pred = _ciq.ciq_mlp_predict(theta, F, bf16=True)
    under = (Y[:, 1] - pred[:, 1]).double().cpu()
    return max(0.0, float(torch.quantile(under, quantile)))


def batch_schedule(pred_log_iters, batch=512, long_iters=500):
    """Batches of problem indices sized ahead of time from the predicted log
    iteration counts (column 2 of ciq_mlp_predict): the problems predicted
    to need at least `long_iters` iterations form one batch of their own
    (a batch runs as long as its slowest problem, so they are kept out of
    the others), and the rest run in batches of `batch` in order of
    predicted iterations, shortest first."""
    import numpy as np
    pred = np.asarray(pred_log_iters, dtype=np.float64).reshape(-1)
    order = np.argsort(pred, kind="stable")
    cut = math.log(long_iters)
    short = [int(i) for i in order if pred[i] < cut]
    long = [int(i) for i in order if pred[i] >= cut]
    batches = [short[b:b + batch] for b in range(0, len(short), batch)]
    if long:
        batches.append(long)
    return batches

