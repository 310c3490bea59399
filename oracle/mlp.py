"""FP64 reference of the learned spectral-bound predictor (TEST INFRASTRUCTURE:
only tests/, __graft_entry__.smoke() and bench.py's CPU leg may import it).

The paper has no learned component; this is the small regression network
that predicts, from a problem's description, the quantities the Lanczos
pre-pass (App. B.2) and the msMINRES run (App. C) would produce:

  inputs  (38): log N, d, kernel type (0 RBF, 1 Matern-5/2), log lengthscale,
                log outputscale, log sigma^2 (floored at 1e-12), the mean of
                each of the 16 coordinates of X and the variance of each
                (coordinates >= d are 0);
  outputs  (3): log theta_min, log theta_max (the pre-pass's Ritz extremes)
                and log of the msMINRES iteration count.

Network: standardised inputs -> 64 tanh -> 64 tanh -> 3 linear, outputs
de-standardised.  Loss: mean over samples and outputs of the squared error
of the standardised outputs.  Training: Adam (Kingma and Ba, 2015) with the
published default moments (0.9, 0.999, 1e-8) and bias correction, minibatch
indices drawn with replacement from splitmix64 (ciq_inputs).

Flat parameter layout (floats), shared with the CUDA kernels by definition
(not by code):
  [0, 38)       input means            [38, 76)    input standard deviations
  [76, 79)      output means           [79, 82)    output standard deviations
  W1 38x64 row-major (input-major), b1 64, W2 64x64, b2 64, W3 64x3, b3 3.
Only the entries from W1 on are trained.
"""
from __future__ import annotations

import numpy as np

import ciq_inputs as ci

N_IN = 38
N_HID = 64
N_OUT = 3
MAX_DIM = 16
OFF_NORM = 0
OFF_W1 = 2 * N_IN + 2 * N_OUT
OFF_B1 = OFF_W1 + N_IN * N_HID
OFF_W2 = OFF_B1 + N_HID
OFF_B2 = OFF_W2 + N_HID * N_HID
OFF_W3 = OFF_B2 + N_HID
OFF_B3 = OFF_W3 + N_HID * N_OUT
N_PARAMS = OFF_B3 + N_OUT


def features(X: np.ndarray, kind: str, lengthscale: float, outputscale: float, noise: float) -> np.ndarray:
    """Input vector of one problem (population mean and variance of X's columns)."""
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    f = np.zeros(N_IN)
    f[0] = np.log(n)
    f[1] = d
    f[2] = 0.0 if kind == "rbf" else 1.0
    f[3] = np.log(lengthscale)
    f[4] = np.log(outputscale)
    f[5] = np.log(max(noise, 1e-12))
    f[6:6 + d] = X.mean(axis=0)
    f[6 + MAX_DIM:6 + MAX_DIM + d] = X.var(axis=0)
    return f


def unpack(theta: np.ndarray):
    """Views (fmu, fsd, ymu, ysd, W1, b1, W2, b2, W3, b3) of a flat parameter vector."""
    t = np.asarray(theta, dtype=np.float64)
    return (t[0:N_IN], t[N_IN:2 * N_IN], t[2 * N_IN:2 * N_IN + N_OUT], t[2 * N_IN + N_OUT:OFF_W1],
            t[OFF_W1:OFF_B1].reshape(N_IN, N_HID), t[OFF_B1:OFF_W2],
            t[OFF_W2:OFF_B2].reshape(N_HID, N_HID), t[OFF_B2:OFF_W3],
            t[OFF_W3:OFF_B3].reshape(N_HID, N_OUT), t[OFF_B3:N_PARAMS])


def normaliser(F: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """The first 82 parameters: column means and standard deviations (1 where a column is constant)."""
    F = np.asarray(F, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    fsd = F.std(axis=0)
    ysd = Y.std(axis=0)
    fsd[fsd <= 0] = 1.0
    ysd[ysd <= 0] = 1.0
    return np.concatenate([F.mean(axis=0), fsd, Y.mean(axis=0), ysd])


def forward(theta, F):
    """(Z0, H1, H2, Y_std, Y): standardised inputs, hidden activations,
    standardised outputs and de-standardised outputs for rows of F."""
    fmu, fsd, ymu, ysd, W1, b1, W2, b2, W3, b3 = unpack(theta)
    Z0 = (np.asarray(F, dtype=np.float64) - fmu) / fsd
    H1 = np.tanh(Z0 @ W1 + b1)
    H2 = np.tanh(H1 @ W2 + b2)
    S = H2 @ W3 + b3
    return Z0, H1, H2, S, S * ysd + ymu


def loss_and_grad(theta, F, Y):
    """Mean squared error of the standardised outputs and its gradient with
    respect to every parameter (0 for the normaliser entries), by the chain rule."""
    fmu, fsd, ymu, ysd, W1, b1, W2, b2, W3, b3 = unpack(theta)
    Z0, H1, H2, S, _ = forward(theta, F)
    R = S - (np.asarray(Y, dtype=np.float64) - ymu) / ysd
    m = R.size
    loss = float(np.sum(R * R) / m)
    dS = 2.0 * R / m
    g = np.zeros(N_PARAMS)
    g[OFF_W3:OFF_B3] = (H2.T @ dS).ravel()
    g[OFF_B3:N_PARAMS] = dS.sum(axis=0)
    dA2 = (dS @ W3.T) * (1.0 - H2 * H2)
    g[OFF_W2:OFF_B2] = (H1.T @ dA2).ravel()
    g[OFF_B2:OFF_W3] = dA2.sum(axis=0)
    dA1 = (dA2 @ W2.T) * (1.0 - H1 * H1)
    g[OFF_W1:OFF_B1] = (Z0.T @ dA1).ravel()
    g[OFF_B1:OFF_W2] = dA1.sum(axis=0)
    return loss, g


def init_params(seed: int, norm: np.ndarray) -> np.ndarray:
    """Glorot-uniform weights (bound sqrt(6 / (fan_in + fan_out))), zero
    biases; uniforms from splitmix64 output k for weight entry k."""
    theta = np.zeros(N_PARAMS)
    theta[:OFF_W1] = norm
    u = ci.uniform(seed, N_PARAMS)
    for off, fi, fo in ((OFF_W1, N_IN, N_HID), (OFF_W2, N_HID, N_HID), (OFF_W3, N_HID, N_OUT)):
        a = np.sqrt(6.0 / (fi + fo))
        theta[off:off + fi * fo] = a * (2.0 * u[off:off + fi * fo] - 1.0)
    return theta


def minibatch(seed: int, step: int, batch: int, n: int) -> np.ndarray:
    """Sample indices of Adam step ``step`` (1-based): floor(u n) with u the
    splitmix64 outputs (step - 1) * batch .. step * batch - 1 of ``seed``."""
    u = ci.uniform(seed, batch, offset=(step - 1) * batch)
    return np.minimum(np.floor(u * n).astype(np.int64), n - 1)


def adam_step(theta, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam update of the trained entries (in place)."""
    sl = slice(OFF_W1, N_PARAMS)
    m[sl] = beta1 * m[sl] + (1.0 - beta1) * g[sl]
    v[sl] = beta2 * v[sl] + (1.0 - beta2) * g[sl] * g[sl]
    mhat = m[sl] / (1.0 - beta1 ** step)
    vhat = v[sl] / (1.0 - beta2 ** step)
    theta[sl] -= lr * mhat / (np.sqrt(vhat) + eps)


def train(theta, F, Y, steps, batch, lr, seed, first_step=1, m=None, v=None):
    """Adam steps first_step .. first_step + steps - 1 on minibatches of (F, Y)."""
    theta = np.array(theta, dtype=np.float64)
    m = np.zeros(N_PARAMS) if m is None else m
    v = np.zeros(N_PARAMS) if v is None else v
    losses = []
    for s in range(first_step, first_step + steps):
        idx = minibatch(seed, s, batch, len(F))
        loss, g = loss_and_grad(theta, F[idx], Y[idx])
        adam_step(theta, g, m, v, s, lr)
        losses.append(loss)
    return theta, m, v, np.array(losses)
