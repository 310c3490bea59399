"""Backward pass (Eq. ciq_deriv) through the C ABI against the FP64 oracle
(oracle/vjp.py, pinned by finite differences) at equal nodes and J."""
import numpy as np
import pytest
import torch

import ciq_inputs as ci
import paper_2006_11267_b300 as P
from oracle import ciq as O
from oracle import kernels
from oracle import vjp as VJP
from relerr import fp32_gate, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["rbf", "matern52"])
@pytest.mark.parametrize("op", ["invsqrt", "sqrt"])
@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_vjp_matches_oracle_at_equal_nodes_and_J(kind, op, precision):
    n, d, T, Q, J = 1100, 3, 3, 10, 250
    ls, s, noise = 0.3, 1.2, 2e-2
    X = ci.points(41, n, d).astype(np.float32)
    B = ci.rhs(42, n, T).astype(np.float32)
    G = ci.rhs(43, n, T).astype(np.float32)
    X64 = X.astype(np.float64)
    K = kernels.dense_K(X64, kind, ls, s, noise)
    lam = np.linalg.eigvalsh(K)
    w, t = O.quad_nodes(noise, 1.05 * lam[-1], Q)
    A_o, gB_o, gth_o = VJP.ciq_vjp(K, VJP.dK_dtheta(X64, kind, ls, s), B, G, w, t, op, max_iter=J)
    fn = P.ciq_invsqrt_vjp if op == "invsqrt" else P.ciq_sqrt_vjp
    k = P.Kernel(kind, ls, s, noise)
    out, gB, gth, info = fn(torch.from_numpy(X).cuda(), k, torch.from_numpy(B).cuda(), torch.from_numpy(G).cuda(),
                            Q, 0.0, max_iter=J, nodes=(w, t), lmin=noise, precision=precision)
    assert info["iters"] == J and info["krylov"] == "basis"
    # FP32 kernel entries: within 15 times the oracle's own change when K's
    # entries are rounded to FP32 (relerr.fp32_gate; the forward parity tests'
    # convention), at least 2e-5; FP16-split tiles add 1e-4.
    BG = np.concatenate([B, G]).astype(np.float64)
    ref = np.concatenate([A_o, gB_o])
    tol, floor = fp32_gate(lambda Km: O.ciq_apply(O.dense_mvm(Km), BG, Q, op, max_iter=J, nodes=(w, t),
                                                  lmin=noise)[0], K, ref, least=2e-5)
    if precision == "fp16":
        tol = max(tol, 1e-4)
    e_out, e_gb = rel(out.cpu().numpy(), A_o), rel(gB.cpu().numpy(), gB_o)
    assert e_out < tol and e_gb < tol, (e_out, e_gb, tol, floor)
    np.testing.assert_allclose(gth, gth_o, rtol=10 * tol, atol=10 * tol * np.abs(gth_o).max())


def test_vjp_host_arrays_and_unsupported_forms():
    n, T = 300, 2
    X = ci.points(5, n, 2).astype(np.float32)
    B = ci.rhs(6, n, T).astype(np.float32)
    G = ci.rhs(7, n, T).astype(np.float32)
    k = P.Kernel("rbf", 0.4, 1.0, 1e-2)
    out, gB, gth, info = P.ciq_invsqrt_vjp(X, k, B, G, 8, 1e-6, max_iter=400)          # host arrays
    ref, _ = P.ciq_invsqrt(X, k, B, 8, 1e-6, max_iter=400)
    assert rel(out, ref) < 1e-5 and np.isfinite(gth).all()
    gref, _ = P.ciq_invsqrt(X, k, G, 8, 1e-6, max_iter=400)                              # dL/dB = K^{-1/2} G
    assert rel(gB, gref) < 1e-5
    for bad in (dict(krylov="recurrence"), dict(sqrt_form="mvm")):
        with pytest.raises(P.CiqError) as e:
            (P.ciq_sqrt_vjp if "sqrt_form" in bad else P.ciq_invsqrt_vjp)(X, k, B, G, 8, 1e-6, **bad)
        assert e.value.status == 6


@pytest.mark.parametrize("T,Q", [(1, 1), (40, 6)])
def test_vjp_edge_shapes(T, Q):
    # one column and one shift; and 2T = 80 columns (two tensor-core groups)
    n = 500
    X = ci.points(8, n, 4).astype(np.float32)
    B = ci.rhs(9, n, T).astype(np.float32)
    G = ci.rhs(10, n, T).astype(np.float32)
    ls, s, noise = 0.5, 0.9, 5e-2
    K = kernels.dense_K(X.astype(np.float64), "matern52", ls, s, noise)
    lam = np.linalg.eigvalsh(K)
    w, t = O.quad_nodes(noise, 1.05 * lam[-1], Q)
    J = 150
    A_o, gB_o, gth_o = VJP.ciq_vjp(K, VJP.dK_dtheta(X.astype(np.float64), "matern52", ls, s), B, G, w, t, "sqrt",
                                   max_iter=J)
    out, gB, gth, info = P.ciq_sqrt_vjp(torch.from_numpy(X).cuda(), P.Kernel("matern52", ls, s, noise),
                                        torch.from_numpy(B).cuda(), torch.from_numpy(G).cuda(), Q, 0.0,
                                        max_iter=J, nodes=(w, t), lmin=noise, precision="fp16")
    assert rel(out.cpu().numpy(), A_o) < 1e-4 and rel(gB.cpu().numpy(), gB_o) < 1e-4
    np.testing.assert_allclose(gth, gth_o, rtol=1e-3, atol=1e-3 * np.abs(gth_o).max())
