"""Batched msMINRES-CIQ (ciq_sqrt_batched / ciq_invsqrt_batched) on the GPU.

The batched call runs every problem's arithmetic with the same device bodies
and block decomposition as the single-problem call, so its outputs must
equal ciq_sqrt / ciq_invsqrt bit for bit (same options, same bounds), and
through them the FP64 oracle within the single path's tolerances.
"""
import numpy as np
import pytest
import torch

import ciq_inputs as ci
import paper_2006_11267_b300 as P
from oracle import ciq as O
from oracle import kernels
from relerr import fp32_gate, rel

pytestmark = pytest.mark.gpu

DEV = "cuda"


def recipe_problems(seed, count, t=8):
    """Problems of the uneven-batch recipe as device tensors."""
    out = []
    for pr in ci.batched_problems(seed, count=count, t=t):
        out.append(dict(X=torch.from_numpy(pr["X"].astype(np.float32)).to(DEV),
                        B=torch.from_numpy(pr["B"].astype(np.float32)).to(DEV),
                        kernel=P.Kernel(pr["kernel"], pr["lengthscale"], pr["outputscale"], pr["noise"])))
    return out


def hand_problem(n, d, t, seed, kind, ls, noise):
    return dict(X=torch.from_numpy(ci.points(seed, n, d).astype(np.float32)).to(DEV),
                B=torch.from_numpy(ci.rhs(seed, n, t).astype(np.float32)).to(DEV),
                kernel=P.Kernel(kind, ls, 1.0, noise))


def single(op, pr, Q, tol, **opts):
    # batched solves run the direction recurrence; the single call is asked for it
    opts = dict(opts, krylov="recurrence")
    fn = P.ciq_sqrt if op == "sqrt" else P.ciq_invsqrt
    if pr.get("lmin"):
        opts = dict(opts, lmin=pr["lmin"], lmax=pr["lmax"])
    return fn(pr["X"], pr["kernel"], pr["B"], Q, tol, **opts)


def batched(op, probs, Q, tol, **opts):
    fn = P.ciq_sqrt_batched if op == "sqrt" else P.ciq_invsqrt_batched
    return fn(probs, Q, tol, **opts)


@pytest.mark.parametrize("op", ["sqrt", "invsqrt"])
def test_batched_equals_single_calls_bit_for_bit(op):
    probs = recipe_problems(31, 12)
    outs, infos = batched(op, probs, 8, 1e-4, max_iter=400)
    assert len(outs) == len(probs)
    for pr, out, info in zip(probs, outs, infos):
        ref, rinfo = single(op, pr, 8, 1e-4, max_iter=400)
        assert torch.equal(out, ref), (pr["X"].shape, pr["kernel"])
        for key in ("iters", "iters_min", "converged", "lanczos_iters"):
            assert info[key] == rinfo[key], key
        for key in ("lmin_used", "lmax_used", "ritz_min", "ritz_max", "resid_max"):
            assert info[key] == rinfo[key], key
        np.testing.assert_array_equal(info["w"], rinfo["w"])
        np.testing.assert_array_equal(info["t"], rinfo["t"])


def test_batched_given_bounds_mixed_with_prepass():
    probs = recipe_problems(32, 10)
    for i, pr in enumerate(probs):
        if i % 2 == 0:
            b = P.ciq_lanczos_bounds(pr["X"], pr["kernel"], iters=10)
            pr["lmin"], pr["lmax"] = b["lmin_used"], b["lmax_used"] * 1.1
    outs, infos = batched("invsqrt", probs, 8, 1e-4, max_iter=400)
    for i, (pr, out, info) in enumerate(zip(probs, outs, infos)):
        ref, rinfo = single("invsqrt", pr, 8, 1e-4, max_iter=400)
        assert torch.equal(out, ref)
        assert info["iters"] == rinfo["iters"]
        if i % 2 == 0:
            assert info["lanczos_iters"] == 0
            assert info["lmax_used"] == pr["lmax"]
        else:
            assert info["lanczos_iters"] == 10


@pytest.mark.parametrize("op", ["sqrt", "invsqrt"])
def test_batched_matches_serial_oracle_at_equal_nodes_and_J(op):
    specs = [(200, 2, "rbf", 0.3, 5e-2), (333, 5, "matern52", 0.4, 2e-2), (517, 9, "rbf", 0.8, 1e-1),
             (700, 12, "matern52", 0.6, 3e-2)]
    Q, J, T = 8, 500, 3
    probs, refs, gates = [], [], []
    for n, d, kind, ls, noise in specs:
        pr = hand_problem(n, d, T, 900 + n, kind, ls, noise)
        X = pr["X"].cpu().numpy().astype(np.float64)
        K = kernels.dense_K(X, kind, ls, 1.0, noise)
        lam = np.linalg.eigvalsh(K)
        pr["lmin"], pr["lmax"] = noise, 1.05 * lam[-1]
        nodes = O.quad_nodes(pr["lmin"], pr["lmax"], Q)
        Bp = pr["B"].cpu().numpy().astype(np.float64)
        run = (lambda Km, Bp=Bp, nodes=nodes, noise=noise:
               O.ciq_apply(O.dense_mvm(Km), Bp, Q, op, tol=0.0, max_iter=J, nodes=nodes, lmin=noise, lmax=None)[0])
        ref, info_o = O.ciq_apply(O.dense_mvm(K), Bp, Q, op, tol=0.0, max_iter=J, nodes=nodes, lmin=noise, lmax=None)
        assert np.max(info_o["errbound"] / np.linalg.norm(ref, axis=1)) < 1e-9
        probs.append(pr)
        refs.append(ref)
        gates.append(fp32_gate(run, K, ref))
    outs, infos = batched(op, probs, Q, 0.0, max_iter=J)
    for out, ref, info, (tol, floor) in zip(outs, refs, infos, gates):
        assert info["iters"] == J
        err = rel(out.cpu().numpy(), ref)
        assert err < tol, (err, tol, floor)


def test_batched_edge_cases():
    # one point, a zero right-hand side, d = 1 and d = 16, both kernel types
    probs = [hand_problem(1, 3, 2, 1, "rbf", 0.5, 1e-2), hand_problem(129, 1, 2, 2, "matern52", 0.2, 1e-2),
             hand_problem(300, 16, 2, 3, "rbf", 2.0, 1e-3), hand_problem(257, 4, 2, 4, "matern52", 0.3, 1e-1)]
    probs[3]["B"][1].zero_()
    outs, infos = batched("sqrt", probs, 8, 1e-5, max_iter=300)
    for pr, out, info in zip(probs, outs, infos):
        ref, rinfo = single("sqrt", pr, 8, 1e-5, max_iter=300)
        assert torch.equal(out, ref)
        assert info["iters"] == rinfo["iters"]
    assert torch.count_nonzero(outs[3][1]) == 0
    # K = s + sigma^2 for one point: K^{1/2} b = sqrt(1.01) b
    np.testing.assert_allclose(outs[0].cpu().numpy(), np.sqrt(1.01) * probs[0]["B"].cpu().numpy(), rtol=1e-5)
    # a single problem, one right-hand side
    pr = hand_problem(600, 3, 1, 5, "rbf", 0.3, 1e-2)
    outs, infos = batched("invsqrt", [pr], 12, 1e-5, max_iter=300)
    ref, rinfo = single("invsqrt", pr, 12, 1e-5, max_iter=300)
    assert torch.equal(outs[0], ref) and infos[0]["iters"] == rinfo["iters"]


@pytest.mark.parametrize("t", [17, 40])
def test_batched_wide_tiles_equal_single(t):
    probs = [hand_problem(n, d, t, 40 + n, kind, 0.3, 1e-2)
             for n, d, kind in [(400, 3, "rbf"), (1000, 7, "matern52"), (130, 11, "rbf")]]
    outs, infos = batched("sqrt", probs, 8, 1e-4, max_iter=300)
    for pr, out, info in zip(probs, outs, infos):
        ref, rinfo = single("sqrt", pr, 8, 1e-4, max_iter=300)
        assert torch.equal(out, ref)
        assert info["iters"] == rinfo["iters"]


def test_batched_check_every_does_not_change_results():
    probs = recipe_problems(33, 6)
    a, ia = batched("invsqrt", probs, 8, 1e-4, max_iter=400, check_every=1)
    b, ib = batched("invsqrt", probs, 8, 1e-4, max_iter=400, check_every=16)
    for x, y, p, q in zip(a, b, ia, ib):
        assert torch.equal(x, y)
        assert p["iters"] == q["iters"]
    assert ia[0]["launches"] != ib[0]["launches"]


@pytest.mark.parametrize("prec,t", [("fp16", 8), ("bf16", 8), ("fp16", 40)])
def test_tensor_core_batch_equals_single_tensor_core_calls(prec, t):
    probs = recipe_problems(34, 7, t=t)
    probs.append(hand_problem(1, 3, t, 9, "rbf", 0.5, 1e-2))
    probs.append(hand_problem(300, 14, t, 10, "matern52", 0.8, 1e-2))
    outs, infos = batched("sqrt", probs, 8, 1e-4, max_iter=600, precision=prec)
    for pr, out, info in zip(probs, outs, infos):
        # batches use one CTA per row tile: the single call is asked for the same split
        ref, rinfo = single("sqrt", pr, 8, 1e-4, max_iter=600, precision=prec, tc_split=1)
        assert torch.equal(out, ref), (pr["X"].shape, pr["kernel"])
        assert info["iters"] == rinfo["iters"]


def test_tensor_core_batch_limits():
    too_wide = [hand_problem(200, 15, 4, 1, "rbf", 0.5, 1e-2)]
    with pytest.raises(P.CiqError) as e:
        batched("sqrt", too_wide, 8, 1e-4, precision="fp16")
    assert e.value.status == P._ciq.CIQ_ERR_UNSUPPORTED
    many = [hand_problem(200, 3, 65, 1, "rbf", 0.5, 1e-2)]
    with pytest.raises(P.CiqError) as e:
        batched("sqrt", many, 8, 1e-4, precision="fp16")
    assert e.value.status == P._ciq.CIQ_ERR_UNSUPPORTED


def test_split_policy_and_autotuner_change_only_the_summation_order(tmp_path):
    # Large problems split their row tiles over more CTAs (batch_split_rows /
    # batch_split): each problem's result stays within the stop rule's
    # accuracy of the default launch shape; the autotuner measures its
    # candidates once, stores the fastest and reuses it.
    from paper_2006_11267_b300 import autotune
    specs = [(300, 3, "rbf", 0.3, 1e-2), (2100, 4, "matern52", 0.4, 1e-2), (4200, 5, "rbf", 0.5, 1e-2)]
    probs = [hand_problem(n, d, 8, 700 + n, kind, ls, noise) for n, d, kind, ls, noise in specs]
    outs0, infos0 = batched("sqrt", probs, 8, 1e-5, max_iter=1000, precision="fp16")
    ref = [o.clone() for o in outs0]
    outs1, infos1 = batched("sqrt", probs, 8, 1e-5, max_iter=1000, precision="fp16", batch_split_rows=16,
                            batch_split=4)
    for a, b, i in zip(outs1, ref, infos1):
        assert i["status"] == 0
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-4
    path = str(tmp_path / "tune.json")
    best, timings = autotune.tune(probs, 8, 1e-5, path=path, max_iter=1000, precision="fp16")
    assert len(timings) == len(autotune.CANDIDATES) and best in autotune.CANDIDATES
    _, infos2 = autotune.solve_batched_tuned(probs, 8, 1e-5, path=path, max_iter=1000, precision="fp16")
    assert all(i["status"] == 0 for i in infos2)
