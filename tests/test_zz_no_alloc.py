"""The allocation-free kernel MVM against the allocating one, through the C ABI.

For callers that cannot call cudaMalloc the library offers
ciq_kernel_mvm_noalloc, whose scratch is a static device array.  This file is
collected last so that a run stopping at the first failure has run every
other test first.  The comparison tolerance is the one of the kernel-MVM
parity tests (2e-6 relative, Frobenius).
"""
import ctypes

import numpy as np
import pytest
import torch

import ciq_inputs as ci
import paper_2006_11267_b300 as P
from paper_2006_11267_b300 import _ciq

pytestmark = pytest.mark.gpu


def _case(n, d, t, seed, kind):
    X = torch.from_numpy(np.asarray(ci.points(seed, n, d), np.float32)).cuda()
    V = torch.from_numpy(np.asarray(ci.rhs(seed, n, t), np.float32)).cuda()
    return X, V, P.Kernel(kind, 0.3, 1.2, 1e-3)


def _rel(a, b):
    # Largest relative 2-norm error over the right-hand sides (rows).
    a = a.double()
    b = b.double()
    return float((torch.linalg.norm(a - b, dim=1) / torch.linalg.norm(b, dim=1)).max())


def test_noalloc_mvm_matches_allocating_mvm_on_consecutive_calls():
    # Two different problems in a row (the second smaller, so stale scratch
    # from the first would show up in its padded rows), then the first again.
    cases = [_case(3000, 6, 17, 1, "rbf"), _case(1000, 3, 8, 2, "matern52"), _case(3000, 6, 17, 1, "rbf")]
    for X, V, k in cases:
        ref = P.ciq_kernel_mvm(X, k, V)
        out = torch.full_like(V, float("nan"))
        P.ciq_kernel_mvm_noalloc(X, k, V, out=out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) < 2e-6


def test_noalloc_rejects_problems_larger_than_its_scratch():
    cap = int(P.lib().ciq_noalloc_scratch_floats())
    assert cap == 4 << 20
    n = 200_000                                  # 200,064 rows x (8 + 64) floats > 4 Mi floats
    k = _ciq.Kernel("rbf", 0.3, 1.0, 1e-3).c()
    X = torch.zeros((n, 6), device="cuda")
    V = torch.zeros((64, n), device="cuda")
    out = torch.zeros((64, n), device="cuda")
    st = P.lib().ciq_kernel_mvm_noalloc(ctypes.c_void_p(X.data_ptr()), n, 6, ctypes.byref(k),
                                        ctypes.c_void_p(V.data_ptr()), 64, ctypes.c_void_p(out.data_ptr()), None)
    assert st == _ciq.CIQ_ERR_SCRATCH_TOO_SMALL
    assert float(out.abs().max()) == 0.0
