"""The host eigensolver used by the preconditioner setup (csrc/symeig.h,
header-only C++) against LAPACK: built here with g++ into a throwaway shared
object and called on matrices like the Gram matrix L^T L of a pivoted
Cholesky factor (eigenvalues spanning many decades), on tiny and ragged sizes
and on exactly repeated eigenvalues."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import ciq_inputs as ci
from oracle import kernels
from oracle import precond as PC

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2006_11267_b300", "csrc")


@pytest.fixture(scope="module")
def eigh_lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("symeig")
    src = d / "shim.cpp"
    src.write_text('#include "symeig.h"\n'
                   'extern "C" int shim_eigh(int n, double* A, double* w, double* Z) '
                   '{ return ciq::symeig::eigh(n, A, w, Z) ? 0 : 1; }\n')
    so = d / "shim.so"
    subprocess.run(["g++", "-O2", "-shared", "-fPIC", "-pthread", "-I", CSRC, str(src), "-o", str(so)], check=True)
    return ctypes.CDLL(str(so))


def _eigh(lib, A):
    n = A.shape[0]
    Ac = np.asfortranarray(A.copy())
    w = np.zeros(n)
    Z = np.zeros((n, n), order="F")
    P = ctypes.c_void_p
    rc = lib.shim_eigh(n, P(Ac.ctypes.data), P(w.ctypes.data), P(Z.ctypes.data))
    assert rc == 0
    return w, Z


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 129, 300])
def test_symeig_matches_lapack_on_graded_spd_matrices(eigh_lib, n):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    A = (M * np.logspace(0, -4, n)[None, :]) @ M.T
    A = 0.5 * (A + A.T)
    w, Z = _eigh(eigh_lib, A)
    ref = np.linalg.eigvalsh(A)
    assert np.abs(w - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(Z.T @ Z - np.eye(n)).max() < 1e-12
    assert np.abs(Z @ np.diag(w) @ Z.T - A).max() < 1e-12 * np.abs(A).max()


def test_symeig_on_a_pivoted_cholesky_gram_matrix_and_repeated_eigenvalues(eigh_lib):
    X = ci.points(3, 400, 3)
    Kxx = kernels.kernel_matrix(X, X, "rbf", 0.3, 1.0)
    L, _ = PC.pivoted_cholesky(np.diag(Kxx), lambda i: Kxx[:, i], 120)
    G = L.T @ L
    w, Z = _eigh(eigh_lib, G)
    ref = np.linalg.eigvalsh(G)
    assert np.abs(w - ref).max() <= 1e-12 * ref.max()
    assert np.abs(Z @ np.diag(w) @ Z.T - G).max() < 1e-12 * np.abs(G).max()
    # Exactly repeated eigenvalues: any orthonormal basis of each eigenspace.
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((40, 40)))
    lam = np.repeat([1.0, 2.0, 5.0, 5.0], 10)
    A = (Q * lam) @ Q.T
    w, Z = _eigh(eigh_lib, 0.5 * (A + A.T))
    assert np.abs(w - np.sort(lam)).max() < 1e-13 * 5
    assert np.abs(Z.T @ Z - np.eye(40)).max() < 1e-13
    assert np.abs(Z @ np.diag(w) @ Z.T - A).max() < 1e-13 * 5
