"""Pins for the CPU oracle (no GPU).

Every check here is independent of the oracle's own arithmetic: closed forms,
brute force on tiny inputs (a Python cyclic Jacobi and singular values of
A - lambda B), pairs with constructed spectra, residual identities of the
definition (Algorithm 1), reconstructions of each stage, and a cross-check
against an independent library (LAPACK via scipy).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_1207_1773_gb300 import inputs

EPS = np.finfo(np.float64).eps
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ratios(A, B, w, X):
    n = A.shape[0]
    res = np.linalg.norm(A @ X - (B @ X) * w[None, :]) / (
        max(n, 1) * EPS * np.linalg.norm(A) * max(np.linalg.norm(X), 1e-300))
    orth = np.linalg.norm(X.conj().T @ B @ X - np.eye(X.shape[1])) / (max(n, 1) * EPS)
    return res, orth


def _eig_tol(A, B):
    n = A.shape[0]
    return 10 * n * EPS * np.linalg.norm(A, 2) / np.linalg.eigvalsh(B).min()


def _jacobi_eigvals(H, sweeps=60):
    """Cyclic complex Jacobi on a small Hermitian matrix (brute force)."""
    H = np.array(H, dtype=np.complex128)
    n = H.shape[0]
    for _ in range(sweeps):
        off = np.sqrt(np.sum(np.abs(H - np.diag(np.diag(H))) ** 2))
        if off < 1e-300 or off < 1e-15 * np.linalg.norm(H):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                hpq = H[p, q]
                if abs(hpq) == 0.0:
                    continue
                # unitary 2x2 rotation zeroing H[p,q]: first make it real
                phase = hpq / abs(hpq)
                a, b, c = H[p, p].real, abs(hpq), H[q, q].real
                theta = 0.5 * math.atan2(2 * b, a - c)
                cs, sn = math.cos(theta), math.sin(theta)
                J = np.eye(n, dtype=np.complex128)
                J[p, p] = cs
                J[q, q] = cs
                J[p, q] = -sn * phase
                J[q, p] = sn * np.conj(phase)
                H = J.conj().T @ H @ J
    return np.sort(np.diag(H).real)


def test_closed_form_2x2():
    rows = {}
    with open(os.path.join(GOLDEN, "closed_form_2x2.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            rows[key] = [float(v) for v in vals]
    A = np.array(rows["A"][0::2]) + 1j * np.array(rows["A"][1::2])
    B = np.array(rows["B"][0::2]) + 1j * np.array(rows["B"][1::2])
    A, B = A.reshape(2, 2), B.reshape(2, 2)
    w, X, info = oracle.hegv(A, B)
    assert info == 0
    np.testing.assert_allclose(w, rows["lambda"], rtol=0, atol=1e-14)
    res, orth = _ratios(A, B, w, X)
    assert res < 30 and orth < 30


def test_n1_closed_form():
    w, X, info = oracle.hegv(np.array([[3.0 + 0j]]), np.array([[4.0 + 0j]]))
    assert info == 0
    assert abs(w[0] - 0.75) < 1e-15
    assert abs(abs(X[0, 0]) - 0.5) < 1e-15


@pytest.mark.parametrize("n", [2, 3, 4, 5, 7, 8])
@pytest.mark.parametrize("seed", [0, 1])
def test_brute_force_tiny(n, seed):
    A, B, _ = inputs.make_pair(n, 100 + seed)
    # perturb A off the constructed family so the test does not rely on it
    rng = np.random.default_rng(seed + 7)
    P = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = A + 0.3 * (P + P.conj().T)
    w, X, info = oracle.hegv(A, B)
    assert info == 0
    Lnp = np.linalg.cholesky(B)
    Ap = np.linalg.solve(Lnp, np.linalg.solve(Lnp, A).conj().T).conj().T
    wj = _jacobi_eigvals(0.5 * (Ap + Ap.conj().T))
    tol = _eig_tol(A, B)
    assert np.max(np.abs(w - wj)) < tol
    scale = np.linalg.norm(A, 2) + np.abs(w).max() * np.linalg.norm(B, 2)
    for lam in w:
        smin = np.linalg.svd(A - lam * B, compute_uv=False).min()
        assert smin < 1e3 * n * EPS * scale


@pytest.mark.parametrize("n,seed", [(17, 0), (64, 1), (100, 2), (200, 3), (256, 0)])
def test_known_spectrum_and_residuals(n, seed):
    A, B, lam = inputs.make_pair(n, seed)
    w, X, info = oracle.hegv(A, B)
    assert info == 0
    assert np.all(np.diff(w) >= 0)
    assert np.max(np.abs(w - lam)) < _eig_tol(A, B)
    res, orth = _ratios(A, B, w, X)
    assert res < 30, res
    assert orth < 30, orth


def test_clustered_and_illconditioned():
    n = 160
    A, B, lam = inputs.make_pair(n, 5, "clustered", -1, 1, ldiag="loguniform")
    w, X, info = oracle.hegv(A, B)
    assert info == 0
    assert np.max(np.abs(w - lam)) < _eig_tol(A, B)
    res, orth = _ratios(A, B, w, X)
    assert res < 100
    # B-orthonormality degrades with cond(B); scale by it (generalized bound)
    condB = np.linalg.cond(B)
    assert orth < 30 * condB


def test_library_crosscheck():
    n = 120
    A, B, _ = inputs.make_pair(n, 9, "uniform", -10, 10)
    w, X, info = oracle.hegv(A, B)
    ws, Xs = sl.eigh(A, B)
    assert np.max(np.abs(w - ws)) < _eig_tol(A, B)
    # eigenvectors agree up to a unit phase (spectrum is well separated)
    for j in range(n):
        ph = np.vdot(Xs[:, j], X[:, j])
        ph /= abs(ph)
        assert np.linalg.norm(X[:, j] - ph * Xs[:, j]) < 1e-9 * np.linalg.norm(Xs[:, j])


@pytest.mark.parametrize("il,iu", [(1, 1), (1, 26), (10, 40), (60, 64), (1, 64)])
def test_subset_selector(il, iu):
    n = 64
    A, B, lam = inputs.make_pair(n, 4)
    w_all, X_all, _ = oracle.hegv(A, B)
    w, X, info = oracle.hegv(A, B, il, iu)
    assert info == 0 and w.shape == (iu - il + 1,)
    np.testing.assert_array_equal(w, w_all[il - 1:iu])
    for j in range(iu - il + 1):
        ph = np.vdot(X_all[:, il - 1 + j], B @ X[:, j])  # B-inner product
        assert abs(abs(ph) - 1) < 1e-10


def test_special_cases():
    n = 9
    rng = np.random.default_rng(3)
    dg = rng.uniform(-5, 5, n)
    A = np.diag(dg).astype(np.complex128)
    B = np.eye(n, dtype=np.complex128)
    w, X, info = oracle.hegv(A, B)
    np.testing.assert_allclose(w, np.sort(dg), atol=1e-14)
    # eigenvectors are unit vectors (up to phase) at the sorted positions
    np.testing.assert_allclose(np.abs(X), np.eye(n)[:, np.argsort(dg)], atol=1e-14)
    # B = I: hegst is the identity on a Hermitian A
    A2, _, _ = inputs.make_pair(n, 5)
    Ap = oracle.hegst(A2, np.eye(n))
    np.testing.assert_allclose(Ap, A2, atol=1e-14)


def test_error_paths():
    n = 6
    A, B, _ = inputs.make_pair(n, 0)
    Bbad = B.copy()
    Bbad[3, 3] = -1.0
    _, _, info = oracle.hegv(A, Bbad)
    assert 1 <= info <= 4
    _, info2 = oracle.potrf(-np.eye(3, dtype=np.complex128))
    assert info2 == 1
    _, _, info3 = oracle.hegv(A, B, 3, 9)
    assert info3 == -1


def test_stage_potrf_and_hegst():
    n = 50
    A, B, _ = inputs.make_pair(n, 11)
    L, info = oracle.potrf(B)
    assert info == 0
    np.testing.assert_allclose(L, np.linalg.cholesky(B), atol=1e-12)
    assert np.linalg.norm(L @ L.conj().T - B) < 50 * n * EPS * np.linalg.norm(B)
    Ap = oracle.hegst(A, L)
    assert np.linalg.norm(Ap - Ap.conj().T) == 0.0
    assert np.linalg.norm(L @ Ap @ L.conj().T - A) < 100 * n * EPS * np.linalg.norm(A) * np.linalg.cond(L)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 64])
def test_stage_hetrd_reconstruction(n):
    A, _, _ = inputs.make_pair(n, 12)
    d, e, V, tau = oracle.hetrd(A)
    Q = oracle.unmtr(V, tau, np.eye(n, dtype=np.complex128))
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(n)) < 20 * n * EPS
    T = np.diag(d) + np.diag(e, -1) + np.diag(e, 1)
    assert np.linalg.norm(Q @ T @ Q.conj().T - A) < 20 * n * EPS * np.linalg.norm(A)
    # first reflector leaves e real and the invariants trace / Frobenius norm
    assert abs(np.trace(A).real - d.sum()) < 20 * n * EPS * np.linalg.norm(A)


@pytest.mark.parametrize("n", [1, 2, 5, 40, 150])
def test_stage_steqr(n):
    rng = np.random.default_rng(n)
    d = rng.standard_normal(n)
    e = rng.standard_normal(max(n - 1, 0))
    if n > 10:
        e[n // 3] = 0.0  # a split
        d[n // 2:n // 2 + 3] = 0.25  # repeated diagonal values
    w, Z, info = oracle.steqr(d, e)
    assert info == 0
    w, Z = oracle.sort_eig(w, Z)
    T = np.diag(d) + np.diag(e, -1) + np.diag(e, 1)
    ref = sl.eigvalsh_tridiagonal(d, e) if n > 1 else d
    nt = max(np.linalg.norm(T, 2), 1e-300)
    assert np.max(np.abs(w - ref)) < 10 * n * EPS * nt
    assert np.linalg.norm(T @ Z - Z * w[None, :]) < 20 * n * EPS * nt
    assert np.linalg.norm(Z.T @ Z - np.eye(n)) < 20 * n * EPS


def test_stage_trsm():
    n, m = 40, 7
    _, B, _ = inputs.make_pair(n, 13)
    L = np.linalg.cholesky(B)
    rng = np.random.default_rng(1)
    Y = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    X = oracle.trsm_lh(L, Y)
    assert np.linalg.norm(L.conj().T @ X - Y) < 50 * n * EPS * np.linalg.norm(L) * np.linalg.norm(X)
