"""CPU replays (numpy) of two algebraic rearrangements the CUDA path relies
on, checked against the plain sequential definitions:

* the back-transform's Q2 schedule: reflectors of nb consecutive sweeps at
  one chase step merged into block reflectors, pairs of sweep groups merged
  again (T12 = -T1 V1^H V2 T2), blocks applied in wavefront order; and the
  explicit formation of Q2 from the identity in which a block of pair c
  touches only columns >= 2 c nb + 1 (everything left of that is zero in its
  rows when it is applied);
* the panel QR's single reduction per column: sums over the unscaled column x
  and the pivot row, with v = (x - beta e_j) / (alpha - beta) in the
  library's Householder convention (real beta = -sign(Re alpha) |x|).
Both are exact rearrangements, so the replay must agree to rounding."""
import numpy as np
import pytest


def _reflectors(n, nb, rng):
    J = (n - 1 + nb - 1) // nb
    V2 = np.zeros((n, J, nb), complex)
    tau2 = np.zeros((n, J), complex)
    for s in range(n - 1):
        for j in range((n - 1 - s + nb - 1) // nb):
            a = s + 1 + j * nb
            L = min(nb, n - a)
            v = rng.standard_normal(L) + 1j * rng.standard_normal(L)
            v[0] = 1
            V2[s, j, :L] = v
            tau2[s, j] = 2 / np.vdot(v, v).real * (0.9 + 0.1j)
    return J, V2, tau2


def _sequential(n, nb, V2, tau2, Z):
    X = Z.copy()
    for s in range(n - 2, -1, -1):            # Q2 = H(0) H(1) ... H(n-2)
        for j in range((n - 1 - s + nb - 1) // nb):
            a = s + 1 + j * nb
            L = min(nb, n - a)
            v, t = V2[s, j, :L], tau2[s, j]
            X[a:a + L] -= t * np.outer(v, v.conj() @ X[a:a + L])
    return X


def _diamond(n, nb, V2, tau2, b, j):
    W2, s0, r0 = 2 * nb, b * nb, (b + j) * nb + 1
    V = np.zeros((W2, nb), complex)
    tau = np.zeros(nb, complex)
    for c in range(nb):
        s = s0 + c
        if s <= n - 2 and j < (n - 1 - s + nb - 1) // nb:
            a = s + 1 + j * nb
            L = min(nb, n - a)
            for i in range(W2):
                if c <= i < c + L and r0 + i < n:
                    V[i, c] = V2[s, j, i - c]
            tau[c] = tau2[s, j]
    G = V.conj().T @ V
    T = np.zeros((nb, nb), complex)
    for c in range(nb):
        T[:c, c] = -tau[c] * (T[:c, :c] @ G[:c, c])
        T[c, c] = tau[c]
    return V, T


def _wavefront(n, nb, J, V2, tau2, Y, form_q):
    C = (J + 1) // 2
    for w in range(C + J - 1):
        for c in range(max(0, C - 1 - w), C):
            j = w - (C - 1 - c)
            if j < 0 or j >= J - 2 * c:
                break
            V1, T1 = _diamond(n, nb, V2, tau2, 2 * c, j)
            W3 = 3 * nb
            V = np.zeros((W3, 2 * nb), complex)
            V[:2 * nb, :nb] = V1
            T = np.zeros((2 * nb, 2 * nb), complex)
            T[:nb, :nb] = T1
            if 2 * c + 1 < J and j < J - (2 * c + 1):
                V2b, T2 = _diamond(n, nb, V2, tau2, 2 * c + 1, j)
                V[nb:, nb:] = V2b
                T[:nb, nb:] = -T1 @ (V1[nb:2 * nb].conj().T @ V2b[:nb]) @ T2
                T[nb:, nb:] = T2
            U = V @ T
            r0 = (2 * c + j) * nb + 1
            Wh = min(W3 - 1, n - r0)
            lo = 2 * c * nb + 1 if form_q else 0
            if form_q:
                assert np.all(Y[r0:r0 + Wh, :lo] == 0)
            Xw = Y[r0:r0 + Wh, lo:]
            Wt = Xw.conj().T @ V[:Wh]
            Y[r0:r0 + Wh, lo:] = Xw - U[:Wh] @ Wt.conj().T
    return Y


@pytest.mark.parametrize("n,nb", [(40, 4), (57, 4), (64, 8), (100, 8), (33, 3), (130, 16)])
def test_q2_merged_wavefront_and_explicit_form(n, nb):
    rng = np.random.default_rng(n * 100 + nb)
    J, V2, tau2 = _reflectors(n, nb, rng)
    Z = rng.standard_normal((n, 5)) + 0j
    X = _sequential(n, nb, V2, tau2, Z)
    Y = _wavefront(n, nb, J, V2, tau2, Z.copy(), False)
    scale = np.abs(X).max()
    assert np.abs(X - Y).max() / scale < 1e-13
    Q = _wavefront(n, nb, J, V2, tau2, np.eye(n, dtype=complex), True)
    assert np.abs(X - Q @ Z).max() / scale < 1e-13


def _panel_one_reduction(P, kr):
    P = P.copy()
    mp, nb = P.shape
    T = np.zeros((nb, nb), complex)
    for j in range(kr):
        x = P[:, j].copy()
        xn2 = np.sum(np.abs(x[j + 1:]) ** 2)
        al = x[j]
        D = [np.vdot(x[j:], P[j:, c]) if c > j else 0 for c in range(nb)]
        Gs = [np.vdot(P[j:, c], x[j:]) if c < j else 0 for c in range(nb)]
        row = P[j, :].copy()
        if xn2 == 0 and al.imag == 0:
            t, beta, s = 0, al.real, 0
        else:
            nrm = np.sqrt(abs(al) ** 2 + xn2)
            beta = -nrm if al.real >= 0 else nrm
            t, s = complex((beta - al.real) / beta, -al.imag / beta), 1 / (al - beta)
        cw = [np.conj(t) * np.conj(s) * (D[c] - beta * row[c]) if c > j else 0 for c in range(nb)]
        vv = [s * (Gs[c] - beta * np.conj(row[c])) if c < j else 0 for c in range(nb)]
        P[j + 1:, j] *= s
        P[j, j] = beta
        v = np.zeros(mp, complex)
        v[j] = 1
        v[j + 1:] = P[j + 1:, j]
        for c in range(j + 1, nb):
            P[j:, c] -= v[j:] * cw[c]
        for r in range(j):
            T[r, j] = -t * np.sum(T[r, r:j] * np.array(vv[r:j]))
        T[j, j] = t
    return P, T


@pytest.mark.parametrize("mp,nb", [(50, 8), (200, 16), (33, 8), (7, 8)])
def test_panel_qr_single_reduction(mp, nb):
    rng = np.random.default_rng(mp + nb)
    A = rng.standard_normal((mp, nb)) + 1j * rng.standard_normal((mp, nb))
    kr = min(nb, mp)
    P, T = _panel_one_reduction(A, kr)
    V = np.tril(P[:, :kr], -1)
    V[np.arange(kr), np.arange(kr)] = 1
    Q = np.eye(mp) - V @ T[:kr, :kr] @ V.conj().T
    assert np.abs(Q @ np.triu(P) - A).max() / np.abs(A).max() < 1e-13
    assert np.abs(Q.conj().T @ Q - np.eye(mp)).max() < 1e-13
    assert np.abs(np.diag(P[:kr, :kr]).imag).max() == 0       # real beta on the diagonal
    # the same factor as numpy's QR up to unit-modulus column phases
    R = np.linalg.qr(A, mode="r")
    assert np.allclose(np.abs(np.diag(R)[:kr]), np.abs(np.diag(P)[:kr]), rtol=1e-12)
