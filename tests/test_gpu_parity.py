"""GPU parity: the CUDA path (called through the C-ABI) against the CPU oracle.

Tolerances (floating point, FP64 throughout):
  eigenvalues   |w - w_oracle| <= 10 n eps ||A||_2 ||B^{-1}||_2
                (and against the constructed spectrum with the same bound);
  eigenvectors  residual ratio ||AX - BXW||_F / (n eps ||A||_F ||X||_F) <= 100,
                B-orthonormality ||X^H B X - I||_F / (n eps) <= 100 cond-scaled,
                and subspace agreement with the oracle per eigenvalue cluster:
                sin(angle) <= 1e4 n eps ||A'||/gap (Davis-Kahan style);
  stages        potrf/hegst/trsm/GEMM elementwise against the oracle or a
                direct definition with c n eps relative bounds.
"""
import numpy as np
import pytest

import oracle
from paper_1207_1773_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1207_1773_gb300 import gbhegv
    return gbhegv


DEV = "cuda:0"


def _c(x):
    from paper_1207_1773_gb300 import gbhegv
    return gbhegv.colmajor(x, DEV)


def _np(t):
    return t.detach().cpu().numpy()


def _rand(rng, m, n):
    return (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n)))


# ------------------------------------------------------------------ GEMM
@pytest.mark.parametrize("opA,opB", [("N", "N"), ("N", "C"), ("C", "N"), ("T", "T"), ("H", "N"), ("N", "T")])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (64, 64, 16), (65, 33, 17), (130, 70, 200), (37, 129, 1030)])
def test_zgemm(G, opA, opB, m, n, k):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    if opA == "H":
        k = m
    ra, ca = (m, k) if opA in ("N", "H") else (k, m)
    rb, cb = (k, n) if opB == "N" else (n, k)
    A = _rand(rng, ra, ca)
    B = _rand(rng, rb, cb)
    C = _rand(rng, m, n)
    alpha, beta = 0.7 - 0.2j, -0.3 + 0.5j
    if opA == "H":
        opa = np.tril(A) + np.tril(A, -1).conj().T
        opa = opa - 1j * np.diag(np.diag(opa).imag)
    else:
        opa = {"N": A, "T": A.T, "C": A.conj().T}[opA]
    opb = {"N": B, "T": B.T, "C": B.conj().T}[opB]
    ref = alpha * opa @ opb + beta * C
    Cd = _c(C)
    G.zgemm(opA, opB, _c(A), _c(B), Cd, alpha, beta)
    out = _np(Cd)
    scale = np.abs(opa) @ np.abs(opb) * abs(alpha) + abs(beta) * np.abs(C)
    assert np.all(np.abs(out - ref) <= 8 * (k + 2) * EPS * scale + 1e-300)


def test_zgemm_lower_only(G):
    rng = np.random.default_rng(5)
    n, k = 150, 40
    A = _rand(rng, n, k)
    C = _rand(rng, n, n)
    Cd = _c(C)
    G.zgemm("N", "C", _c(A), _c(A), Cd, -1.0, 1.0, lower=True)
    out = _np(Cd)
    ref = C - A @ A.conj().T
    low = np.tril(np.ones((n, n), bool))
    assert np.allclose(out[low], ref[low], rtol=0, atol=1e-12 * np.abs(ref).max())
    assert np.array_equal(out[~low], C[~low])


# ------------------------------------------------------------------ stages
@pytest.mark.parametrize("n", [1, 2, 7, 64, 65, 100, 257])
def test_potrf(G, n):
    _, B, _ = inputs.make_pair(n, 3)
    Bd = _c(B)
    info = G.potrf(Bd)
    assert info == 0
    L = np.tril(_np(Bd))
    Lo, info_o = oracle.potrf(B)
    assert info_o == 0
    assert np.linalg.norm(L - Lo) <= 50 * n * EPS * np.linalg.norm(Lo) * np.linalg.cond(Lo)


def test_potrf_not_pd(G):
    n = 100
    _, B, _ = inputs.make_pair(n, 3)
    B[70, 70] = -5.0
    Bd = _c(B)
    info = G.potrf(Bd)
    _, info_o = oracle.potrf(B)
    assert info == info_o and info > 0


@pytest.mark.parametrize("n", [1, 5, 64, 97, 200])
def test_hegst(G, n):
    A, B, _ = inputs.make_pair(n, 4)
    Lo, _ = oracle.potrf(B)
    Ao = oracle.hegst(A, Lo)
    Ad = _c(np.tril(A) + np.triu(np.full((n, n), np.nan + 0j), 1))  # upper must not be read
    G.hegst(Ad, _c(Lo))
    Ap = _np(Ad)
    assert np.linalg.norm(Ap - Ao) <= 100 * n * EPS * np.linalg.norm(Ao) * np.linalg.cond(Lo) ** 2


@pytest.mark.parametrize("n,m", [(1, 1), (10, 3), (64, 64), (130, 17), (200, 200)])
def test_trsm_lh(G, n, m):
    _, B, _ = inputs.make_pair(n, 5)
    Lo, _ = oracle.potrf(B)
    rng = np.random.default_rng(n)
    Y = _rand(rng, n, m)
    Xd = _c(Y)
    G.trsm_lh(_c(Lo), Xd)
    X = _np(Xd)
    Xo = oracle.trsm_lh(Lo, Y)
    assert np.linalg.norm(X - Xo) <= 100 * n * EPS * np.linalg.norm(Xo) * np.linalg.cond(Lo)


def _band_eigs(Ab, n, nb):
    Bm = np.zeros((n, n), complex)
    for c in range(n):
        for r in range(c, min(n, c + nb + 1)):
            Bm[r, c] = Ab[r, c]
    Bm = np.tril(Bm) + np.tril(Bm, -1).conj().T
    Bm -= 1j * np.diag(np.diag(Bm).imag)
    return np.linalg.eigvalsh(Bm), Bm


@pytest.mark.parametrize("n,nb", [(2, 1), (9, 4), (64, 16), (100, 32), (131, 8), (256, 32)])
def test_he2hb_band_spectrum(G, n, nb):
    A, _, _ = inputs.make_pair(n, 6)
    Ah = np.tril(A) + np.tril(A, -1).conj().T
    Ad = _c(Ah)
    T1, tau1 = G.he2hb(Ad, nb)
    wb, _ = _band_eigs(_np(Ad), n, nb)
    wo = np.sort(np.linalg.eigvalsh(Ah))
    assert np.max(np.abs(wb - wo)) <= 20 * n * EPS * np.linalg.norm(Ah, 2)


@pytest.mark.parametrize("n,nb", [(2, 1), (3, 2), (17, 4), (64, 16), (100, 7), (150, 32)])
def test_hb2st_spectrum(G, n, nb):
    rng = np.random.default_rng(n + nb)
    M = _rand(rng, n, n)
    H = M + M.conj().T
    mask = np.zeros((n, n), bool)
    for c in range(n):
        mask[c:min(n, c + nb + 1), c] = True
    Bl = np.where(mask, H, 0)
    Bm = np.tril(Bl) + np.tril(Bl, -1).conj().T
    Bm -= 1j * np.diag(np.diag(Bm).imag)
    Ad = _c(np.tril(Bm))
    d, e, V2, tau2 = G.hb2st(Ad, nb)
    d, e = _np(d), _np(e)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    wt = np.linalg.eigvalsh(T)
    wb = np.linalg.eigvalsh(Bm)
    assert np.max(np.abs(wt - wb)) <= 20 * n * EPS * np.linalg.norm(Bm, 2)


@pytest.mark.parametrize("n", [1, 2, 5, 32, 33, 64, 100, 257, 600])
def test_stedc_vs_oracle(G, n):
    rng = np.random.default_rng(n)
    d = rng.standard_normal(n)
    e = rng.standard_normal(max(n - 1, 0))
    w, Z = G.stedc(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV))
    w, Z = _np(w), _np(Z)
    wo, Zo, info = oracle.steqr(d, e)
    wo, Zo = oracle.sort_eig(wo, Zo)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    nt = max(np.linalg.norm(T, 2), 1e-300)
    assert np.max(np.abs(w - wo)) <= 10 * n * EPS * nt
    assert np.linalg.norm(T @ Z - Z * w[None, :]) <= 50 * n * EPS * nt
    assert np.linalg.norm(Z.T @ Z - np.eye(n)) <= 50 * n * EPS


def test_stedc_deflation_cases(G):
    n = 300
    rng = np.random.default_rng(1)
    d = np.repeat(rng.standard_normal(n // 10), 10)  # repeated values
    e = rng.standard_normal(n - 1) * 1e-3
    e[::7] = 0.0  # splits
    w, Z = G.stedc(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV))
    w, Z = _np(w), _np(Z)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    nt = np.linalg.norm(T, 2)
    assert np.max(np.abs(w - np.linalg.eigvalsh(T))) <= 10 * n * EPS * nt
    assert np.linalg.norm(T @ Z - Z * w[None, :]) <= 50 * n * EPS * nt
    assert np.linalg.norm(Z.T @ Z - np.eye(n)) <= 50 * n * EPS
    # diagonal matrix: everything deflates
    d2 = rng.standard_normal(200)
    w2, Z2 = G.stedc(torch.tensor(d2, device=DEV), torch.zeros(199, dtype=torch.float64, device=DEV))
    # exact up to the two roundings of the internal scaling by max |T|
    assert np.all(np.abs(_np(w2) - np.sort(d2)) <= 4 * EPS * np.abs(d2).max())


@pytest.mark.parametrize("il,iu", [(1, 40), (100, 180), (250, 300)])
def test_stedc_subset(G, il, iu):
    n = 300
    rng = np.random.default_rng(2)
    d = rng.standard_normal(n)
    e = rng.standard_normal(n - 1)
    wa, Za = G.stedc(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV))
    w, Z = G.stedc(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), il, iu)
    np.testing.assert_allclose(_np(w), _np(wa)[il - 1:iu], rtol=0, atol=1e-13)
    dots = np.abs(np.sum(_np(Z) * _np(Za)[:, il - 1:iu], axis=0))
    assert np.all(np.abs(dots - 1) < 1e-10)


# ------------------------------------------------------------------ end to end
def _cluster_subspace_check(A, B, w, X, wo, Xo):
    """Compare eigenvectors as B-orthonormal subspaces per eigenvalue cluster."""
    n = A.shape[0]
    Lo = np.linalg.cholesky(B)
    # map to the standard problem: y = L^H x (orthonormal)
    Y = Lo.conj().T @ X
    Yo = Lo.conj().T @ Xo
    Ap = np.linalg.solve(Lo, np.linalg.solve(Lo, A).conj().T).conj().T
    nA = np.linalg.norm(Ap, 2)
    gtol = 1e3 * n * EPS * nA
    i = 0
    m = len(w)
    while i < m:
        j = i + 1
        while j < m and wo[j] - wo[j - 1] < gtol:
            j += 1
        gap_l = wo[i] - wo[i - 1] if i > 0 else np.inf
        gap_r = wo[j] - wo[j - 1] if j < m else np.inf
        gap = min(gap_l, gap_r)
        if np.isfinite(gap):
            P = Yo[:, i:j]
            S = Y[:, i:j]
            resid = S - P @ (P.conj().T @ S)
            sin_angle = np.linalg.norm(resid, 2)
            assert sin_angle <= 1e4 * n * EPS * nA / gap + 1e-12, (i, j, sin_angle, gap)
        i = j


@pytest.fixture(params=["crt", "dmma"])
def engine(G, request):
    G.set_engine(request.param)
    yield request.param
    G.set_engine("crt")


@pytest.mark.parametrize("n,nb,seed", [(1, 1, 0), (2, 1, 0), (5, 2, 1), (33, 8, 2), (64, 16, 3), (100, 32, 4),
                                       (129, 16, 5), (256, 32, 0), (700, 64, 6)])
def test_hegv_all(G, engine, n, nb, seed):
    A, B, lam = inputs.make_pair(n, seed)
    w, X = G.hegv(_c(A), _c(B), 1, n, nb=nb)
    w, X = _np(w), _np(X)
    wo, Xo, info = oracle.hegv(A, B)
    assert info == 0
    tol = 10 * n * EPS * np.linalg.norm(A, 2) / np.linalg.eigvalsh(B).min()
    assert np.max(np.abs(w - wo)) <= tol
    assert np.max(np.abs(w - lam)) <= tol
    res = np.linalg.norm(A @ X - (B @ X) * w[None, :]) / (n * EPS * np.linalg.norm(A) * np.linalg.norm(X))
    orth = np.linalg.norm(X.conj().T @ B @ X - np.eye(n)) / (n * EPS)
    assert res <= 100, res
    assert orth <= 100 * max(1.0, np.linalg.cond(B) / 100), orth
    _cluster_subspace_check(A, B, w, X, wo, Xo)


@pytest.mark.parametrize("frac", [0.25, 0.10])
def test_hegv_fraction(G, frac):
    n, nb = 300, 32
    A, B, lam = inputs.make_pair(n, 7, "uniform", -10, 10)
    iu = inputs.fraction_iu(n, frac)
    w, X = G.hegv(_c(A), _c(B), 1, iu, nb=nb)
    w, X = _np(w), _np(X)
    wo, Xo, info = oracle.hegv(A, B, 1, iu)
    tol = 10 * n * EPS * np.linalg.norm(A, 2) / np.linalg.eigvalsh(B).min()
    assert np.max(np.abs(w - wo)) <= tol
    res = np.linalg.norm(A @ X - (B @ X) * w[None, :]) / (n * EPS * np.linalg.norm(A) * np.linalg.norm(X))
    orth = np.linalg.norm(X.conj().T @ B @ X - np.eye(iu)) / (n * EPS)
    assert res <= 100 and orth <= 100
    _cluster_subspace_check(A, B, w, X, wo, Xo)


@pytest.mark.parametrize("n,il,iu", [(1, 1, 1), (2, 1, 2), (33, 1, 33), (100, 1, 100), (130, 1, 13), (257, 20, 90)])
def test_hegv_onestage(G, n, il, iu):
    A, B, lam = inputs.make_pair(n, 11)
    w, X = G.hegv(_c(A), _c(B), il, iu, onestage=True)
    w, X = _np(w), _np(X)
    wo, Xo, info = oracle.hegv(A, B, il, iu)
    m = iu - il + 1
    tol = 10 * n * EPS * np.linalg.norm(A, 2) / np.linalg.eigvalsh(B).min()
    assert np.max(np.abs(w - wo)) <= tol
    res = np.linalg.norm(A @ X - (B @ X) * w[None, :]) / (n * EPS * np.linalg.norm(A) * np.linalg.norm(X))
    orth = np.linalg.norm(X.conj().T @ B @ X - np.eye(m)) / (n * EPS)
    assert res <= 100 and orth <= 100, (res, orth)
    _cluster_subspace_check(A, B, w, X, wo, Xo)


def test_hegv_clustered_illconditioned(G):
    n = 320
    A, B, lam = inputs.make_pair(n, 2, "clustered", -1, 1, ldiag="loguniform")
    w, X = G.hegv(_c(A), _c(B), 1, n, nb=32)
    w, X = _np(w), _np(X)
    wo, Xo, info = oracle.hegv(A, B)
    tol = 10 * n * EPS * np.linalg.norm(A, 2) / np.linalg.eigvalsh(B).min()
    assert np.max(np.abs(w - wo)) <= tol
    assert np.max(np.abs(w - lam)) <= tol
    res = np.linalg.norm(A @ X - (B @ X) * w[None, :]) / (n * EPS * np.linalg.norm(A) * np.linalg.norm(X))
    assert res <= 100
    _cluster_subspace_check(A, B, w, X, wo, Xo)


def test_hegv_not_pd_reports_and_recovers(G):
    """B not positive definite: the solve reports it through the status word
    (non-PD minor or non-finite tridiagonal) and the device stays usable."""
    n = 200
    A, B, _ = inputs.make_pair(n, 3)
    B[70, 70] = -5.0
    with pytest.raises(G.GbheError) as e:
        G.hegv(_c(A), _c(B), 1, n, nb=32)
    assert e.value.code > 0 or e.value.code == -104
    A, B, lam = inputs.make_pair(n, 4)
    w, _ = G.hegv(_c(A), _c(B), 1, n, nb=32)
    tol = 10 * n * EPS * np.linalg.norm(A, 2) / np.linalg.eigvalsh(B).min()
    assert np.max(np.abs(_np(w) - lam)) <= tol


def test_stedc_nonfinite_input(G):
    """A NaN in the tridiagonal: GBHE_ENONFINITE, no eigenvector work."""
    n = 300
    rng = np.random.default_rng(9)
    d = rng.standard_normal(n)
    e = rng.standard_normal(n - 1)
    d[17] = np.nan
    with pytest.raises(G.GbheError) as ex:
        G.stedc(torch.from_numpy(d).to(DEV), torch.from_numpy(e).to(DEV))
    assert ex.value.code == -104
    d[17] = 0.5
    w, _ = G.stedc(torch.from_numpy(d).to(DEV), torch.from_numpy(e).to(DEV))
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    assert np.max(np.abs(_np(w) - np.linalg.eigvalsh(T))) <= 100 * n * EPS * np.abs(T).max()
