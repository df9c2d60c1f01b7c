"""Stage reconstructions of the two-stage reduction (Section 4.2, Algorithm
2): after he2hb and hb2st, the back-transform applied to the identity gives
Q = Q1 Q2, and Q must be unitary with Q T Q^H = A' for the tridiagonal T of
(d, e); the trace is preserved.  These hold for any Hermitian A' and check
the reflector storage (V1, T1, V2, tau2) and both back-transforms directly,
without the tridiagonal eigensolver in between.

Bounds: ||Q^H Q - I||_F <= c n eps and ||Q T Q^H - A'||_F <= c n eps ||A'||_F
with c = 1000 -- a backward-stable product of O(n/nb) block reflectors sits
orders of magnitude below it, while a wrong reflector, sign or index makes
either quantity O(1)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.late]

EPS = np.finfo(np.float64).eps
DEV = "cuda:0"
C = 1000.0


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1207_1773_gb300 import gbhegv
    return gbhegv


def _hermitian(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return 0.5 * (M + M.conj().T)


@pytest.mark.parametrize("n,nb", [(2, 1), (33, 8), (100, 16), (129, 32), (300, 64)])
def test_q1q2_reconstructs_a(G, n, nb):
    A = _hermitian(n, 1000 + n)
    Ad = G.colmajor(A, DEV)
    T1, _ = G.he2hb(Ad, nb)
    d, e, V2, tau2 = G.hb2st(Ad, nb)
    Q = G.unmtr_2stage(nb, Ad, T1, V2, tau2, G.colmajor(np.eye(n), DEV)).cpu().numpy()
    d, e = d.cpu().numpy(), e.cpu().numpy()
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    orth = np.linalg.norm(Q.conj().T @ Q - np.eye(n)) / (n * EPS)
    rec = np.linalg.norm(Q @ T @ Q.conj().T - A) / (n * EPS * np.linalg.norm(A))
    assert orth <= C, orth
    assert rec <= C, rec
    assert abs(d.sum() - np.trace(A).real) <= C * n * EPS * np.linalg.norm(A)


@pytest.mark.parametrize("n,nb", [(1, 1), (40, 40), (40, 64)])
def test_he2hb_band_at_least_n_is_noop(G, n, nb):
    """With nb >= n the matrix already is a band: stage 1 leaves the lower
    triangle as it is and stores no reflectors."""
    A = _hermitian(n, 2000 + n)
    Ad = G.colmajor(A, DEV)
    T1, tau1 = G.he2hb(Ad, nb)
    out = Ad.cpu().numpy()
    assert np.array_equal(np.tril(out), np.tril(A))
    assert not T1.abs().max().item() and not tau1.abs().max().item()
