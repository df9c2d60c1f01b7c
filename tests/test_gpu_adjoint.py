"""Reverse-mode derivative of the selected eigenpairs (gbhe_hegv_adjoint behind
torch.autograd.Function), on the loss sum_i w_i lambda_i + sum_i |x_i^H C x_i|^2
(phase-invariant): against central finite differences (h = 1e-6) along random
Hermitian directions, and against an FP64 CPU reference gradient built from
scipy's full decomposition."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1207_1773_gb300 import gbhegv
    gbhegv.set_engine("crt")
    return gbhegv


def _herm(rng, n):
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return (M + M.conj().T) / 2


def _loss_np(w, X, wts, C):
    s = np.einsum("ij,jk,ki->i", X.conj().T, C, X).real
    return float(np.dot(wts, w) + np.sum(s ** 2))


def _reference_grad(A, B, il, iu, wts, C):
    """dL/dA, dL/dB from first-order perturbation theory on the full decomposition."""
    import scipy.linalg
    lam, V = scipy.linalg.eigh(A, B)
    S = slice(il - 1, iu)
    X, w = V[:, S], lam[S]
    s = np.einsum("ij,jk,ki->i", X.conj().T, C, X).real
    gX = 4 * s[None, :] * (C @ X)
    K = V.conj().T @ gX
    gap = w[None, :] - lam[:, None]
    Kp = np.where(np.abs(gap) > 1e-9, K / np.where(gap == 0, 1, gap), 0)
    U = V @ Kp
    c = np.real(np.einsum("ij,ji->i", X.conj().T, gX))
    WA = X * wts[None, :] + U
    WB = X * (w * wts + 0.5 * c)[None, :] + U * w[None, :]
    GA, GB = X @ WA.conj().T, -(X @ WB.conj().T)
    return (GA + GA.conj().T) / 2, (GB + GB.conj().T) / 2


def test_adjoint_fd_and_reference(G):
    from paper_1207_1773_gb300 import inputs
    from paper_1207_1773_gb300.autograd import generalized_eigh
    n, il, iu = 48, 1, 8
    A, B, _ = inputs.make_pair(n, 4)
    rng = np.random.default_rng(5)
    C = _herm(rng, n)
    wts = rng.standard_normal(iu - il + 1)
    At = G.colmajor(A, DEV).requires_grad_(True)
    Bt = G.colmajor(B, DEV).requires_grad_(True)
    w, X = generalized_eigh(At, Bt, il, iu)
    Ct = torch.from_numpy(C).to(DEV)
    s = torch.einsum("ij,jk,ki->i", X.conj().t(), Ct, X).real
    L = (torch.from_numpy(wts).to(DEV) * w).sum() + (s ** 2).sum()
    L.backward()
    dA, dB = At.grad.cpu().numpy(), Bt.grad.cpu().numpy()
    # Hermitian gradients
    assert np.allclose(dA, dA.conj().T, atol=1e-12 * np.abs(dA).max())
    # FP64 CPU reference
    rA, rB = _reference_grad(A, B, il, iu, wts, C)
    assert np.abs(dA - rA).max() <= 1e-8 * np.abs(rA).max()
    assert np.abs(dB - rB).max() <= 1e-8 * np.abs(rB).max()

    def loss_at(Ap, Bp):
        wv, Xv = G.hegv(G.colmajor(Ap, DEV), G.colmajor(Bp, DEV), il, iu)
        return _loss_np(wv.cpu().numpy(), Xv.cpu().numpy(), wts, C)

    h = 1e-6
    for trial in range(3):
        EA = _herm(rng, n) if trial != 1 else np.zeros((n, n))
        EB = 0.1 * _herm(rng, n) if trial != 0 else np.zeros((n, n))
        fd = (loss_at(A + h * EA, B + h * EB) - loss_at(A - h * EA, B - h * EB)) / (2 * h)
        an = np.real(np.vdot(dA, EA)) + np.real(np.vdot(dB, EB))
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (trial, fd, an)


def test_forward_leaves_inputs_unchanged(G):
    from paper_1207_1773_gb300 import inputs
    from paper_1207_1773_gb300.autograd import generalized_eigh
    A, B, _ = inputs.make_pair(64, 6)
    At, Bt = G.colmajor(A, DEV), G.colmajor(B, DEV)
    w1, _ = generalized_eigh(At, Bt, 1, 10)
    w2, _ = generalized_eigh(At, Bt, 1, 10)
    assert np.array_equal(At.cpu().numpy(), A) and np.array_equal(Bt.cpu().numpy(), B)
    assert np.array_equal(w1.cpu().numpy(), w2.cpu().numpy())
