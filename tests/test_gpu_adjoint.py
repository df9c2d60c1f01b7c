"""Reverse-mode derivative of the selected eigenpairs (gbhe_hegv_adjoint behind
torch.autograd.Function), on the loss sum_i w_i lambda_i + sum_i |x_i^H C x_i|^2
(phase-invariant): against central finite differences along random Hermitian
directions, and against an FP64 CPU reference built from the oracle's full
decomposition.

The reference is forward-mode first-order perturbation theory (the
directional derivative along (E_A, E_B) of every selected eigenpair, summed
into the loss's derivative), so it shares neither the decomposition nor the
reverse-mode algebra (K = X^H G, gap scaling, U, W_A, W_B) with the library:

  d lambda_i = x_i^H (E_A - lambda_i E_B) x_i
  d x_i      = sum_{j != i} x_j x_j^H (E_A - lambda_i E_B) x_i / (lambda_i - lambda_j)
               - 1/2 x_i (x_i^H E_B x_i)
  d L        = sum_i w_i d lambda_i + sum_i 2 s_i 2 Re(x_i^H C d x_i),  s_i = x_i^H C x_i
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
EPS = np.finfo(np.float64).eps


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


def _reference_directional(wall, Xall, il, iu, wts, C, EA, EB):
    """Directional derivative of the loss along (EA, EB) from the full
    decomposition (wall ascending, Xall B-orthonormal), forward mode."""
    S = slice(il - 1, iu)
    X, w = Xall[:, S], wall[S]
    M = EA @ X - (EB @ X) * w[None, :]
    P = Xall.conj().T @ M                       # P_ji = x_j^H (E_A - lambda_i E_B) x_i
    idx = np.arange(il - 1, iu)
    dlam = np.real(P[idx, np.arange(len(idx))])
    gap = w[None, :] - wall[:, None]            # lambda_i - lambda_j
    gap[idx, np.arange(len(idx))] = 1.0
    K = P / gap
    K[idx, np.arange(len(idx))] = 0.0
    beta = np.real(np.einsum("ij,ji->i", X.conj().T, EB @ X))
    dX = Xall @ K - 0.5 * X * beta[None, :]
    CX = C @ X
    s = np.real(np.einsum("ij,ji->i", X.conj().T, CX))
    ds = 2.0 * np.real(np.einsum("ij,ji->i", CX.conj().T, dX))
    return float(np.dot(wts, dlam) + np.sum(2.0 * s * ds))


def _grad(G, A, B, il, iu, wts, C):
    from paper_1207_1773_gb300.autograd import generalized_eigh
    At = G.colmajor(A, DEV).requires_grad_(True)
    Bt = G.colmajor(B, DEV).requires_grad_(True)
    w, X = generalized_eigh(At, Bt, il, iu)
    Ct = torch.from_numpy(C).to(DEV)
    s = torch.einsum("ij,jk,ki->i", X.conj().t(), Ct, X).real
    L = (torch.from_numpy(wts).to(DEV) * w).sum() + (s ** 2).sum()
    L.backward()
    return At.grad.cpu().numpy(), Bt.grad.cpu().numpy()


def test_adjoint_fd_and_reference(G):
    from paper_1207_1773_gb300 import inputs
    n, il, iu = 48, 1, 8
    A, B, _ = inputs.make_pair(n, 4)
    rng = np.random.default_rng(5)
    C = _herm(rng, n)
    wts = rng.standard_normal(iu - il + 1)
    dA, dB = _grad(G, A, B, il, iu, wts, C)
    # Hermitian gradients
    assert np.allclose(dA, dA.conj().T, atol=1e-12 * np.abs(dA).max())
    wall, Xall, info = oracle.hegv(A, B)
    assert info == 0

    def loss_at(Ap, Bp):
        wv, Xv = G.hegv(G.colmajor(Ap, DEV), G.colmajor(Bp, DEV), il, iu)
        return _loss_np(wv.cpu().numpy(), Xv.cpu().numpy(), wts, C)

    h = 1e-6
    for trial in range(3):
        EA = _herm(rng, n) if trial != 1 else np.zeros((n, n))
        EB = 0.1 * _herm(rng, n) if trial != 0 else np.zeros((n, n))
        an = np.real(np.vdot(dA, EA)) + np.real(np.vdot(dB, EB))
        ref = _reference_directional(wall, Xall, il, iu, wts, C, EA, EB)
        assert abs(an - ref) <= 1e-8 * max(1.0, abs(ref)), (trial, an, ref)
        fd = (loss_at(A + h * EA, B + h * EB) - loss_at(A - h * EA, B - h * EB)) / (2 * h)
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (trial, fd, an)


def test_adjoint_n2048_lowest64(G):
    """The adjoint workload's shape: n = 2048 pair (seed 4), lowest 64 pairs.
    (1) The eigenvalue part of the gradient has a closed form,
        dL/dA = X diag(w) X^H, dL/dB = -X diag(w lambda) X^H, checked element
        by element with the oracle's eigenvectors;
    (2) the full gradient against the oracle-based forward-mode reference
        along 8 random Hermitian directions (A only, B only, both);
    (3) central differences along 4 of them at h in {1e-5, 1e-6, 1e-7}: the
        best h must agree within 1e-3 (the floor of finite differences of an
        eigensolver: truncation ~ (h/gap)^2 against rounding ~ err(L)/h); the
        error at every h is part of the assertion message."""
    from paper_1207_1773_gb300 import inputs
    n, il, iu = 2048, 1, 64
    m = iu - il + 1
    A, B, _ = inputs.make_pair(n, 4, "uniform", -1.0, 1.0)
    rng = np.random.default_rng(4)
    C = _herm(rng, n)
    wts = rng.standard_normal(m)
    wall, Xall, info = oracle.hegv(A, B)
    assert info == 0
    X, w = Xall[:, :m], wall[:m]
    gmin = np.min(np.diff(wall[:m + 1]))
    # (1) eigenvalue part alone (C = 0): unique, phase-free
    gA, gB = _grad(G, A, B, il, iu, wts, np.zeros((n, n), complex))
    rA = (X * wts[None, :]) @ X.conj().T
    rB = -(X * (wts * w)[None, :]) @ X.conj().T
    tol1 = 100 * n * EPS * np.max(np.abs(wall)) / gmin
    assert np.abs(gA - rA).max() <= tol1 * np.abs(rA).max(), np.abs(gA - rA).max() / np.abs(rA).max()
    assert np.abs(gB - rB).max() <= tol1 * np.abs(rB).max(), np.abs(gB - rB).max() / np.abs(rB).max()
    # (2) the whole loss against the forward-mode reference
    dA, dB = _grad(G, A, B, il, iu, wts, C)
    dirs = []
    for trial in range(8):
        EA = _herm(rng, n) / np.sqrt(n) if trial % 3 != 1 else np.zeros((n, n), complex)
        EB = 0.1 * _herm(rng, n) / np.sqrt(n) if trial % 3 != 0 else np.zeros((n, n), complex)
        an = np.real(np.vdot(dA, EA)) + np.real(np.vdot(dB, EB))
        ref = _reference_directional(wall, Xall, il, iu, wts, C, EA, EB)
        assert abs(an - ref) <= tol1 * max(1.0, abs(ref)), (trial, an, ref)
        dirs.append((EA, EB, an))

    def loss_at(Ap, Bp):
        wv, Xv = G.hegv(G.colmajor(Ap, DEV), G.colmajor(Bp, DEV), il, iu)
        return _loss_np(wv.cpu().numpy(), Xv.cpu().numpy(), wts, C)

    # (3) finite differences, h sweep
    for EA, EB, an in dirs[:4]:
        errs = {}
        for h in (1e-5, 1e-6, 1e-7):
            fd = (loss_at(A + h * EA, B + h * EB) - loss_at(A - h * EA, B - h * EB)) / (2 * h)
            errs[h] = abs(fd - an) / max(1.0, abs(an))
        assert min(errs.values()) <= 1e-3, errs


def test_forward_leaves_inputs_unchanged(G):
    from paper_1207_1773_gb300 import inputs
    from paper_1207_1773_gb300.autograd import generalized_eigh
    A, B, _ = inputs.make_pair(64, 6)
    At, Bt = G.colmajor(A, DEV), G.colmajor(B, DEV)
    w1, _ = generalized_eigh(At, Bt, 1, 10)
    w2, _ = generalized_eigh(At, Bt, 1, 10)
    assert np.array_equal(At.cpu().numpy(), A) and np.array_equal(Bt.cpu().numpy(), B)
    assert np.array_equal(w1.cpu().numpy(), w2.cpu().numpy())
