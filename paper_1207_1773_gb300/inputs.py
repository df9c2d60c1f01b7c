"""Seeded synthetic Hermitian-definite pairs with known spectra.

This module only draws random numbers and forms the products that define a
test pair; it contains none of the solver's arithmetic and is shared by the
tests, the benchmark and the oracle checks.

Construction (the workloads of the paper's Section 5 are complex128
generalized problems of order a few thousand to twenty thousand):
  L lower triangular: strictly-lower entries complex N(0,1)/sqrt(n), where a
    complex N(0,1) is (a + i b)/sqrt(2) with a, b real N(0,1); diagonal
    1 + |N(0,1)| (or log-uniform in [1, 100] for the ill-conditioned B);
  Q Haar unitary: QR of a complex Gaussian matrix G = QR, with the phase fix
    Q <- Q diag(R_ii / |R_ii|);
  Lambda given (uniform or clustered);
  B = L L^H,  A = L Q Lambda Q^H L^H  (both Hermitised),
so that A x = lambda B x has exactly the eigenvalues Lambda.

Draw order from numpy.random.default_rng(seed): G (real, then imaginary
parts), Lambda, L strictly-lower (real, imaginary), L diagonal.
"""
from __future__ import annotations

import math

import numpy as np


def _cnormal(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


def spectrum(rng, n, kind="uniform", lo=-1.0, hi=1.0, cluster_frac=0.10, cluster_size=8,
             cluster_gap=1e-10):
    if kind == "uniform":
        return rng.uniform(lo, hi, n)
    if kind == "clustered":
        nclu = int(round(n * cluster_frac)) // cluster_size
        nuni = n - nclu * cluster_size
        uni = rng.uniform(lo, hi, nuni)
        centres = rng.uniform(lo, hi, nclu)
        clu = (centres[:, None] + cluster_gap * np.arange(cluster_size)[None, :]).reshape(-1)
        return np.concatenate([uni, clu])
    raise ValueError(kind)


def make_pair(n, seed, lam_kind="uniform", lam_lo=-1.0, lam_hi=1.0, ldiag="abs_normal",
              device=None):
    """Return (A, B, lam_sorted) as complex128 Fortran-ordered numpy arrays.

    With ``device`` set (a torch device), the O(n^3) products and the QR are
    formed there with torch (for large n); the random draws stay on numpy."""
    rng = np.random.default_rng(seed)
    G = _cnormal(rng, (n, n))
    lam = spectrum(rng, n, lam_kind, lam_lo, lam_hi)
    Loff = _cnormal(rng, (n, n)) / math.sqrt(n)
    if ldiag == "abs_normal":
        dg = 1.0 + np.abs(rng.standard_normal(n))
    elif ldiag == "loguniform":
        dg = np.exp(rng.uniform(math.log(1.0), math.log(100.0), n))
    else:
        raise ValueError(ldiag)
    L = np.tril(Loff, -1) + np.diag(dg.astype(np.complex128))
    if device is None:
        Q, R = np.linalg.qr(G)
        ph = np.diag(R) / np.abs(np.diag(R))
        Q = Q * ph[None, :]
        M = (Q * lam[None, :]) @ Q.conj().T
        A = L @ M @ L.conj().T
        B = L @ L.conj().T
    else:
        import torch
        Gt = torch.from_numpy(G).to(device)
        Q, R = torch.linalg.qr(Gt)
        dR = torch.diagonal(R)
        Q = Q * (dR / dR.abs())[None, :]
        lt = torch.from_numpy(lam).to(device=device, dtype=torch.complex128)
        M = (Q * lt[None, :]) @ Q.conj().T
        del Q, Gt, R
        Lt = torch.from_numpy(L).to(device)
        A = (Lt @ M @ Lt.conj().T)
        B = Lt @ Lt.conj().T
        A = A.cpu().numpy()
        B = B.cpu().numpy()
        del Lt, M
    A = 0.5 * (A + A.conj().T)
    B = 0.5 * (B + B.conj().T)
    return np.asfortranarray(A), np.asfortranarray(B), np.sort(lam)


def config_pair(name, device=None):
    """Named workloads: (A, B, lam, il, iu, nb) lists per run.

    cfg0  n=256,  Lambda ~ U[-1,1],  seed 0, all pairs, nb=32
    cfg1  n=4096, Lambda ~ U[-10,10], seed 1, all / lowest 25% / lowest 10%
    cfg2  n=20000, clustered Lambda, log-uniform diag(L), seed 2
    n10k  n=10000, as cfg1, seed 10 (the headline timing workload)
    """
    if name == "cfg0":
        return make_pair(256, 0, "uniform", -1.0, 1.0, device=device)
    if name == "cfg1":
        return make_pair(4096, 1, "uniform", -10.0, 10.0, device=device)
    if name == "cfg2":
        return make_pair(20000, 2, "clustered", -1.0, 1.0, ldiag="loguniform", device=device)
    if name == "n10k":
        return make_pair(10000, 10, "uniform", -10.0, 10.0, device=device)
    raise ValueError(name)


def fraction_iu(n, frac):
    """Upper selector for the lowest fraction of the spectrum: ceil(frac*n)."""
    return int(math.ceil(frac * n - 1e-9))
