"""Parity at the workloads' full sizes: the n = 4096 pair (all eigenpairs,
lowest 25 %, lowest 10 %), the n = 10000 pair in the launch configuration
the benchmark times (all eigenpairs, nb = 64), and -- only with GBHE_CFG2=1,
since it needs about 100 GB of device and 25 GB of host memory -- the
n = 20000 pair with a clustered spectrum and an ill-conditioned B (all
eigenpairs and the lowest 20 %).  The oracle cannot run at these
sizes inside a test, so the checks are properties that hold at any size:

  * eigenvalues against the constructed spectrum Lambda (known exactly):
    |w - lambda| <= 10 n eps max|Lambda| kappa_2(B), a bound on
    10 n eps ||A||_2 ||B^-1||_2 since ||A||_2 <= ||B||_2 max|Lambda|;
  * residual ratio ||A x - w B x||_F / (n eps ||A||_F ||x||_F) <= 100 and
    B-orthonormality ||X^H B X - I||_F / (n eps) <= 100 on 64 sampled columns
    (both products formed with torch on the device; test arithmetic only).
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps
DEV = "cuda:0"


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1207_1773_gb300 import gbhegv
    gbhegv.set_engine("crt")
    return gbhegv


def _pair(n, seed, kind="uniform", lo=-10.0, hi=10.0, ldiag="abs_normal"):
    from paper_1207_1773_gb300 import inputs
    A, B, lam = inputs.make_pair(n, seed, kind, lo, hi, ldiag=ldiag, device=torch.device(DEV))
    A0 = torch.from_numpy(A).to(DEV).t().contiguous().t()
    B0 = torch.from_numpy(B).to(DEV).t().contiguous().t()
    return A0, B0, lam


def _check(G, A0, B0, lam, iu, nb, kappa):
    n = A0.shape[0]
    w, X = G.hegv(A0.clone(), B0.clone(), 1, iu, nb=nb)
    w = w.cpu().numpy()
    tol = 10 * n * EPS * np.max(np.abs(lam)) * kappa
    err = np.max(np.abs(w - lam[:iu]))
    assert err <= tol, (err, tol)
    cols = np.unique(np.linspace(0, iu - 1, 64).astype(int))
    Xs = X[:, torch.from_numpy(cols).to(DEV)]
    ws = torch.from_numpy(w[cols]).to(DEV)
    R = A0 @ Xs - (B0 @ Xs) * ws[None, :]
    res = (torch.linalg.norm(R) / (n * EPS * torch.linalg.norm(A0) * torch.linalg.norm(Xs))).item()
    O = Xs.conj().t() @ (B0 @ Xs) - torch.eye(len(cols), dtype=torch.complex128, device=DEV)
    orth = (torch.linalg.norm(O) / (n * EPS)).item()
    assert res <= 100, res
    assert orth <= 100, orth
    return err, res, orth


@pytest.fixture(scope="module")
def pair4096():
    return _pair(4096, 1)


@pytest.mark.parametrize("frac,nb", [(1.0, 64), (0.25, 64), (0.10, 32)])
def test_hegv_n4096(G, pair4096, frac, nb):
    from paper_1207_1773_gb300 import inputs
    A0, B0, lam = pair4096
    ev = torch.linalg.eigvalsh(B0).cpu().numpy()
    _check(G, A0, B0, lam, inputs.fraction_iu(4096, frac), nb, ev[-1] / ev[0])


def test_hegv_n10000_bench_config(G):
    A0, B0, lam = _pair(10000, 10)
    ev = torch.linalg.eigvalsh(B0).cpu().numpy()
    _check(G, A0, B0, lam, 10000, 64, ev[-1] / ev[0])


@pytest.fixture(scope="module")
def pair20000():
    return _pair(20000, 2, "clustered", -1.0, 1.0, ldiag="loguniform")


@pytest.mark.skipif(os.environ.get("GBHE_CFG2") != "1",
                    reason="n = 20000 workload (about 100 GB device, 25 GB host memory): set GBHE_CFG2=1")
@pytest.mark.parametrize("frac", [1.0, 0.20])
def test_hegv_n20000_clustered_illconditioned(G, pair20000, frac):
    from paper_1207_1773_gb300 import inputs
    A0, B0, lam = pair20000
    ev = torch.linalg.eigvalsh(B0).cpu().numpy()
    _check(G, A0, B0, lam, inputs.fraction_iu(20000, frac), 64, ev[-1] / ev[0])
