"""Failure detection on the GPU without a fault: a bounded device wait whose
partner never arrives gives up after its time limit, the status word reports
GBHE_ETIMEOUT, and the same handle then solves correctly."""
import time

import numpy as np
import pytest

import oracle
from paper_1207_1773_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.late]

EPS = np.finfo(np.float64).eps
DEV = "cuda:0"


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1207_1773_gb300 import gbhegv
    return gbhegv


def test_bounded_wait_expires_and_handle_recovers(G):
    h = G.handle(DEV)
    assert h.status() == 0
    t0 = time.perf_counter()
    st = G.wait_selftest(DEV)
    dt = time.perf_counter() - t0
    assert st == -103, G.status_string(st)
    assert 1.5 <= dt <= 30.0, dt       # the 2 s limit of %globaltimer
    assert h.status() == 0             # reported once, then cleared
    n = 96
    A, B, lam = inputs.make_pair(n, 11)
    w, _ = G.hegv(G.colmajor(A, DEV), G.colmajor(B, DEV))
    wo, _, info = oracle.hegv(A, B)
    assert info == 0
    tol = 10 * n * EPS * np.linalg.norm(A, 2) / np.linalg.eigvalsh(B).min()
    assert np.max(np.abs(w.cpu().numpy() - wo)) <= tol
