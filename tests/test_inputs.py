"""Host-side logic: the seeded generator and the eigenvalue-fraction selector."""
import numpy as np
import pytest

from paper_1207_1773_gb300 import inputs


def test_fraction_iu():
    assert inputs.fraction_iu(4096, 0.10) == 410
    assert inputs.fraction_iu(4096, 0.25) == 1024
    assert inputs.fraction_iu(10000, 1.0) == 10000
    assert inputs.fraction_iu(7, 0.5) == 4


def test_pair_is_deterministic_and_definite():
    A1, B1, l1 = inputs.make_pair(40, 3)
    A2, B2, l2 = inputs.make_pair(40, 3)
    assert np.array_equal(A1, A2) and np.array_equal(B1, B2) and np.array_equal(l1, l2)
    assert np.allclose(A1, A1.conj().T, atol=0) and np.allclose(B1, B1.conj().T, atol=0)
    assert np.linalg.eigvalsh(B1).min() > 0
    # the constructed spectrum is the generalized spectrum
    w = np.sort(np.linalg.eigvals(np.linalg.solve(B1, A1)).real)
    assert np.max(np.abs(w - l1)) < 1e-10


def test_clustered_spectrum_layout():
    rng = np.random.default_rng(0)
    lam = inputs.spectrum(rng, 20000, "clustered", -1, 1)
    assert lam.shape == (20000,)
    clu = lam[18000:].reshape(250, 8)
    gaps = np.diff(clu, axis=1)
    assert np.allclose(gaps, 1e-10, rtol=1e-4, atol=0)


@pytest.mark.parametrize("kind", ["abs_normal", "loguniform"])
def test_ldiag(kind):
    A, B, lam = inputs.make_pair(30, 1, ldiag=kind)
    L = np.linalg.cholesky(B)
    d = np.abs(np.diag(L))
    if kind == "loguniform":
        assert d.min() >= 1 - 1e-9 and d.max() <= 100 + 1e-9
    else:
        assert d.min() >= 1 - 1e-9
