"""gbhe_zgemm_static: the DMMA GEMM whose split-K scratch is the library's
static device array.  Two calls in a row (the second reuses the scratch the
first left behind) must each match the handle-based gbhe_zgemm on the same
engine and numpy, and products beyond the static limit must be refused with C
left untouched.  Collected last so it also runs after every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.last]
EPS = np.finfo(np.float64).eps
DEV = "cuda:0"


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1207_1773_gb300 import gbhegv
    gbhegv.set_engine("dmma")
    yield gbhegv
    gbhegv.set_engine("crt")


def _operands(rng, opA, opB, m, n, k):
    ra, ca = (m, k) if opA in ("N", "H") else (k, m)
    rb, cb = (k, n) if opB == "N" else (n, k)
    A = rng.standard_normal((ra, ca)) + 1j * rng.standard_normal((ra, ca))
    B = rng.standard_normal((rb, cb)) + 1j * rng.standard_normal((rb, cb))
    C = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    if opA == "H":
        a = np.tril(A) + np.tril(A, -1).conj().T
        a = a - 1j * np.diag(np.diag(a).imag)
    else:
        a = {"N": A, "T": A.T, "C": A.conj().T}[opA]
    b = {"N": B, "T": B.T, "C": B.conj().T}[opB]
    return A, B, C, a, b


# split-K shapes (few output tiles, long k), the largest accepted m * n (its
# split count cut to what the static array holds), a Hermitian operand and one
# product with no split at all
@pytest.mark.parametrize("opA,opB,m,n,k,lower", [
    ("C", "N", 64, 64, 8192, False),
    ("C", "N", 64, 200, 20000, False),
    ("C", "N", 512, 512, 4096, False),
    ("N", "C", 192, 192, 4096, True),
    ("H", "N", 1500, 48, 1500, False),
    ("N", "N", 300, 40, 100, False),
])
def test_static_matches_zgemm_twice(G, opA, opB, m, n, k, lower):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    alpha, beta = -1.0 + 0.5j, 0.75
    for _ in range(2):
        A, B, C, a, b = _operands(rng, opA, opB, m, n, k)
        Ad, Bd = G.colmajor(A, DEV), G.colmajor(B, DEV)
        Cs, Ch = G.colmajor(C, DEV), G.colmajor(C, DEV)
        G.zgemm_static(opA, opB, Ad, Bd, Cs, alpha, beta, lower=lower)
        G.zgemm(opA, opB, Ad, Bd, Ch, alpha, beta, lower=lower)
        out_s, out_h = Cs.cpu().numpy(), Ch.cpu().numpy()
        ref = alpha * (a @ b) + beta * C
        scale = abs(alpha) * (np.abs(a) @ np.abs(b)) + abs(beta) * np.abs(C)
        tol = 8 * (k + 2) * EPS * scale
        mask = np.tril(np.ones((m, n), bool)) if lower else np.ones((m, n), bool)
        assert np.all(np.abs(out_s - out_h)[mask] <= 2 * tol[mask])
        assert np.all(np.abs(out_s - ref)[mask] <= tol[mask])
        if lower:
            assert np.array_equal(out_s[~mask], C[~mask])


def test_static_rejects_oversize(G):
    m, n, k = 1024, 257, 64  # m * n = 263168 > 2**18
    rng = np.random.default_rng(5)
    A, B, C, _, _ = _operands(rng, "N", "N", m, n, k)
    Cd = G.colmajor(C, DEV)
    with pytest.raises(G.GbheError) as e:
        G.zgemm_static("N", "N", G.colmajor(A, DEV), G.colmajor(B, DEV), Cd, 1.0, 1.0)
    assert e.value.code == -106
    assert np.array_equal(Cd.cpu().numpy(), C)
