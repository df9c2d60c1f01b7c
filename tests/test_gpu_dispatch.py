"""The engine dispatcher cuts products larger than one CRT block into blocks;
with the block set to 4096 these shapes exercise every block kind (interior,
ragged edge, Hermitian diagonal/off-diagonal, lower-only diagonal, K blocks
accumulated in C) against numpy FP64."""
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
    gbhegv.set_crt_block(4096)
    yield gbhegv
    gbhegv.set_crt_block(16384)


@pytest.mark.parametrize("opA,opB,m,n,k,lower", [
    ("N", "N", 5000, 4500, 64, False),
    ("N", "C", 4500, 4500, 64, True),
    ("C", "N", 64, 4200, 9000, False),
    ("H", "N", 4300, 64, 4300, False),
    ("N", "T", 4200, 100, 300, False),
])
def test_dispatch_blocks(G, opA, opB, m, n, k, lower):
    rng = np.random.default_rng(m + n + k)
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
    Cd = G.colmajor(C, DEV)
    G.zgemm(opA, opB, G.colmajor(A, DEV), G.colmajor(B, DEV), Cd, -1.0, 1.0, lower=lower)
    out = Cd.cpu().numpy()
    ref = C - a @ b
    scale = np.abs(a) @ np.abs(b) + np.abs(C)
    ok = np.abs(out - ref) <= 8 * (k + 2) * EPS * scale
    if lower:
        low = np.tril(np.ones((m, n), bool))
        assert np.all(ok[low])
        assert np.array_equal(out[~low], C[~low])
    else:
        assert np.all(ok)
