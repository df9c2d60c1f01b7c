"""FP64-exact modular GEMM on the FP16 tensor cores, against exact references.
Shapes cover both product kernels (one exact chunk, several chunks) with both
tile widths (64 columns when n <= 64, else 128) and ragged edges.

The reference is the product computed in numpy FP64 plus its own error bound;
the CRT result must agree within the FP64 GEMM error bound
8 (k + 2) eps |op(A)| |op(B)| (the modular path itself only rounds once at the
end, plus the per-row/column rounding of the operands to 53-bit integers).
"""
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
    return gbhegv


def _c(x):
    from paper_1207_1773_gb300 import gbhegv
    return gbhegv.colmajor(x, DEV)


def _ops(A, B, opA, opB):
    if opA == "H":
        a = np.tril(A) + np.tril(A, -1).conj().T
        a = a - 1j * np.diag(np.diag(a).imag)
    else:
        a = {"N": A, "T": A.T, "C": A.conj().T}[opA]
    b = {"N": B, "T": B.T, "C": B.conj().T}[opB]
    return a, b


@pytest.mark.parametrize("opA,opB", [("N", "N"), ("N", "C"), ("C", "N"), ("T", "T"), ("H", "N"), ("N", "T")])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (64, 64, 16), (129, 65, 33), (200, 70, 700), (37, 300, 1500),
                                   (200, 64, 700), (130, 33, 300)])
def test_crt_complex(G, opA, opB, m, n, k):
    rng = np.random.default_rng(m + 3 * n + 7 * k)
    if opA == "H":
        k = m
    ra, ca = (m, k) if opA in ("N", "H") else (k, m)
    rb, cb = (k, n) if opB == "N" else (n, k)
    A = rng.standard_normal((ra, ca)) + 1j * rng.standard_normal((ra, ca))
    B = rng.standard_normal((rb, cb)) + 1j * rng.standard_normal((rb, cb))
    C = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    alpha, beta = 0.7 - 0.2j, -0.3 + 0.5j
    a, b = _ops(A, B, opA, opB)
    ref = alpha * (a @ b) + beta * C
    Cd = _c(C)
    G.gemm_crt(opA, opB, _c(A), _c(B), Cd, alpha, beta)
    out = Cd.cpu().numpy()
    scale = abs(alpha) * (np.abs(a) @ np.abs(b)) + abs(beta) * np.abs(C)
    assert np.all(np.abs(out - ref) <= 8 * (k + 2) * EPS * scale)


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (100, 64, 512), (257, 129, 1031), (150, 40, 1500)])
def test_crt_real(G, m, n, k):
    rng = np.random.default_rng(m * k)
    A = rng.standard_normal((m, k))
    B = rng.standard_normal((k, n))
    C = np.zeros((m, n))
    Cd = G.colmajor(C, DEV, torch.float64)
    G.gemm_crt("N", "N", G.colmajor(A, DEV, torch.float64), G.colmajor(B, DEV, torch.float64), Cd, 1.0, 0.0)
    ref = A @ B
    assert np.all(np.abs(Cd.cpu().numpy() - ref) <= 8 * (k + 2) * EPS * (np.abs(A) @ np.abs(B)))


def test_crt_exact_on_integers(G):
    """Integer operands whose exact product fits in 53 bits come out exact."""
    rng = np.random.default_rng(1)
    m, n, k = 96, 80, 2048
    A = rng.integers(-2 ** 20, 2 ** 20, (m, k)).astype(np.float64)
    B = rng.integers(-2 ** 20, 2 ** 20, (k, n)).astype(np.float64)
    Cd = torch.zeros((n, m), dtype=torch.float64, device=DEV).t()
    G.gemm_crt("N", "N", G.colmajor(A, DEV, torch.float64), G.colmajor(B, DEV, torch.float64), Cd, 1.0, 0.0)
    ref = (A.astype(object) @ B.astype(object)).astype(np.float64)  # exact big-int product, rounded once
    assert np.array_equal(Cd.cpu().numpy(), ref)


def test_crt_wide_range_and_zeros(G):
    """Rows/columns of very different magnitude (scaled independently), zero rows."""
    rng = np.random.default_rng(2)
    m, n, k = 70, 50, 300
    A = (rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))) * (10.0 ** rng.integers(-30, 30, (m, 1)))
    B = (rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))) * (10.0 ** rng.integers(-30, 30, (1, n)))
    A[5] = 0
    B[:, 7] = 0
    Cd = torch.zeros((n, m), dtype=torch.complex128, device=DEV).t()
    G.gemm_crt("N", "N", _c(A), _c(B), Cd, 1.0, 0.0)
    out = Cd.cpu().numpy()
    ref = A @ B
    scale = np.abs(A) @ np.abs(B)
    assert np.all(np.abs(out - ref) <= 8 * (k + 2) * EPS * scale)
    assert np.all(out[5] == 0) and np.all(out[:, 7] == 0)


def test_crt_lower_only(G):
    rng = np.random.default_rng(3)
    n, k = 150, 64
    A = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    C = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Cd = _c(C)
    G.gemm_crt("N", "C", _c(A), _c(A), Cd, -1.0, 1.0, lower=True)
    out = Cd.cpu().numpy()
    ref = C - A @ A.conj().T
    low = np.tril(np.ones((n, n), bool))
    scale = np.abs(A) @ np.abs(A).T + np.abs(C)
    assert np.all(np.abs(out - ref)[low] <= 8 * (k + 2) * EPS * scale[low])
    assert np.array_equal(out[~low], C[~low])


def test_crt_exact_at_max_k(G):
    """K = 65536, the largest contraction of the exactness margin (|C| <= K 2^106 < M/8):
    integer operands, exact big-integer product rounded once."""
    rng = np.random.default_rng(4)
    m, n, k = 16, 8, 65536
    A = rng.integers(-2 ** 10, 2 ** 10, (m, k)).astype(np.float64)
    B = rng.integers(-2 ** 10, 2 ** 10, (k, n)).astype(np.float64)
    Cd = torch.zeros((n, m), dtype=torch.float64, device=DEV).t()
    G.gemm_crt("N", "N", G.colmajor(A, DEV, torch.float64), G.colmajor(B, DEV, torch.float64), Cd, 1.0, 0.0)
    ref = (A.astype(object) @ B.astype(object)).astype(np.float64)
    assert np.array_equal(Cd.cpu().numpy(), ref)


@pytest.mark.parametrize("k,cplx", [(256, True), (257, True), (512, False), (513, False)])
def test_crt_chunk_boundaries(G, k, cplx):
    """Either side of one exact chunk (256 complex / 512 real contraction terms):
    the single-chunk (warp-specialised) and the multi-chunk product kernels."""
    rng = np.random.default_rng(k)
    m, n = 130, 70
    if cplx:
        A = rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))
        B = rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
        Ad, Bd = _c(A), _c(B)
        Cd = torch.zeros((n, m), dtype=torch.complex128, device=DEV).t()
    else:
        A = rng.standard_normal((m, k))
        B = rng.standard_normal((k, n))
        Ad, Bd = G.colmajor(A, DEV, torch.float64), G.colmajor(B, DEV, torch.float64)
        Cd = torch.zeros((n, m), dtype=torch.float64, device=DEV).t()
    G.gemm_crt("N", "N", Ad, Bd, Cd, 1.0, 0.0)
    ref = A @ B
    assert np.all(np.abs(Cd.cpu().numpy() - ref) <= 8 * (k + 2) * EPS * (np.abs(A) @ np.abs(B)))


def _exact(a, b):
    """op(A) op(B) in extended precision (numpy longdouble: 64-bit or more
    mantissa), so the reference's own rounding is far below the bound tested."""
    return (a.astype(np.clongdouble) @ b.astype(np.clongdouble))


@pytest.mark.parametrize("opA,opB,m,n,k", [("N", "N", 130, 70, 64), ("C", "N", 130, 70, 300),
                                           ("N", "C", 97, 129, 1031)])
def test_crt_graded_within_rows_and_columns(G, opA, opB, m, n, k):
    """Entries graded inside every row of op(A) and column of op(B)
    (a_ik = g_ik 10^u, u ~ U[-12, 0]).  The engine rounds each row of op(A)
    (column of op(B)) to 53-bit integers relative to its largest entry, so its
    error bound is normwise per row and column:
        |err_ij| <= 4 eps (max_k |a_ik| sum_k |b_kj| + sum_k |a_ik| max_k |b_kj|) + eps |c_ij|,
    independent of k (the modular products are exact).  This is weaker than an
    FP64 GEMM's componentwise gamma_k |A||B| for graded rows: the test pins
    the bound the engine does guarantee."""
    rng = np.random.default_rng(m + n + k)
    ra, ca = (m, k) if opA == "N" else (k, m)
    rb, cb = (k, n) if opB == "N" else (n, k)
    A = (rng.standard_normal((ra, ca)) + 1j * rng.standard_normal((ra, ca))) * 10.0 ** rng.uniform(-12, 0, (ra, ca))
    B = (rng.standard_normal((rb, cb)) + 1j * rng.standard_normal((rb, cb))) * 10.0 ** rng.uniform(-12, 0, (rb, cb))
    a, b = _ops(A, B, opA, opB)
    Cd = torch.zeros((n, m), dtype=torch.complex128, device=DEV).t()
    G.gemm_crt(opA, opB, _c(A), _c(B), Cd, 1.0, 0.0)
    out = Cd.cpu().numpy()
    ref = _exact(a, b)
    err = np.abs(out.astype(np.clongdouble) - ref).astype(np.float64)
    absa, absb = np.abs(a), np.abs(b)
    bound = 4 * EPS * (absa.max(axis=1)[:, None] * absb.sum(axis=0)[None, :]
                       + absa.sum(axis=1)[:, None] * absb.max(axis=0)[None, :]) + EPS * np.abs(out)
    assert np.all(err <= bound), float(np.max(err / bound))
