"""The Python binding fails loudly instead of falling back (no GPU needed):
CPU tensors are refused before any work, row-major matrices are refused, and
a missing library raises instead of importing any other implementation."""
import pytest

torch = pytest.importorskip("torch")

from paper_1207_1773_gb300 import gbhegv  # noqa: E402


def test_cpu_tensors_are_refused():
    A = torch.eye(4, dtype=torch.complex128).t()
    B = torch.eye(4, dtype=torch.complex128).t()
    with pytest.raises(ValueError, match="CUDA"):
        gbhegv.hegv(A, B)
    with pytest.raises(ValueError, match="CUDA"):
        gbhegv.Handle("cpu")


def test_row_major_is_refused():
    X = torch.zeros((3, 5), dtype=torch.complex128)   # row-major, stride (5, 1)
    with pytest.raises(ValueError, match="column-major"):
        gbhegv._ld(X)
    assert gbhegv._ld(X.t().contiguous().t()) == 3


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(gbhegv, "_lib", None)
    monkeypatch.setattr(gbhegv, "_LIBPATH", str(tmp_path / "libgbhegv.so"))
    with pytest.raises(RuntimeError, match="not built"):
        gbhegv._load()
    with pytest.raises(RuntimeError, match="not built"):
        gbhegv.nb_rule_pick([], 100)


def test_host_device_never_maps_to_a_cached_gpu_handle(monkeypatch):
    """A CPU tensor must not pick up the handle cached for GPU 0: its host
    address would reach the GPU kernels."""
    monkeypatch.setattr(gbhegv, "_handles", {0: object()})
    with pytest.raises(ValueError, match="CUDA"):
        gbhegv.handle("cpu")
    with pytest.raises(ValueError, match="CUDA"):
        gbhegv.hegv(torch.eye(2, dtype=torch.complex128), torch.eye(2, dtype=torch.complex128))


class _FakeCuda:
    """Stands in for a CUDA tensor in the host-side argument checks."""

    def __init__(self, dtype, device="cuda:0"):
        self.is_cuda = True
        self.dtype = dtype
        self.device = torch.device(device)


def test_element_type_and_device_are_checked():
    dev = torch.device("cuda:0")
    gbhegv._want(torch.complex128, dev, _FakeCuda(torch.complex128))
    with pytest.raises(TypeError, match="complex128"):
        gbhegv._want(torch.complex128, dev, _FakeCuda(torch.complex64))
    with pytest.raises(TypeError):
        gbhegv._want(torch.float64, dev, _FakeCuda(torch.float32))
    with pytest.raises(ValueError, match="cuda:1"):
        gbhegv._want(torch.complex128, dev, _FakeCuda(torch.complex128, "cuda:1"))
    with pytest.raises(ValueError, match="CUDA"):
        gbhegv._want(torch.float64, dev, torch.zeros(3, dtype=torch.float64))
    with pytest.raises(ValueError, match="CUDA"):
        gbhegv._ptr(torch.zeros(3))
    assert gbhegv._ptr(None) is None


def test_shapes_are_checked():
    sq = torch.zeros((4, 4), dtype=torch.complex128)
    assert gbhegv._square(sq, sq) == 4
    with pytest.raises(ValueError, match="4 x 4"):
        gbhegv._square(sq, torch.zeros((3, 3), dtype=torch.complex128))
    with pytest.raises(ValueError):
        gbhegv._square(torch.zeros((4, 3), dtype=torch.complex128))
    with pytest.raises(ValueError):
        gbhegv._square(torch.zeros(4, dtype=torch.complex128))
    gbhegv._block(torch.zeros((4, 2)), 4, 2, "X")
    with pytest.raises(ValueError, match="X must be 4 x 3"):
        gbhegv._block(torch.zeros((4, 2)), 4, 3, "X")
    with pytest.raises(ValueError):
        gbhegv._block(torch.zeros((5, 3)), 4, 3, "X")


def test_gemm_operand_shapes_are_checked():
    """Operands too small (or too large) for (opA, opB, m, n, k) are refused
    before any pointer reaches the library (the C-ABI sees only ld)."""
    z = lambda r, c: torch.zeros((r, c), dtype=torch.complex128)  # noqa: E731
    assert gbhegv._gemm_dims("N", "N", z(5, 3), z(3, 4), z(5, 4)) == (5, 4, 3)
    assert gbhegv._gemm_dims("C", "N", z(3, 5), z(3, 4), z(5, 4)) == (5, 4, 3)
    assert gbhegv._gemm_dims("N", "C", z(5, 3), z(4, 3), z(5, 4)) == (5, 4, 3)
    assert gbhegv._gemm_dims("H", "T", z(5, 5), z(4, 5), z(5, 4)) == (5, 4, 5)
    with pytest.raises(ValueError, match="opN\\(A\\)"):
        gbhegv._gemm_dims("N", "N", z(4, 3), z(3, 4), z(5, 4))   # A has too few rows
    with pytest.raises(ValueError, match="opN\\(B\\)"):
        gbhegv._gemm_dims("N", "N", z(5, 3), z(2, 4), z(5, 4))   # B has too few rows
    with pytest.raises(ValueError, match="opN\\(B\\)"):
        gbhegv._gemm_dims("N", "N", z(5, 3), z(3, 3), z(5, 4))   # B has too few columns
    with pytest.raises(ValueError, match="opC\\(B\\)"):
        gbhegv._gemm_dims("N", "C", z(5, 3), z(3, 3), z(5, 4))
    with pytest.raises(ValueError, match="opH\\(A\\)"):
        gbhegv._gemm_dims("H", "N", z(5, 4), z(4, 4), z(5, 4))   # Hermitian A must be square
    with pytest.raises(ValueError, match="modes"):
        gbhegv._gemm_dims("X", "N", z(5, 3), z(3, 4), z(5, 4))
    with pytest.raises(ValueError, match="matrix"):
        gbhegv._gemm_dims("N", "N", torch.zeros(5, dtype=torch.complex128), z(3, 4), z(5, 4))


def test_gemm_entry_points_check_shapes_before_the_library(monkeypatch):
    """zgemm, zgemm_static and gemm_crt raise on mismatched operands before
    they touch a handle or the library."""
    monkeypatch.setattr(gbhegv, "_want", lambda *a, **k: None)
    monkeypatch.setattr(gbhegv, "handle", lambda *a, **k: pytest.fail("reached the library"))
    monkeypatch.setattr(gbhegv, "_load", lambda: pytest.fail("reached the library"))
    A = torch.zeros((4, 3), dtype=torch.complex128)
    B = torch.zeros((3, 4), dtype=torch.complex128)
    C = torch.zeros((5, 4), dtype=torch.complex128)
    for fn in (gbhegv.zgemm, gbhegv.zgemm_static, gbhegv.gemm_crt):
        with pytest.raises(ValueError, match="opN\\(A\\)"):
            fn("N", "N", A, B, C)


def test_adjoint_argument_lengths_are_checked(monkeypatch):
    monkeypatch.setattr(gbhegv, "_want", lambda *a, **k: None)
    monkeypatch.setattr(gbhegv, "handle", lambda *a, **k: pytest.fail("reached the library"))
    n, m = 6, 3
    X = torch.zeros((n, n), dtype=torch.complex128)
    w = torch.zeros(n, dtype=torch.float64)
    gw = torch.zeros(m, dtype=torch.float64)
    gX = torch.zeros((n, m), dtype=torch.complex128)
    with pytest.raises(ValueError, match="w_all"):
        gbhegv.hegv_adjoint(w[:n - 1], X, 1, m, gw, gX, 0.0)
    with pytest.raises(ValueError, match="gw"):
        gbhegv.hegv_adjoint(w, X, 1, m, gw[:m - 1], gX, 0.0)
    with pytest.raises(ValueError, match="gX"):
        gbhegv.hegv_adjoint(w, X, 1, m, gw, gX[:, :m - 1], 0.0)
    with pytest.raises(ValueError, match="gX"):
        gbhegv.hegv_adjoint(w, X, 1, m, gw, gX[:n - 1], 0.0)
    with pytest.raises(ValueError, match="il"):
        gbhegv.hegv_adjoint(w, X, 2, n + 1, gw, gX, 0.0)
    with pytest.raises(ValueError):
        gbhegv.hegv_adjoint(w, X[:, :n - 1], 1, m, gw, gX, 0.0)
