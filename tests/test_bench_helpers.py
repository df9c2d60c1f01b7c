"""Host-side arithmetic of bench.py (no GPU): the nominal flop count and the
bulge chase's two rooflines."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_nominal_flops():
    n, m = 10000, 10000
    assert bench.nominal_flops(n, m) == pytest.approx(32.0 / 3.0 * n ** 3 + 12.0 * n * n * m)
    assert bench.nominal_flops(10000, 10000) == pytest.approx(2.267e13, rel=1e-3)


def test_chase_roofline():
    r = bench.chase_roofline({"ms": 500.0, "bytes": 1e9, "flops": 2e11}, 8000.0, 1.0)
    assert r["hbm_gbs"] == pytest.approx(2.0) and r["hbm_frac"] == pytest.approx(2.0 / 8000.0)
    assert r["fp64_tflops"] == pytest.approx(0.4) and r["dfma_frac"] == pytest.approx(0.4)
    assert bench.chase_roofline(None, 8000.0, 1.0) is None
    assert bench.chase_roofline({"ms": 0.0, "bytes": 1.0, "flops": 1.0}, 8000.0, 1.0) is None
    r = bench.chase_roofline({"ms": 1.0, "bytes": 1e6, "flops": 0.0}, None, None)
    assert r["hbm_frac"] is None and r["dfma_frac"] is None


def test_library_comparator_algebra():
    """The context comparator's solve (run on CUDA by --cusolver) is the
    generalized eigensolution: checked on the CPU at small n."""
    import numpy as np
    import torch
    from paper_1207_1773_gb300 import inputs
    n = 40
    A, B, lam = inputs.make_pair(n, 3)
    At, Bt = torch.from_numpy(A), torch.from_numpy(B)
    w, X = bench.library_solve(At, Bt)
    eps = np.finfo(np.float64).eps
    assert np.max(np.abs(w.numpy() - lam)) <= 10 * n * eps * np.linalg.norm(A, 2) / np.linalg.eigvalsh(B).min()
    R = At @ X - (Bt @ X) * w[None, :]
    assert torch.linalg.norm(R).item() <= 100 * n * eps * torch.linalg.norm(At).item() * torch.linalg.norm(X).item()
    O = X.conj().T @ Bt @ X - torch.eye(n, dtype=torch.complex128)
    assert torch.linalg.norm(O).item() <= 100 * n * eps


def test_contraction_flops_and_tensor_roofline():
    """The algorithmic FP64 flops of the engine-served stages at n = m = 10000
    (potrf 4n^3/3 + hegst 4n^3 + he2hb 16n^3/3 + Q2 8n^2m + Q1 8n^2m + trsm 4n^2m
    = 3.0667e13), and the roofline built from them: 16 x those flops over the
    product kernels' time, independent of what the engine counted as executed."""
    import bench
    n = m = 10000
    assert abs(bench.contraction_flops(n, m) - (32.0 / 3.0 * n ** 3 + 20.0 * n * n * m)) < 1.0
    assert abs(bench.contraction_flops(n, m) / 3.0666666666666668e13 - 1.0) < 1e-12
    prof = {"crt_mma": {"ms": 2 * 3096.0, "flops": 2 * 4.69e13, "launches": 2 * 2978}}
    tr = bench.tensor_roofline(prof, n, m, 2, 1941.1)
    assert abs(tr["achieved"] - 16 * 3.0666666666666668e13 / 3.096 / 1e12) < 1e-6
    assert abs(tr["frac"] - tr["achieved"] / 1941.1) < 1e-12
    assert abs(tr["executed_fp64_flops_per_solve"] - 4.69e13) < 1.0
    assert bench.tensor_roofline({"crt_mma": {"ms": 0.0, "flops": 0.0, "launches": 0}}, n, m, 1, 1.0) is None


def test_product_traffic_scaling(monkeypatch):
    """Traffic per launch = bytes per algorithmic flop (from the capture of a
    smaller solve) x the solve's algorithmic flops / its launches; None
    without a capture of the current kernels."""
    monkeypatch.setitem(bench.PRODUCT_TRAFFIC, "bytes_per_algorithmic_flop", None)
    assert bench.product_traffic(3e13, 5000) is None
    monkeypatch.setitem(bench.PRODUCT_TRAFFIC, "bytes_per_algorithmic_flop", 0.1)
    assert bench.product_traffic(3e13, 5000) == pytest.approx(6e8)
    assert bench.product_traffic(3e13, 0) is None
    assert bench.product_traffic(3e13, 5000, 10000, 10000) == pytest.approx(6e8)
    assert bench.product_traffic(3e13, 5000, 10000, 2500) is None     # the other Q2 path
