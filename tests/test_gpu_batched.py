"""Batched solves of uneven-size problems on worker streams, directly and
replayed from one captured CUDA graph; every problem against the oracle."""
import math

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


def _check(A, B, lam, w, X, n, m):
    import oracle
    wo, _, info = oracle.hegv(A, B, 1, m)
    assert info == 0
    tol = 10 * n * EPS * np.linalg.norm(A, 2) / np.linalg.eigvalsh(B).min()
    assert np.max(np.abs(w - wo)) <= tol
    assert np.max(np.abs(w - lam[:m])) <= tol
    res = np.linalg.norm(A @ X - (B @ X) * w[None, :]) / (n * EPS * np.linalg.norm(A) * np.linalg.norm(X))
    orth = np.linalg.norm(X.conj().T @ B @ X - np.eye(m)) / (n * EPS)
    assert res <= 100 and orth <= 100, (n, res, orth)


def test_batched_direct_and_graph(G):
    from paper_1207_1773_gb300 import inputs
    rng = np.random.default_rng(3)
    ns = [int(v) for v in rng.integers(40, 320, 10)]
    ms = [math.ceil(n / 4) for n in ns]
    nbs = [16 if n < 128 else 32 for n in ns]
    pairs = [inputs.make_pair(n, 100 + i) for i, n in enumerate(ns)]
    A0 = [G.colmajor(A, DEV) for A, _, _ in pairs]
    B0 = [G.colmajor(B, DEV) for _, B, _ in pairs]
    As = [a.clone() for a in A0]
    Bs = [b.clone() for b in B0]
    ws = [torch.zeros(m, dtype=torch.float64, device=DEV) for m in ms]
    Xs = [torch.zeros((m, n), dtype=torch.complex128, device=DEV).t() for n, m in zip(ns, ms)]
    pool = G.BatchPool(4, DEV)
    pool.prepare(ns, nbs, ms)
    G.hegv_batched(pool, As, Bs, [1] * len(ns), ms, nbs, ws, Xs)
    torch.cuda.synchronize()
    for h in pool.handles:
        assert h.status() == 0
    direct = [(w.cpu().numpy(), X.cpu().numpy()) for w, X in zip(ws, Xs)]
    for (A, B, lam), (w, X), n, m in zip(pairs, direct, ns, ms):
        _check(A, B, lam, w, X, n, m)
    # one graph: restore the inputs, solve all; replayed twice
    for w, X in zip(ws, Xs):
        w.zero_()
        X.zero_()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(DEV)
    side.wait_stream(torch.cuda.current_stream(DEV))
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
            for a, a0, b, b0 in zip(As, A0, Bs, B0):
                a.copy_(a0)
                b.copy_(b0)
            G.hegv_batched(pool, As, Bs, [1] * len(ns), ms, nbs, ws, Xs)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        for h in pool.handles:
            assert h.status() == 0
        for (w0, X0), w, X, n in zip(direct, ws, Xs, ns):
            tol = 1e3 * n * EPS * max(1.0, np.max(np.abs(w0)))
            assert np.max(np.abs(w.cpu().numpy() - w0)) <= tol


def test_batched_workload_sizes(G):
    """The batched workload's shapes: 64 pairs, n ~ U[500, 3000] (seed 3),
    lowest 25 % each, in one captured CUDA graph on 8 worker streams.  Every
    problem: eigenvalues against its constructed spectrum (10 n eps ||A|| ||B^-1||
    with ||A|| <= ||B|| max|Lambda|), residual and B-orthonormality ratios on 32
    sampled columns (formed on the device); the smallest problem and the one
    nearest n = 1000 also element by element against the oracle."""
    from paper_1207_1773_gb300 import inputs
    rng = np.random.default_rng(3)
    ns = [int(v) for v in rng.integers(500, 3001, 64)]
    ms = [math.ceil(n / 4) for n in ns]
    nbs = [32 if n < 1024 else 64 for n in ns]
    dev = torch.device(DEV)
    pairs = [inputs.make_pair(n, 1000 + i, "uniform", -1.0, 1.0, device=dev) for i, n in enumerate(ns)]
    A0 = [G.colmajor(A, DEV) for A, _, _ in pairs]
    B0 = [G.colmajor(B, DEV) for _, B, _ in pairs]
    As = [a.clone() for a in A0]
    Bs = [b.clone() for b in B0]
    ws = [torch.zeros(m, dtype=torch.float64, device=DEV) for m in ms]
    Xs = [torch.zeros((m, n), dtype=torch.complex128, device=DEV).t() for n, m in zip(ns, ms)]
    pool = G.BatchPool(8, DEV)
    pool.prepare(ns, nbs, ms)
    G.hegv_batched(pool, As, Bs, [1] * len(ns), ms, nbs, ws, Xs)  # one-time set-ups outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(DEV)
    side.wait_stream(torch.cuda.current_stream(DEV))
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
            for a, a0, b, b0 in zip(As, A0, Bs, B0):
                a.copy_(a0)
                b.copy_(b0)
            G.hegv_batched(pool, As, Bs, [1] * len(ns), ms, nbs, ws, Xs)
    for w, X in zip(ws, Xs):
        w.zero_()
        X.zero_()
    g.replay()
    torch.cuda.synchronize()
    for h in pool.handles:
        assert h.status() == 0
    for i, ((A, B, lam), a0, b0, w, X, n, m) in enumerate(zip(pairs, A0, B0, ws, Xs, ns, ms)):
        ev = torch.linalg.eigvalsh(b0).cpu().numpy()
        tol = 10 * n * EPS * np.max(np.abs(lam)) * ev[-1] / ev[0]
        wn = w.cpu().numpy()
        assert np.max(np.abs(wn - lam[:m])) <= tol, (i, n)
        cols = torch.from_numpy(np.unique(np.linspace(0, m - 1, 32).astype(int))).to(DEV)
        Xc, wc = X[:, cols], w[cols]
        res = (torch.linalg.norm(a0 @ Xc - (b0 @ Xc) * wc[None, :])
               / (n * EPS * torch.linalg.norm(a0) * torch.linalg.norm(Xc))).item()
        orth = (torch.linalg.norm(Xc.conj().t() @ (b0 @ Xc) - torch.eye(len(cols), dtype=torch.complex128,
                                                                         device=DEV)) / (n * EPS)).item()
        assert res <= 100 and orth <= 100, (i, n, res, orth)
    near = int(np.argmin([abs(n - 1000) for n in ns]))
    for i in sorted({int(np.argmin(ns)), near}):
        A, B, lam = pairs[i]
        _check(A, B, lam, ws[i].cpu().numpy(), Xs[i].cpu().numpy(), ns[i], ms[i])
