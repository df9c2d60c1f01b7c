"""The band-width autotuner on the GPU: it times real solves, installs a rule
whose lookup gives each tuned point its fastest nb, and a solve with nb = 0
then uses that rule and still meets the oracle's eigenvalue bound."""
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


def test_autotune_installs_rule_and_solves(G):
    from paper_1207_1773_gb300 import autotune
    h = G.handle(DEV)
    try:
        results = autotune.tune([200, 400], fracs=(0.5, 1.0), candidates=(16, 32), handle=h, reps=1)
        assert set(results) == {(200, 0.5), (200, 1.0), (400, 0.5), (400, 1.0)}
        for tm in results.values():
            assert set(tm) == {16, 32} and all(0.0 < t < 60.0 for t in tm.values())
        rule = autotune.rule_from_timings(results)
        h.set_nb_rule(rule)
        for (n, f), tm in results.items():
            assert h.resolve_nb(n, autotune.pairs_for(n, f)) == autotune.winner(tm)
        n = 400
        A, B, lam = inputs.make_pair(n, 5)
        w, X = G.hegv(G.colmajor(A, DEV), G.colmajor(B, DEV))  # nb = 0: the rule
        w = w.cpu().numpy()
        wo, _, info = oracle.hegv(A, B)
        assert info == 0
        tol = 10 * n * EPS * np.linalg.norm(A, 2) / np.linalg.eigvalsh(B).min()
        assert np.max(np.abs(w - wo)) <= tol
    finally:
        h.set_nb_rule([])
    assert h.resolve_nb(400) == G._load().gbhe_default_nb(400)
