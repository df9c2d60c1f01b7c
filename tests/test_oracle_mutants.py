"""Pin strength: plausible mistakes planted in a copy of the oracle must fail.

Each mutant is a textual change to a temporary copy of ``oracle/oracle.c``
(a dropped term, a wrong sign, a missing conjugate, a wrong order), compiled
on the CPU; the pins of the definition (constructed spectrum, residual ratio,
B-orthonormality, ascending order) must reject every one of them, and must
accept the unmodified source.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1207_1773_gb300 import inputs

EPS = np.finfo(np.float64).eps
SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "potrf_no_conj": ("zc ljk = conj(AT(B, j, k, ldb));", "zc ljk = AT(B, j, k, ldb);"),
    "hegst_transpose_no_conj": ("AT(Y, i, j, n) = conj(AT(W, j, i, n));", "AT(Y, i, j, n) = AT(W, j, i, n);"),
    "reflector_tau_conj": ("zc tau = (beta - alpha) / beta;", "zc tau = (beta - conj(alpha)) / beta;"),
    "hetrd_dropped_term": ("-= v[i] * conj(p[j]) + p[i] * conj(v[j]);", "-= v[i] * conj(p[j]);"),
    "hetrd_half_factor": ("zc half = 0.5 * t * pv;", "zc half = t * pv;"),
    "steqr_sign": ("d[k + 1] = s * s * a - 2.0 * c * s * b + c * c * cc;",
                   "d[k + 1] = s * s * a + 2.0 * c * s * b + c * c * cc;"),
    "steqr_vector_rotation": ("AT(Z, row, k + 1, ldz) = -s * zk + c * zk1;",
                              "AT(Z, row, k + 1, ldz) = s * zk + c * zk1;"),
    "unmtr_wrong_order": ("for (int k = n - 2; k >= 0; --k) {", "for (int k = 0; k <= n - 2; ++k) {"),
    "trsm_no_conj": ("s -= conj(AT(L, j, i, ldl)) * AT(X, j, c, ldx);", "s -= AT(L, j, i, ldl) * AT(X, j, c, ldx);"),
    "sort_descending": ("while (j >= 0 && w[idx[j]] > w[t])", "while (j >= 0 && w[idx[j]] < w[t])"),
}


def _pins_pass(n=24, seed=21):
    A, B, lam = inputs.make_pair(n, seed, "uniform", -3, 3)
    w, X, info = oracle.hegv(A, B)
    if info != 0 or not np.all(np.isfinite(w)) or not np.all(np.isfinite(X)):
        return False
    tol = 10 * n * EPS * np.linalg.norm(A, 2) / np.linalg.eigvalsh(B).min()
    ok = np.all(np.diff(w) >= 0) and np.max(np.abs(w - lam)) < tol
    res = np.linalg.norm(A @ X - (B @ X) * w[None, :]) / (n * EPS * np.linalg.norm(A) * np.linalg.norm(X))
    orth = np.linalg.norm(X.conj().T @ B @ X - np.eye(n)) / (n * EPS)
    return bool(ok and res < 30 and orth < 30)


def _build(tmp_path, name, mutation):
    src = open(SRC).read()
    if mutation is not None:
        old, new = mutation
        assert src.count(old) == 1, name
        src = src.replace(old, new)
    c = tmp_path / (name + ".c")
    so = tmp_path / (name + ".so")
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"])
    return oracle.bind(str(so))


def test_unmodified_source_passes(tmp_path, monkeypatch):
    monkeypatch.setattr(oracle, "_lib", _build(tmp_path, "control", None))
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, monkeypatch, name):
    monkeypatch.setattr(oracle, "_lib", _build(tmp_path, name, MUTANTS[name]))
    assert not _pins_pass(), "planted mistake %s was not caught" % name
