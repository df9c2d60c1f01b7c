"""Band-width rule and autotuner host logic (no GPU): the C lookup behind
nb = 0 against its documented semantics, the tuner's choice of winners and
rule entries with a fake timer, and the JSON cache."""
import math
import os
import random

import pytest

from paper_1207_1773_gb300 import autotune, gbhegv


def _default(n):
    return 16 if n <= 128 else (32 if n <= 1024 else 64)


def _spec_pick(rule, n, m):
    """The rule as the header states it, written out plainly."""
    if not rule:
        return _default(n)
    above = [e for e in rule if e[0] >= n]
    n_sel = min(e[0] for e in above) if above else max(e[0] for e in rule)
    group = [e for e in rule if e[0] == n_sel]
    f = m / n if n > 0 else 1.0
    fit = [e for e in group if e[1] >= f]
    if fit:
        best = min(e[1] for e in fit)
        e = next(e for e in group if e[1] == best)
    else:
        big = max(e[1] for e in group)
        e = next(e for e in group if e[1] == big)
    return e[2] if e[2] < n else _default(n)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1207_1773_gb300 import build
    build.build()


def test_empty_rule_is_default():
    for n in (0, 1, 100, 128, 129, 1024, 1025, 20000):
        assert gbhegv.nb_rule_pick([], n) == _default(n)


def test_rule_lookup_matches_spec_random():
    rnd = random.Random(7)
    for trial in range(300):
        k = rnd.randint(1, 8)
        ns = [rnd.choice([64, 200, 500, 1000, 3000, 10000]) for _ in range(k)]
        rule = [(nm, rnd.choice([0.1, 0.25, 0.5, 1.0]), rnd.choice([8, 16, 32, 48, 64])) for nm in ns]
        n = rnd.randint(1, 12000)
        m = rnd.randint(0, n)
        assert gbhegv.nb_rule_pick(rule, n, m) == _spec_pick(rule, n, m), (rule, n, m)


def test_rule_boundaries():
    rule = [(500, 0.3, 16), (500, 1.0, 32), (4000, 1.0, 64)]
    assert gbhegv.nb_rule_pick(rule, 500, 150) == 16     # m/n = 0.3 exactly: the 0.3 entry
    assert gbhegv.nb_rule_pick(rule, 500, 151) == 32
    assert gbhegv.nb_rule_pick(rule, 501, 10) == 64      # next size bucket
    assert gbhegv.nb_rule_pick(rule, 9000, 9000) == 64   # beyond the largest: the largest
    assert gbhegv.nb_rule_pick(rule, 20, 20) == 16       # 32 >= n = 20: the default for n = 20


def test_rule_argument_errors():
    lib = gbhegv._load()
    import ctypes
    out = ctypes.c_int()
    cnt, nm, fm, nbs = gbhegv._rule_arrays([(100, 1.0, 32)])
    assert lib.gbhe_nb_rule_pick(-1, nm, fm, nbs, 10, 10, ctypes.byref(out)) == -1
    assert lib.gbhe_nb_rule_pick(65, nm, fm, nbs, 10, 10, ctypes.byref(out)) == -1  # > GBHE_NB_RULE_MAX
    for bad, code in (([(0, 1.0, 32)], -2), ([(100, 0.0, 32)], -3), ([(100, 1.5, 32)], -3),
                      ([(100, float("nan"), 32)], -3), ([(100, 1.0, 0)], -4), ([(100, 1.0, 65)], -4)):
        c, a, b, d = gbhegv._rule_arrays(bad)
        assert lib.gbhe_nb_rule_pick(c, a, b, d, 10, 10, ctypes.byref(out)) == code, bad
    assert lib.gbhe_nb_rule_pick(cnt, nm, fm, nbs, 10, 11, ctypes.byref(out)) == -5
    assert lib.gbhe_nb_rule_pick(cnt, nm, fm, nbs, -1, 0, ctypes.byref(out)) == -5
    assert lib.gbhe_nb_rule_pick(cnt, nm, fm, nbs, 10, 10, None) == -6
    # handle entry points check the handle first (no device work)
    assert lib.gbhe_set_nb_rule(None, cnt, nm, fm, nbs) == -1
    assert lib.gbhe_resolve_nb(None, 10, 10, ctypes.byref(out)) == -1


def test_winner_and_rule_from_timings():
    assert autotune.winner({16: 2.0, 32: 1.0, 64: 1.5}) == 32
    assert autotune.winner({16: 1.0, 32: 1.0}) == 16  # ties to the smaller nb
    res = {(1000, 0.1): {16: 3.0, 32: 2.0, 64: 2.5},
           (1000, 1.0): {16: 3.0, 32: 2.5, 64: 2.0},
           (4000, 1.0): {16: 9.0, 32: 8.0, 64: 7.0}}
    rule = autotune.rule_from_timings(res)
    mid = int(math.floor(math.sqrt(1000 * 4000)))
    assert rule == [(mid, 0.55, 32), (mid, 1.0, 64), (4000, 1.0, 64)]
    # the rule gives every tuned point its winner
    for (n, f), tm in res.items():
        assert gbhegv.nb_rule_pick(rule, n, autotune.pairs_for(n, f)) == autotune.winner(tm)


def test_tune_with_fake_timer():
    calls = []

    def timer(n, m, nb):
        calls.append((n, m, nb))
        return abs(nb - (32 if n < 2000 else 64)) + 1.0 + 1e-3 * m / n

    res = autotune.tune([40, 1500, 3000], fracs=(0.25, 1.0), candidates=(16, 32, 64), timer=timer)
    assert set(res) == {(40, 0.25), (40, 1.0), (1500, 0.25), (1500, 1.0), (3000, 0.25), (3000, 1.0)}
    assert set(res[(40, 1.0)]) == {16, 32}                  # nb < n only
    assert (40, 10, 16) in calls and (1500, 375, 64) in calls
    rule = autotune.rule_from_timings(res)
    assert gbhegv.nb_rule_pick(rule, 1500, 1500) == 32
    assert gbhegv.nb_rule_pick(rule, 3000, 750) == 64
    with pytest.raises(ValueError):
        autotune.tune([100], fracs=(0.0,), timer=timer)
    assert autotune.tune([1], timer=timer) == {}            # no candidate below n


def test_cache_roundtrip(tmp_path):
    res = {(1000, 1.0): {16: 3.0, 32: 2.0}, (4000, 0.25): {32: 5.0, 64: 4.0}}
    p = os.path.join(tmp_path, "nb.json")
    autotune.save(p, res, "GPU-X")
    assert autotune.load(p, "GPU-X") == res
    assert autotune.load(p) == res
    assert autotune.load(p, "GPU-Y") is None
    assert autotune.load(os.path.join(tmp_path, "missing.json")) is None


def test_pairs_for():
    assert autotune.pairs_for(4096, 1.0) == 4096
    assert autotune.pairs_for(4096, 0.25) == 1024
    assert autotune.pairs_for(4096, 0.10) == 410
    assert autotune.pairs_for(3, 0.01) == 1
