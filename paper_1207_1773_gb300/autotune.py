"""Band-width autotuner for the two-stage solve.

The band width nb is a free parameter of the two-stage reduction (Section
4.2): a wider band makes stage 1's panels and trailing products larger and
the stage-2 bulge chase and the Q2 back-transform (both O(n^2 nb) work)
slower.  The tuner times ``gbhe_hegv`` for candidate band widths on seeded
synthetic pairs of the sizes and eigenvector fractions asked for (the pair
construction of ``inputs.make_pair``), keeps the fastest nb per (n, fraction)
and installs the result on a handle as its band-width rule, which is what
nb = 0 then selects (``gbhe_set_nb_rule``).  Results can be cached in a JSON
file keyed by the device name.

Rule entries are (n_max, frac_max, nb): each tuned size owns the orders up to
the geometric midpoint to the next tuned size (the largest tuned size owns
everything above), each tuned fraction the fractions up to the midpoint to
the next tuned fraction (the largest owns everything up to 1).
"""
from __future__ import annotations

import json
import math
import os

CANDIDATES = (16, 32, 64)


def pairs_for(n, frac):
    """Number of selected eigenpairs for the lowest fraction `frac` of n."""
    return max(1, min(n, int(math.ceil(frac * n - 1e-9))))


def winner(timings):
    """The fastest nb of {nb: seconds}; ties go to the smaller nb."""
    return min(sorted(timings), key=lambda nb: (timings[nb], nb))


def rule_from_timings(results):
    """{(n, frac): {nb: seconds}} -> [(n_max, frac_max, nb), ...]."""
    sizes = sorted({n for n, _ in results})
    rule = []
    for i, n in enumerate(sizes):
        n_max = n if i + 1 == len(sizes) else int(math.floor(math.sqrt(n * sizes[i + 1])))
        fracs = sorted(f for (nn, f) in results if nn == n)
        for j, f in enumerate(fracs):
            f_max = 1.0 if j + 1 == len(fracs) else 0.5 * (f + fracs[j + 1])
            rule.append((n_max, f_max, winner(results[(n, f)])))
    return rule


class GpuTimer:
    """Seconds of one two-stage solve (best of `reps` after one warm-up), CUDA
    events on the current stream around gbhegv.hegv, on a fresh copy of the
    seeded pair each time (the solve overwrites A and B)."""

    def __init__(self, handle, seed=0, reps=2):
        self.h = handle
        self.seed = seed
        self.reps = reps
        self._pairs = {}

    def _pair(self, n):
        if n not in self._pairs:  # one size held at a time
            from . import gbhegv, inputs
            dev = self.h.device
            A, B, _ = inputs.make_pair(n, self.seed, device=dev if n > 512 else None)
            self._pairs = {n: (gbhegv.colmajor(A, dev), gbhegv.colmajor(B, dev))}
        return self._pairs[n]

    def __call__(self, n, m, nb):
        import torch
        from . import gbhegv
        A0, B0 = self._pair(n)
        dev = self.h.device
        gbhegv.handle(dev).ensure_workspace(n, nb, m)
        st = torch.cuda.current_stream(dev)
        best = math.inf
        for r in range(self.reps + 1):
            A = torch.empty_strided((n, n), (1, n), dtype=A0.dtype, device=dev).copy_(A0)
            B = torch.empty_strided((n, n), (1, n), dtype=B0.dtype, device=dev).copy_(B0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            gbhegv.hegv(A, B, 1, m, nb=nb, check=False)
            e1.record(st)
            status = gbhegv.handle(dev).status()
            if status != 0:
                raise gbhegv.GbheError("gbhe_hegv", status)
            if r > 0:
                best = min(best, e0.elapsed_time(e1) / 1e3)
        return best


def tune(sizes, fracs=(1.0,), candidates=CANDIDATES, timer=None, handle=None, seed=0, reps=2):
    """Time every candidate nb (1 <= nb <= 64, nb < n) at every (n, frac);
    returns {(n, frac): {nb: seconds}}.  `timer(n, m, nb)` -> seconds
    replaces the GPU timing."""
    if timer is None:
        from . import gbhegv
        timer = GpuTimer(handle if handle is not None else gbhegv.handle(), seed, reps)
    out = {}
    for n in sorted(set(int(s) for s in sizes)):
        for f in sorted(set(float(x) for x in fracs)):
            if not 0.0 < f <= 1.0:
                raise ValueError("fractions lie in (0, 1]")
            cands = [nb for nb in candidates if 1 <= nb <= 64 and nb < n]
            if not cands:
                continue
            m = pairs_for(n, f)
            out[(n, f)] = {nb: float(timer(n, m, nb)) for nb in cands}
    return out


def save(path, results, device_name):
    data = {"device": device_name,
            "entries": [{"n": n, "frac": f, "seconds": {str(nb): t for nb, t in sorted(tm.items())}}
                        for (n, f), tm in sorted(results.items())]}
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1)
    os.replace(tmp, path)


def load(path, device_name=None):
    """Cached results, or None when the file is missing or was written for
    another device."""
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        data = json.load(fh)
    if device_name is not None and data.get("device") != device_name:
        return None
    return {(int(e["n"]), float(e["frac"])): {int(k): float(v) for k, v in e["seconds"].items()}
            for e in data["entries"]}


def autotune(handle=None, sizes=(1024, 4096), fracs=(1.0,), candidates=CANDIDATES, cache=None, seed=0,
             reps=2, timer=None):
    """Tune (or read the cache), install the rule on the handle and return it."""
    from . import gbhegv
    h = handle if handle is not None else gbhegv.handle()
    dev_name = None
    if timer is None:
        import torch
        dev_name = torch.cuda.get_device_name(h.device)
    results = load(cache, dev_name) if cache else None
    if results is None:
        results = tune(sizes, fracs, candidates, timer=timer, handle=h, seed=seed, reps=reps)
        if cache:
            save(cache, results, dev_name)
    rule = rule_from_timings(results)
    h.set_nb_rule(rule)
    return rule
