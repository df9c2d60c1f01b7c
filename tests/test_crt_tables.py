"""Number theory of the tensor-core FP64 engine, on the tables exactly as the
library copies them to the device (host-only, no GPU): the moduli are
pairwise coprime and small enough for exact FP16 residues and exact FP32
chunk sums, their product leaves the margin the reconstruction relies on, the
CRT weights form the idempotent basis, the limb weights are what their
definition says, the FP32 residue split is exact over the operand range, and
reconstruction from residues returns every integer in the engine's range."""
import math
import random

import numpy as np
import pytest

from paper_1207_1773_gb300 import gbhegv

KMAX = 1 << 16        # largest contraction the engine accepts
VMAX = 1 << 52        # operands are scaled to integers |v| <= 2^52


@pytest.fixture(scope="module")
def T():
    from paper_1207_1773_gb300 import build
    build.build()
    return gbhegv.crt_tables()


def test_moduli(T):
    p = T["p"]
    assert len(p) == 16 and len(set(p)) == 16
    assert all(2 <= x <= 256 for x in p)
    for i in range(16):
        for j in range(i + 1, 16):
            assert math.gcd(p[i], p[j]) == 1, (p[i], p[j])
    # symmetric residues |r| <= 128 are exact in FP16 (11-bit significand)
    assert max(p) // 2 <= 2048
    # a chunk of 512 products |r r'| <= 128^2 sums below 2^23: exact in FP32
    assert 512 * (max(p) // 2) ** 2 <= 1 << 23


def test_product_and_margin(T):
    M = math.prod(T["p"])
    assert T["M"] == M
    # complex: |Re C|, |Im C| <= K * 2 * VMAX^2 = K 2^105, and this must stay below M / 8
    assert 8 * KMAX * 2 * VMAX * VMAX < M


def test_crt_basis(T):
    p, W, M = T["p"], T["W"], T["M"]
    for l, Wl in enumerate(W):
        assert 0 <= Wl < M
        for j, pj in enumerate(p):
            assert Wl % pj == (1 if j == l else 0), (l, j)


def _sym(x, p):
    r = x % p
    return r - p if r > p // 2 else r


def test_limb_weights(T):
    for pl, k13, k26, k39 in zip(T["p"], T["k13"], T["k26"], T["k39"]):
        assert (k13, k26, k39) == (_sym(1 << 13, pl), _sym(1 << 26, pl), _sym(1 << 39, pl))
        assert max(abs(k13), abs(k26), abs(k39)) <= 128


def test_reconstruction_roundtrip(T):
    p, W, M = T["p"], T["W"], T["M"]
    bound = KMAX * 2 * VMAX * VMAX
    rnd = random.Random(1)
    cases = [0, 1, -1, bound, -bound] + [rnd.randint(-bound, bound) for _ in range(2000)]
    for C in cases:
        res = [C % pl for pl in p]
        res = [r - pl if r > pl // 2 else r for r, pl in zip(res, p)]   # symmetric residues
        assert all(abs(r) <= 128 for r in res)
        s = sum(r * Wl for r, Wl in zip(res, W)) % M
        if s > M // 2:
            s -= M
        assert s == C


def _fmaf(a, b, c):
    """float32 fused multiply-add: a*b + c is exact in float64 for a an 8-bit
    integer, b and c float32 below 2^12 (fewer than 53 significant bits), so
    one rounding to float32 gives the fused result."""
    return np.float32(float(a) * float(b) + float(c))


def test_quotient_estimate_and_160bit_reconstruction(T):
    """The device sums unsigned residues c_l in [0, p_l): S = sum c_l W_l,
    F = fmaf chain of c_l * frac_l (l = 0..15), q = rintf(F), C = S - q M.
    Over the engine's whole range this returns C exactly; the FP32 estimate
    stays within 2^-8 of the exact sum_l c_l y_l / p_l."""
    p, W, M, frac = T["p"], T["W"], T["M"], T["frac"]
    y = [(pow(M // pl, -1, pl)) for pl in p]
    for l, pl in enumerate(p):
        assert frac[l] == np.float32(y[l] / pl)
    bound = KMAX * 2 * VMAX * VMAX
    rnd = random.Random(2)
    cases = [0, 1, -1, bound, -bound, bound - 1, -bound + 1] + [rnd.randint(-bound, bound) for _ in range(3000)]
    worst = 0.0
    for C in cases:
        cv = [C % pl for pl in p]
        F = np.float32(0.0)
        for l in range(16):
            F = _fmaf(np.float32(cv[l]), np.float32(frac[l]), F)
        exact = sum(c * yl / pl for c, yl, pl in zip(cv, y, p))
        worst = max(worst, abs(float(F) - exact))
        q = int(np.rint(F))                      # round half to even, as rintf
        S = sum(c * Wl for c, Wl in zip(cv, W))
        assert S - q * M == C, C
    assert worst < 2.0 ** -8, worst


def test_residue_split_replay(T):
    """The device's residue of a scaled integer |v| <= 2^52: four signed
    13-bit limbs l_i (the sign of v on each), t = l0 + l1 w1 + l2 w2 + l3 w3
    by an FP32 fma chain with the symmetric limb weights w_i, then
    r = fmaf(-rintf(t * pinv), p, t) with pinv = 1/p rounded to float.  Every
    partial sum of t is an integer below 2^23 (so the fma chain is exact, and
    so is the final fma, whose result is an integer), the only rounding is
    t * pinv; the replay checks that r = v mod p with |r| <= 128 (within
    the bound of the FP32 chunk sums), and that the device's fold of 128 to
    -128 (p = 256 only) gives a signed byte congruent to v."""
    rng = np.random.default_rng(3)
    top = 1 << 52
    # largest magnitude that the rounding to 52 bits can produce: (2^53 - 1 + 1) >> 1
    assert ((1 << 53) - 1 + 1) >> 1 == top
    mags = np.array([0, 1, top, top - 1, (1 << 39) - 1, 1 << 39, (1 << 26) - 1, (1 << 13) - 1] +
                    [int(x) for x in rng.integers(0, top, 20000, dtype=np.int64)], dtype=np.int64)
    limbs = [(mags >> (13 * i)) & 0x1FFF for i in range(3)] + [mags >> 39]
    assert int(limbs[3].max()) <= 1 << 13
    for pl, k13, k26, k39 in zip(T["p"], T["k13"], T["k26"], T["k39"]):
        pinv = np.float32(1.0) / np.float32(pl)
        for sign in (1, -1):
            l0, l1, l2, l3 = (sign * x for x in limbs)
            t = l0 + l1 * k13 + l2 * k26 + l3 * k39       # exact integers (int64)
            for part in (l0 + l1 * k13, l0 + l1 * k13 + l2 * k26, t):
                assert int(np.abs(part).max()) < 1 << 23
            q = np.rint(t.astype(np.float32) * pinv).astype(np.int64)   # one float32 rounding, half to even
            r = t - q * pl
            assert int(np.abs(r).max()) <= 128
            assert np.all((r - sign * mags) % pl == 0)
            b = np.where(r > 127, r - pl, r)                # the stored signed byte
            assert int(b.min()) >= -128 and int(b.max()) <= 127
            assert np.all((b - sign * mags) % pl == 0)
            if pl % 2:                                      # odd moduli never reach 128
                assert int(np.abs(r).max()) <= 127


def _int160_to_double(C, sc):
    """Replay of the device's 160-bit two's-complement integer -> double
    conversion (leading word and two below it, sticky bit for the rest,
    round to nearest even, carry into a new bit, scale 2^sc, flush below the
    normal range)."""
    M64 = (1 << 64) - 1
    D = [(C >> (32 * i)) & 0xFFFFFFFF for i in range(5)]   # two's complement words
    negv = D[4] >= 1 << 31
    if negv:
        v = (-C) & ((1 << 160) - 1)
        D = [(v >> (32 * i)) & 0xFFFFFFFF for i in range(5)]
    for top in (4, 3, 2, 1, 0):
        if D[top]:
            break
    else:
        return 0.0
    t2 = D[top]
    t1 = D[top - 1] if top >= 1 else 0
    t0 = D[top - 2] if top >= 2 else 0
    sticky = any(D[i] for i in range(0, max(top - 2, 0)))
    lz = 32 - t2.bit_length()
    hi = (t2 << 32) | t1
    lo = (t0 << 32) & M64
    if lz:
        hi = ((hi << lz) | (lo >> (64 - lz))) & M64
        lo = (lo << lz) & M64
    sticky = sticky or lo != 0
    mant, rem = hi >> 11, hi & 0x7FF
    if rem > 0x400 or (rem == 0x400 and (sticky or mant & 1)):
        mant += 1
        if mant == 1 << 53:
            mant >>= 1
            sc += 1
    e2 = 32 * top + 31 - lz - 52 + sc
    expo = e2 + 52 + 1023
    if expo <= 0:
        return 0.0
    if expo >= 2047:
        return -math.inf if negv else math.inf
    return math.ldexp(-mant if negv else mant, e2)


def test_int160_to_double_rounds_once_to_nearest_even():
    rnd = random.Random(4)
    cases = [1, -1, 2, (1 << 53) - 1, 1 << 53, (1 << 53) + 1, (1 << 54) + 2, (1 << 54) + 6,
             (1 << 127) - 1, -(1 << 127), (1 << 159) - 1, -(1 << 159)]
    for _ in range(3000):
        k = rnd.randint(54, 150)
        m = rnd.getrandbits(53) | (1 << 52)
        s = k - 53
        base = m << s
        half = 1 << (s - 1)
        cases += [base, base + half, base + half - 1, base + half + 1, base - 1, rnd.getrandbits(k)]
    for C in cases:
        for v in (C, -C):
            if not -(1 << 159) <= v < 1 << 159:
                continue
            assert _int160_to_double(v, 0) == float(v), v
            assert _int160_to_double(v, -104) == math.ldexp(float(v), -104), v


def _crt_ws(m, n, k, cplx):
    import ctypes
    out = ctypes.c_size_t()
    rc = gbhegv._load().gbhe_crt_workspace_size(m, n, k, cplx, ctypes.byref(out))
    return rc, out.value


def test_crt_workspace_matches_the_layout(T):
    """Residue planes 16 x (Re, Im) x rows x K padded to 32 (bytes) for both
    operands, output residue bytes in 128 x 64 tiles per modulus and
    component, one exponent per row and column, plus alignment."""
    for m, n, k, cplx in [(1, 1, 1, 1), (128, 64, 32, 0), (129, 65, 33, 1), (4096, 4096, 64, 1),
                          (10000, 10000, 10000, 1), (300, 7000, 65536, 0)]:
        nc = 2 if cplx else 1
        kp = -(-k // 32) * 32
        tiles = -(-m // 128) * -(-n // 64)
        want = 16 * nc * (m + n) * kp + tiles * 16 * nc * 128 * 64 + (m + n) * 4 + 4 * 256
        rc, got = _crt_ws(m, n, k, cplx)
        assert rc == 0 and got == want, (m, n, k, cplx, got, want)
    # about 9.7 GB for one complex product of order 10000 in every dimension
    assert abs(_crt_ws(10000, 10000, 10000, 1)[1] / 1e9 - 9.66) < 0.05
    assert _crt_ws(-1, 1, 1, 1)[0] == -1
    assert _crt_ws(1, -1, 1, 1)[0] == -2
    assert _crt_ws(1, 1, 65537, 1)[0] == -3          # beyond the exactness bound K <= 2^16


def _prmt(a, b, sel):
    """PTX prmt.b32 (default mode): byte i of the result is byte
    (sel >> 4 i) & 7 of the eight bytes b:a (a the low four)."""
    src = [(a >> (8 * i)) & 0xFF for i in range(4)] + [(b >> (8 * i)) & 0xFF for i in range(4)]
    return sum(src[(sel >> (4 * i)) & 7] << (8 * i) for i in range(4))


def test_byte_widening_replay():
    """The product kernels' producers widen 16 stored signed bytes (residues
    at k .. k+15 of one row) to two FP16 core-matrix rows: each byte is
    biased by xor 0x80, placed under the exponent bits of 1024 by prmt
    (0x64uu = 1024 + u in FP16) and 1152 (0x6480) is subtracted.  The replay
    checks every byte value and the element order of both rows."""
    one = np.array([0x6480], dtype=np.uint16).view(np.float16)[0]
    assert float(one) == 1152.0
    b = np.arange(-128, 128)
    u = (b & 0xFF) ^ 0x80
    h = (0x6400 | u).astype(np.uint16).view(np.float16)
    assert np.all(h.astype(np.float64) == 1024 + u)
    assert np.all((h - one).astype(np.float64) == b)      # FP16 difference, exact
    rng = np.random.default_rng(5)
    for _ in range(50):
        row = rng.integers(-128, 128, 16)
        words = [int(sum(((int(row[4 * w + i]) & 0xFF) << (8 * i)) for i in range(4))) for w in range(4)]
        biased = [x ^ 0x80808080 for x in words]
        out = []
        for x in biased:
            for sel in (0x4140, 0x4342):
                pair = _prmt(x, 0x64646464, sel)
                halves = np.array([pair & 0xFFFF, pair >> 16], dtype=np.uint16).view(np.float16)
                out.extend((halves - one).astype(np.float64))
        assert out == [float(v) for v in row]                 # lo row k..k+7, hi row k+8..k+15
