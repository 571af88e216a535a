"""The FP64-storage stencils' integer-digit arithmetic, emulated bit by bit on the CPU (no GPU, no
library call): the split of a value into two digits on its tile's grid, the int32 digit sums, the
ties-to-even rounding and the one-FMA scaling of the combination, and the cubic user function's
integer term Q formed in packed FP32 double-float steps.  Each step is written here from its
definition (integer shifts, IEEE round-to-nearest-even, one rounding per FMA) and the results are
checked against exact rational arithmetic:

* the digits are the two's-complement value sgn(x) floor(|x| / 2^(G-F)), low digit in [0, 2^DB);
* the rounding of the digit sums is round-half-even, exhaustively over a window;
* a sum of integer-weight taps is within (2^-47 + 2^-44 / sum|n| + 2^-50) of sum|w| * max|x|
  for 24-bit digits, and within (2^-55 + 2^-48 / sum|n| + 2^-50) for 28-bit digits (the last term:
  the weight scale c rounded to 51 bits, and the FMA's own rounding);
* Q is within one unit U = c 2^(G-44) of (u^3 - u) / U, across exponents and at the extremum of
  u^3 - u; the whole user function c^3 - c - Lap c is within the digit bound plus 2^-46.

These are the bounds the library's header states for CS_FP64_AUTO; the GPU parity tests compare
the kernels with the oracle at 1e-12 of the same scale.
"""
import math
import struct
from fractions import Fraction as Fr

import numpy as np
import pytest

f32 = np.float32


# ---- bit helpers -----------------------------------------------------------------------------
def dbits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def dfrom(b: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", b & (2 ** 64 - 1)))[0]


def fbits(x) -> int:
    return struct.unpack("<I", struct.pack("<f", float(x)))[0]


def ffrom(b: int):
    return f32(struct.unpack("<f", struct.pack("<I", b & 0xFFFFFFFF))[0])


def round_f32(x: Fr):
    """x rounded to the nearest float32, ties to even (normal range)."""
    if x == 0:
        return f32(0.0)
    neg, a = x < 0, abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fr(2) ** e > a:
        e -= 1
    while Fr(2) ** (e + 1) <= a:
        e += 1
    e = max(e, -126)
    q = a / Fr(2) ** (e - 23)
    n = q.numerator // q.denominator
    rem = q - n
    if rem > Fr(1, 2) or (rem == Fr(1, 2) and n % 2 == 1):
        n += 1
    v = float(n * Fr(2) ** (e - 23))
    return f32(-v if neg else v)


def fmul(a, b):
    return round_f32(Fr(float(a)) * Fr(float(b)))


def fadd(a, b):
    return round_f32(Fr(float(a)) + Fr(float(b)))


def ffma(a, b, c):
    return round_f32(Fr(float(a)) * Fr(float(b)) + Fr(float(c)))


def fsub(a, b):  # a - b as fma(b, -1, a)
    return ffma(b, f32(-1.0), a)


def dfma(a: float, b: float, c: float) -> float:
    return float(Fr(a) * Fr(b) + Fr(c))  # exact, then one correctly rounded conversion


# ---- the digit scheme --------------------------------------------------------------------------
DIGITS = {24: dict(F=48, RS=4), 28: dict(F=56, RS=8)}


def round51(c: float) -> float:
    b = dbits(c)
    return dfrom((b + 2) & ~3)


def tile_exp(values) -> int:
    return max((dbits(v) >> 52) & 0x7FF for v in values)


def split(x: float, tile_e: int, DB: int):
    F = DIGITS[DB]["F"]
    b = dbits(x)
    hi, lo = b >> 32, b & 0xFFFFFFFF
    e = (hi >> 20) & 0x7FF
    M = (((hi & 0xFFFFF) | 0x100000) << 32) | lo
    if F <= 53:
        sh, v = tile_e - e + 53 - F, M
    else:
        sh, v = tile_e - e, (M << (F - 53)) & (2 ** 64 - 1)
    A = v >> sh if sh < 64 else 0  # PTX shr.b64 clamps the amount to 64
    As = -A if hi >> 31 else A
    return As >> DB, As & ((1 << DB) - 1)  # arithmetic shift (floor) and the low digit


def consts(c: float, tile_e: int, DB: int):
    """Words of 2^RS scale and -1.5 2^(52+RS) scale (scale = c 2^(G-F)) by exponent-field
    arithmetic, as the kernels form them; None where the tile takes native FP64."""
    F, RS = DIGITS[DB]["F"], DIGITS[DB]["RS"]
    k1 = RS - F
    k2 = k1 + 52
    c15 = -1.5 * c
    G = tile_e - 1022
    cb, db = dbits(c), dbits(c15)
    ec, ed = (cb >> 52) & 0x7FF, (db >> 52) & 0x7FF
    if not (1023 - 900 <= tile_e <= 1023 + 900) or ec in (0, 0x7FF):
        return None
    if ec + G + k1 < 1 or ed + G + k2 > 2046:
        return None
    return dfrom(cb + ((G + k1) << 52)), dfrom(db + ((G + k2) << 52))


def combine(S0: int, S1: int, sc: float, cs: float, DB: int, qa: int = 0, qb: int = 0) -> float:
    RS = DIGITS[DB]["RS"]
    assert -2 ** 31 <= S0 < 2 ** 31 and -2 ** 31 <= S1 + 2 ** RS < 2 ** 31
    r = (S1 + ((1 << (RS - 1)) - 1) + ((S1 >> RS) & 1)) >> RS
    V = (S0 + qa) * 2 ** (DB - RS) + (r + qb) + 2 ** 51
    assert 0 <= V < 2 ** 52
    D = dfrom(0x4330000000000000 + V)
    assert Fr(D) == 2 ** 52 + V
    return dfma(D, sc, cs)


def digit_sum(n, x, c, DB):
    te = tile_exp(x)
    w = consts(c, te, DB)
    assert w is not None
    d = [split(v, te, DB) for v in x]
    S0 = sum(int(k) * a for k, (a, _) in zip(n, d))
    S1 = sum(int(k) * b for k, (_, b) in zip(n, d))
    return S0, S1, w, te, d


# ---- tests ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("DB", [24, 28])
def test_split_is_the_truncated_value_on_the_tile_grid(DB):
    F = DIGITS[DB]["F"]
    rng = np.random.default_rng(5 + DB)
    for _ in range(400):
        mag = 2.0 ** int(rng.integers(-60, 60))
        x = list(rng.uniform(-1, 1, 9) * mag * 2.0 ** rng.integers(-70, 1, size=9))
        x[int(rng.integers(0, 9))] = 0.0
        x.append(-0.0)
        te = tile_exp(x)
        G = te - 1022
        for v in x:
            d0, d1 = split(v, te, DB)
            assert 0 <= d1 < 2 ** DB and -2 ** DB <= d0 < 2 ** DB
            A = int(abs(Fr(v)) / Fr(2) ** (G - F))  # floor of the magnitude on the grid
            assert d0 * 2 ** DB + d1 == (-A if v < 0 else A)


@pytest.mark.parametrize("DB", [24, 28])
def test_sum_rounding_is_ties_to_even(DB):
    RS = DIGITS[DB]["RS"]
    for S1 in list(range(-5 * 2 ** RS, 5 * 2 ** RS)) + [2 ** 30 - 3, -2 ** 30 + 3, 7 * (2 ** 28 - 1)]:
        r = (S1 + ((1 << (RS - 1)) - 1) + ((S1 >> RS) & 1)) >> RS
        q = Fr(S1, 2 ** RS)
        fl = math.floor(q)
        exp = fl + 1 if q - fl > Fr(1, 2) or (q - fl == Fr(1, 2) and fl % 2) else fl
        assert r == exp, S1


def test_weight_scale_rounded_to_51_bits_keeps_one_and_a_half_exact():
    rng = np.random.default_rng(2)
    for c in list(rng.uniform(-1e6, 1e6, 500)) + [1.0 / 3, 2.0 ** -40 / 7, -1e-300, 1e300]:
        r = round51(float(c))
        assert abs(Fr(r) - Fr(float(c))) <= abs(Fr(float(c))) * Fr(1, 2 ** 51)  # two units in the last place
        assert Fr(-1.5 * r) == -Fr(3, 2) * Fr(r)


STENCILS = {  # integer ratios n_k of the library's digit stencils (the c factor is separate)
    "lap9": [1, 4, 1, 4, -20, 4, 1, 4, 1],
    "biharm13": [1, 2, -8, 2, 1, -8, 20, -8, 1, 2, -8, 2, 1],
    "ddx4": [1, -8, 8, -1],
    "lap5": [1, 1, -4, 1, 1],
}


@pytest.mark.parametrize("DB", [24, 28])
@pytest.mark.parametrize("name", sorted(STENCILS))
def test_digit_sum_within_the_stated_bound(DB, name):
    n = STENCILS[name]
    sn = sum(abs(k) for k in n)
    if DB == 28 and (sn > 8 or sum(k for k in n if k > 0) > 7):
        pytest.skip("28-bit digits serve sum|n| <= 8 with positive weights summing to at most 7")
    F, RS = DIGITS[DB]["F"], DIGITS[DB]["RS"]
    # truncation of the values, rounding of the sum, c rounded to 51 bits plus the FMA's rounding
    rel = Fr(1, 2 ** (F - 1)) + Fr(2 ** (RS - 1), 2 ** (F - 1)) / sn + Fr(1, 2 ** 50)
    rng = np.random.default_rng(sum(map(ord, name)) + DB)
    worst = Fr(0)
    for trial in range(300):
        c = float(rng.uniform(0.1, 10) * 2.0 ** rng.integers(-30, 30) * (1 if trial % 2 else -1))
        mag = 2.0 ** int(rng.integers(-40, 40))
        x = rng.uniform(-1, 1, len(n)) * mag
        if trial % 3 == 0:
            x = x * 2.0 ** rng.integers(-60, 1, size=len(n))
        if trial % 5 == 0:  # low digits all ones / extreme digit patterns
            x[0] = (1 - 2.0 ** -52) * mag
            x[-1] = -(1 - 2.0 ** -52) * mag
        x = [float(v) for v in x]
        S0, S1, (sc, cs), te, _ = digit_sum(n, x, round51(c), DB)
        got = combine(S0, S1, sc, cs, DB)
        exact = sum(Fr(k) * Fr(c) * Fr(v) for k, v in zip(n, x))
        scale = abs(Fr(c)) * sn * max(abs(Fr(v)) for v in x)
        err = abs(Fr(got) - exact) / scale
        worst = max(worst, err)
        assert err <= rel, (name, trial, float(err), float(rel))
    print(f"[digits] {name} DB={DB}: worst {float(worst):.3e} of sum|w| max|x| (bound {float(rel):.3e})")


# ---- the cubic user function's integer term --------------------------------------------------
M1, M2 = f32(1.5 * 2 ** 44), f32(1.5 * 2 ** 23)


def cubic_ok(tile_e: int, c: float) -> bool:
    if tile_e == 0:
        return True
    G = tile_e - 1022
    ec = ((dbits(c) >> 52) & 0x7FF) - 1023
    return 1023 - 69 <= tile_e < 1023 + 60 and 2 * G <= ec - 2


def q_of(d0: int, d1: int, tile_e: int, c: float):
    """Q = qa 2^20 + qb for one lane, in the kernel's order of FP32 operations."""
    G = tile_e - 1022
    inv = 1.0 / c
    inv_hi = f32(inv)
    inv_lo = f32(inv - float(inv_hi))
    p1 = ffrom((G - 24 + 127) << 23)
    p2 = ffrom((G - 48 + 127) << 23)
    ih = ffrom(fbits(inv_hi) + ((44 - G) << 23))
    il = f32(0.0) if inv_lo == 0 else ffrom(fbits(inv_lo) + ((44 - G) << 23))
    D0, D1 = f32(d0), f32(d1)
    assert int(D0) == d0 and int(D1) == d1
    uh, nuh = fmul(D0, p1), fmul(D0, -p1)
    ul, nul = fmul(D1, p2), fmul(D1, -p2)
    m2 = fmul(nuh, uh)
    e2 = ffma(uh, uh, m2)
    e2 = ffma(fmul(D0, f32(2.0) * p1), ul, e2)
    m3 = fmul(m2, uh)
    e3 = ffma(m2, nuh, m3)
    e3 = ffma(m2, nul, e3)
    e3 = ffma(e2, uh, e3)
    s = fadd(m3, uh)
    bb = fsub(s, m3)
    err = fadd(fsub(m3, fsub(s, bb)), fsub(uh, bb))
    lo = fadd(fsub(err, e3), ul)
    nph = fmul(s, -ih)
    pl = ffma(s, ih, nph)
    pl = ffma(lo, ih, pl)
    pl = ffma(s, il, pl)
    qh = fsub(pl, nph)
    ql = fsub(pl, fadd(qh, nph))
    t = fadd(qh, M1)
    rest = fadd(fsub(qh, fsub(t, M1)), ql)
    assert abs(float(rest)) < 2 ** 22
    t2 = fadd(rest, M2)
    return 2 * (fbits(M1) - fbits(t)), fbits(M2) - fbits(t2)


def test_cubic_term_within_one_unit():
    rng = np.random.default_rng(11)
    worst, cases = Fr(0), 0
    while cases < 400:
        c = round51(float(rng.uniform(1, 2) * 2.0 ** rng.integers(2, 41) * (1 if cases % 2 else -1)))
        ec = math.floor(math.log2(abs(c)))
        G = int(rng.integers(-67, (ec - 2) // 2 + 1))
        te = G + 1022
        if not cubic_ok(te, c):
            continue
        mag = 2.0 ** G
        mode = cases % 4
        if mode == 0:
            u = rng.uniform(-1, 1) * mag
        elif mode == 1:
            u = rng.uniform(-1, 1) * mag * 2.0 ** -int(rng.integers(0, 40))
        elif mode == 2:
            u = (1 - 2.0 ** -int(rng.integers(1, 50))) * mag * (1 if rng.random() < 0.5 else -1)
        else:  # the extremum of u^3 - u
            u = math.sqrt(1 / 3) * mag * (1 + rng.uniform(-1e-3, 1e-3)) * (1 if rng.random() < 0.5 else -1)
        u = float(u)
        if abs(u) >= mag or u == 0.0:
            continue
        d0, d1 = split(u, te, 24)
        qa, qb = q_of(d0, d1, te, c)
        U = Fr(c) * Fr(2) ** (G - 44)
        err = abs(Fr(qa * 2 ** 20 + qb) - (Fr(u) ** 3 - Fr(u)) / U)
        worst = max(worst, err)
        assert err < 1, (u, c, float(err))
        cases += 1
    print(f"[digits] cubic term: worst |Q - (u^3 - u)/U| = {float(worst):.3f} units")


def test_cubic_minus_laplacian_within_bound():
    """u^3 - u + sum w_k u_k with w = c (0, -1, 0, -1, 4, -1, 0, -1, 0) (the library's
    c^3 - c - Lap c, c = 1/h^2): the digit sum, Q joined as (qa, qb), one FMA."""
    n = [-1, -1, 4, -1, -1]  # north, west, centre, east, south
    rng = np.random.default_rng(3)
    bound = Fr(1, 2 ** 47) + Fr(1, 2 ** 44) / 8 + Fr(1, 2 ** 50) + Fr(1, 2 ** 46)
    worst, cases = Fr(0), 0
    while cases < 200:
        h = 2 * math.pi / float(2 ** int(rng.integers(6, 14)))
        c_user = 1.0 / (h * h)
        c = round51(c_user)
        mag = float(rng.uniform(0.05, 1.0))
        x = [float(v) for v in rng.uniform(-1, 1, 5) * mag]
        te = tile_exp(x)
        if not cubic_ok(te, c):
            continue
        S0, S1, (sc, cs), _, d = digit_sum(n, x, c, 24)
        qa, qb = q_of(d[2][0], d[2][1], te, c)
        got = combine(S0, S1, sc, cs, 24, qa, qb)
        u = Fr(x[2])
        exact = u ** 3 - u + sum(Fr(k) * Fr(c_user) * Fr(v) for k, v in zip(n, x))
        scale = abs(Fr(c)) * 8 * max(abs(Fr(v)) for v in x)
        err = abs(Fr(got) - exact) / scale
        worst = max(worst, err)
        assert err <= bound, (float(err), float(bound))
        cases += 1
    print(f"[digits] c^3 - c - Lap c: worst {float(worst):.3e} of sum|w| max|x| (bound {float(bound):.3e})")
