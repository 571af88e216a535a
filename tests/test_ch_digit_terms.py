"""The Cahn-Hilliard right-hand side's Z = alpha (u^3 - u) - a Lap(Cbar) with the cubic term joined
to the Laplacian's digit sum (Sec. 5.1, the factored RHS), emulated bit by bit on the CPU: the split
of a double u into the float pair h + l by integer operations, the packed double-float steps that
give the integer Q = round(alpha (u^3 - u) / (c 2^(G-48))), and the one-FMA combination of the
28-bit digit sum with Q.  Each step is written from its definition (IEEE round-to-nearest-even,
one rounding per FMA, integer shifts) and checked against exact rational arithmetic:

* h + l is u truncated to 48 significant bits (|u - h - l| < 2^-47 |u|), zero for zero;
* Q is within 0.6 of a unit U = |c| 2^(G-48) of the exact quotient (0.5 for the rounding, the rest
  the double-float error) wherever the kernel takes the digit form (alpha / |c| <= 2^-6, u in the
  exponent window, |qh| < 2^43);
* Z is within 2.2 U + 2^-52 |Z| of alpha (u^3 - u) - a Lap(Cbar) with the unrounded a: the digits'
  truncation (U / 32), the sum's rounding (U / 2), Q (0.6 U), a rounded to 51 bits (U) and the
  FMA's own rounding; the FP64 formula's own bound differs only by Q's 0.6 U.

And the invariants' per-thread sums (Eq. 1's mass and free energy, the gradient part summed by
parts) in exact integer arithmetic on the 28-bit digit grid of C's tile, from 32 x 32 -> 64-bit
products of the digits only: sum d0, sum d1; sum U L as three digit-product sums; u^2 - 1 as
W = round((U^2 - 2^(112-2G)) / 2^61) formed from d0^2 and 2 d0 d1 + floor(d1^2 / 2^28); W^2 from W's
two 29-bit digits.  Each sum of a thread's 8 points stays below 2^63, the joined sums within 2^-50
of the exact sums of the digit values (the truncation of values below an eighth of the tile's
largest is the digits' own), W within 2^-33 of a unit of its rounding, for every G in [-3, 3]."""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from test_digit_arithmetic import (dbits, fbits, ffrom, f32, fmul, fadd, ffma, fsub, round51, split,
                                   consts, combine, tile_exp)

M1, M2 = f32(1.5 * 2 ** 44), f32(1.5 * 2 ** 23)


def ch_params(n: int, gamma: float = 0.01, D: float = 1.0):
    """alpha and a of the scheme on [0, 2 pi)^2 with dt = 0.1 h (the paper's setup)."""
    h = 2 * math.pi / n
    dt = 0.1 * h
    return (2.0 / 3.0) * D * dt / (h * h), (2.0 / 3.0) * D * gamma * dt / h ** 4


def cubic_inv(alpha: float, c: float):
    r = alpha / c
    if not abs(r) <= 2.0 ** -6 or r == 0.0:
        return None
    hi = f32(r)
    return hi, f32(r - float(hi))


def split_hl(u: float):
    b = dbits(u)
    hw, lw = b >> 32, b & 0xFFFFFFFF
    top = ((((hw ^ 0x08000000) << 3) | (lw >> 29)) & 0xFFFFFFFF)
    hb = (top & 0x7FFFFFFF) | (hw & 0x80000000)
    x = f32((lw >> 5) & 0xFFFFFF)
    sc = ffrom(((hb & 0xFF800000) - (47 << 23)) & 0xFFFFFFFF)
    if hw & 0x7FF00000 == 0:
        return f32(0.0), f32(0.0)
    return ffrom(hb), fmul(x, sc)


def scaled_inv(inv, tile_e: int):
    hi, lo = inv
    sh = 1070 - tile_e
    eh = ((fbits(hi) >> 23) & 0xFF) + sh
    if eh < 25 or eh > 254:
        return None
    ih = ffrom(fbits(hi) + (sh << 23))
    el = ((fbits(lo) >> 23) & 0xFF) + sh
    il = f32(0.0) if lo == 0 or el < 1 else ffrom(fbits(lo) + (sh << 23))
    return ih, il


def cubic_q(h, l, ih, il):
    """One lane of the packed steps, in the kernel's order."""
    nh, nl = fmul(h, f32(-1.0)), fmul(l, f32(-1.0))
    nA = fmul(nh, h)
    a2 = ffma(fadd(h, h), l, ffma(h, h, nA))
    ns3 = fmul(nA, h)
    b = ffma(nA, nh, ns3)
    b = ffma(nA, nl, b)
    b = ffma(a2, h, b)
    S = fadd(ns3, h)
    bb = fsub(S, ns3)
    t = fadd(fsub(ns3, fsub(S, bb)), fsub(h, bb))
    lo = fadd(fsub(t, b), l)
    np_ = fmul(S, -ih)
    pl = ffma(S, ih, np_)
    pl = ffma(lo, ih, pl)
    pl = ffma(S, il, pl)
    qh = fsub(pl, np_)
    ql = fsub(pl, fadd(qh, np_))
    t1 = fadd(qh, M1)
    rest = fadd(fsub(qh, fsub(t1, M1)), ql)
    t2 = fadd(rest, M2)
    return 2 * (fbits(M1) - fbits(t1)), fbits(M2) - fbits(t2), qh


def cubic_ok(u: float, tile_e: int, qh, s0: int) -> bool:
    e = (dbits(u) >> 52) & 0x7FF
    return (e == 0 or 944 <= e <= tile_e + 1) and abs(float(qh)) < 2.0 ** 43 and abs(s0) <= 2 ** 31 - 1 - (2 ** 24 - 1)


def test_split_is_u_truncated_to_48_bits():
    rng = np.random.default_rng(5)
    for k in range(2000):
        e = int(rng.integers(944 - 1023, 1150 - 1023))
        u = float(rng.uniform(1, 2) * 2.0 ** e * (1 if k % 2 else -1))
        h, l = split_hl(u)
        b = dbits(u)
        trunc = dfrom_trunc(b)
        assert Fr(float(h)) + Fr(float(l)) == trunc, (u, h, l)
        assert abs(Fr(u) - trunc) < Fr(2) ** -47 * abs(Fr(u))
        assert abs(Fr(float(h))) <= abs(Fr(u)) and (float(h) == 0 or np.sign(float(h)) == np.sign(u))
    for z in (0.0, -0.0, 5e-324):
        assert split_hl(z) == (0.0, 0.0)


def dfrom_trunc(b: int) -> Fr:
    """The double with bits b, its lowest 5 significand bits cleared (48 significant bits)."""
    import struct
    return Fr(struct.unpack("<d", struct.pack("<Q", b & ~0x1F))[0])


@pytest.mark.parametrize("n", [512, 1024, 4096, 8192])
def test_cubic_q_within_0p6_unit(n):
    alpha, a = ch_params(n)
    c = round51(-a)
    inv = cubic_inv(alpha, c)
    assert inv is not None
    rng = np.random.default_rng(n)
    worst, cases = Fr(0), 0
    while cases < 300:
        mag = float(rng.uniform(0.02, 1.6))  # the tile's largest |Cbar|
        te = tile_exp([mag])
        G = te - 1022
        k = scaled_inv(inv, te)
        assert k is not None
        ih, il = k
        mode = cases % 4
        if mode == 0:
            u = rng.uniform(-1.2, 1.2) * min(mag, 1.0)
        elif mode == 1:  # near the wells and the extremum of u^3 - u, where the terms cancel
            u = (1.0, math.sqrt(1 / 3))[int(rng.integers(0, 2))] * (1 + rng.uniform(-1e-6, 1e-6)) * (1 if rng.random() < 0.5 else -1)
        elif mode == 2:  # small values
            u = rng.uniform(-1, 1) * 2.0 ** -int(rng.integers(5, 70))
        else:
            u = 0.0
        u = float(u)
        h, l = split_hl(u)
        qa, qb, qh = cubic_q(h, l, ih, il)
        if not cubic_ok(u, te, qh, 0):
            continue
        U = Fr(c) * Fr(2) ** (G - 48)
        exact = Fr(alpha) * (Fr(u) ** 3 - Fr(u)) / U
        err = abs(Fr(qa * 2 ** 20 + qb) - exact)
        worst = max(worst, err)
        assert err <= Fr(6, 10), (n, u, float(err))
        cases += 1
    print(f"[ch cubic] n={n}: worst |Q - alpha N / U| = {float(worst):.4f} units")


def test_inverse_is_zero_above_2_pow_minus_6():
    # alpha / a = h^2 / gamma: the digit form serves n >= 512 at gamma = 0.01, and not n = 256
    for n, ok in ((256, False), (512, True), (4096, True)):
        alpha, a = ch_params(n)
        assert (cubic_inv(alpha, round51(-a)) is not None) == ok


@pytest.mark.parametrize("n", [512, 1024, 4096])
def test_z_within_bound(n):
    """Z at the centre of a 5-point Laplacian of random Cbar values: digits of Cbar on its tile's
    grid, the 28-bit digit sum, Q joined as (qa, qb), one FMA; against exact arithmetic."""
    alpha, a = ch_params(n)
    c = round51(-a)
    inv = cubic_inv(alpha, c)
    w = [1, 1, -4, 1, 1]
    rng = np.random.default_rng(7 + n)
    worst, cases = 0.0, 0
    while cases < 150:
        mag = float(rng.uniform(0.05, 1.2))
        cb = [float(v) for v in rng.uniform(-1, 1, 5) * mag]
        if cases % 3 == 0:  # a smooth patch: the Laplacian is small against its terms
            base, slope = float(rng.uniform(-1, 1) * mag), float(rng.uniform(-1e-3, 1e-3))
            cb = [base + slope * d for d in (-1.0, 0.0, 0.0, 0.0, 1.0)]
            cb[2] = base + float(rng.uniform(-1e-6, 1e-6))
        u = float(cb[2] * (1 + rng.uniform(-0.1, 0.1)))  # C^n, close to Cbar
        te = tile_exp(cb)
        G = te - 1022
        sc, cs = consts(c, te, 28)
        d = [split(v, te, 28) for v in cb]
        S0 = sum(k * x for k, (x, _) in zip(w, d))
        S1 = sum(k * y for k, (_, y) in zip(w, d))
        ih, il = scaled_inv(inv, te)
        h, l = split_hl(u)
        qa, qb, qh = cubic_q(h, l, ih, il)
        if not cubic_ok(u, te, qh, S0):
            continue
        z = combine(S0, S1, sc, cs, 28, qa, qb)
        lap = sum(k * Fr(v) for k, v in zip(w, cb))
        exact = Fr(alpha) * (Fr(u) ** 3 - Fr(u)) - Fr(a) * lap
        U = abs(Fr(c)) * Fr(2) ** (G - 48)
        err = abs(Fr(z) - exact)
        bound = Fr(22, 10) * U + Fr(2) ** -52 * abs(Fr(z))
        worst = max(worst, float(err / U))
        assert err <= bound, (n, float(err / U))
        cases += 1
    print(f"[ch cubic] n={n}: worst |Z - exact| = {worst:.3f} units")


def i128_to_double(v: int) -> float:
    """The kernel's conversion: the magnitude's two 64-bit halves, each rounded to a double, joined
    by one FMA (exact product 2^64 hi, then one rounding)."""
    a = abs(v)
    hi, lo = a >> 64, a & (2 ** 64 - 1)
    r = float(Fr(float(hi)) * 2 ** 64 + Fr(float(lo)))
    return -r if v < 0 else r


@pytest.mark.parametrize("G", [-3, -1, 0, 1, 3])
def test_invariant_sums_in_integers(G):
    """Eight points of a thread: u and its four neighbours, on a tile whose largest value lies in
    [2^(G-1), 2^G); the kernel's integer sums against exact rational sums of the digit values."""
    rng = np.random.default_rng(100 + G)
    te = G + 1022
    I63 = 2 ** 63
    for trial in range(60):
        mag = float(rng.uniform(0.5, 1.0)) * 2.0 ** G
        vals = rng.uniform(-1, 1, (8, 5)) * mag
        if trial % 4 == 0:  # the wells: u near +-1 where u^2 - 1 cancels (where the tile allows)
            vals = np.sign(vals) * np.minimum(1.0 + rng.uniform(-1e-7, 1e-7, vals.shape), 0.999 * 2.0 ** G)
        if trial % 4 == 1:  # the extremes of the digit ranges: values at the tile's top
            vals = np.sign(vals) * (2.0 ** G) * (1 - 2.0 ** -50)
        vals = [[float(v) for v in row] for row in vals]
        K56 = 1 << (56 - 2 * G)
        s0 = s1 = g2 = g1 = g0 = w2 = w1 = w0 = 0
        ex_m = ex_g = ex_w = Fr(0)
        worst_w = Fr(0)
        for row in vals:  # centre, north, south, west, east
            d = [split(v, te, 28) for v in row]
            d0, d1 = d[0]
            q0 = d[1][0] + d[2][0] + d[3][0] + d[4][0] - 4 * d0
            q1 = d[1][1] + d[2][1] + d[3][1] + d[4][1] - 4 * d1
            assert -2 ** 31 <= q0 < 2 ** 31 and -2 ** 31 <= q1 < 2 ** 31
            s0 += d0
            s1 += d1
            g2 += d0 * q0
            g1 += d0 * q1 + d1 * q0
            g0 += d1 * q1
            A = d0 * d0 - K56
            B = d0 * (2 * d1) + ((d1 * d1) >> 28)
            assert abs(A) < I63 and abs(B) < I63
            W = (A >> 5) + ((((A & 31) << 28) + B + (1 << 32)) >> 33)
            U = d0 * 2 ** 28 + d1
            exact_W = Fr(U * U - (1 << (112 - 2 * G)), 2 ** 61)
            worst_w = max(worst_w, abs(W - exact_W))
            assert abs(W) <= 2 ** 57 + 1
            wh, wl = W >> 29, W & (2 ** 29 - 1)
            assert -2 ** 31 <= wh < 2 ** 31
            w2 += wh * wh
            w1 += wh * wl
            w0 += wl * wl
            for acc in (g2, g1, g0, w2, w1, w0):
                assert abs(acc) < I63
            sc = Fr(2) ** (G - 56)
            u = [Fr(x * 2 ** 28 + y) * sc for x, y in d]
            ex_m += u[0]
            ex_g += u[0] * (u[1] + u[2] + u[3] + u[4] - 4 * u[0])
            ex_w += (u[0] ** 2 - 1) ** 2
        assert abs(s0) < 2 ** 31 and s1 < 2 ** 31
        assert worst_w <= Fr(1, 2) + Fr(1, 2 ** 33)  # round half up, d1^2's dropped bits
        sg = (g2 << 56) + (g1 << 28) + g0
        sw = (w2 << 58) + (w1 << 30) + w0
        m = float(Fr(float(Fr(s0) * 2 ** 28 + s1)) * Fr(2) ** (G - 56))
        eg = float(Fr(i128_to_double(sg)) * Fr(2) ** (2 * G - 112))
        ew = float(Fr(i128_to_double(sw)) * Fr(2) ** (4 * G - 102))
        assert abs(Fr(m) - ex_m) <= Fr(2) ** -53 * abs(ex_m) + Fr(2) ** -300
        assert abs(Fr(eg) - ex_g) <= Fr(2) ** -51 * abs(ex_g) + Fr(2) ** -300
        # W within (1/2 + 2^-33) of its unit 2^(2G-51): |delta W^2| <= (2 |w| + unit) unit per point
        unit = Fr(2) ** (2 * G - 51)
        tol = sum(2 * abs(Fr(r[0]) ** 2 - 1) + unit for r in vals) * unit
        assert abs(Fr(ew) - ex_w) <= tol + Fr(2) ** -51 * ex_w, (G, trial)


def test_block_totals_fit_in_128_bits():
    """The block (256 threads of 8 points) reduces the thread sums in integers: the per-thread
    bounds (|sum d0|, sum d1 < 2^31; |sum U L| < 2^118; sum W^2 <= 8 (2^57 + 1)^2) times 256 stay below the
    64-bit (mass digits) and 128-bit (energy) limits."""
    threads, pts = 256, 8
    assert threads * pts * 2 ** 28 < 2 ** 63  # sum d0, sum d1 over the block
    assert threads * pts * 2 ** 56 * 2 ** 59 < 2 ** 127  # sum U L: |U| < 2^56, |L| < 8 2^56
    assert threads * pts * (2 ** 57 + 1) ** 2 < 2 ** 127  # sum W^2: |U^2 - K| <= 2^118, |W| <= 2^57 + 1
