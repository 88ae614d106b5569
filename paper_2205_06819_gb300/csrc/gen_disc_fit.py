"""Generates disc_fit.h: float32 polynomial fits of F(y) = y^2 [I0(y)K0(y) - I1(y)K1(y)].

F is the shape of the Freeman exponential-disc rotation curve, v^2 = (2 G M_d / R_d) F(y)
with y = r / (2 R_d) (Eq. 9 of the paper, Binney & Tremaine form).  CUDA has no K0/K1,
and for large y the difference I0K0 - I1K1 ~ 1/(4 y^3) cancels catastrophically if the
four Bessel functions are evaluated separately in float32.  F is therefore fitted directly:

  * y <= 1:  F = s (P(s) - ln(y) Q(s)), s = y^2, with Q = I0^2 + I1^2 (the coefficient of
    the logarithm in the small-argument expansion) and P = (I0K0 - I1K1) + ln(y) Q, both
    smooth in s; fitted by least squares on Chebyshev points of s in [0, 1].
  * y >= 1:  F = Gf(u) / (4 y), u = 1/y, where Gf = 4 y^3 (I0K0 - I1K1) -> 1 as y -> inf
    (DLMF 10.40.6).  u in (0, 1] is cut into [1/2, 1], [1/4, 1/2], [1/8, 1/4], [1/16, 1/8],
    [0, 1/16], each fitted in t = (u - mid) / half in [-1, 1].

Reference values come from mpmath at 40 digits.  The script then emulates the float32
evaluation (Horner, one rounding per operation) and reports the worst relative error of F
and F'.  Run:  python gen_disc_fit.py > disc_fit.h
"""
import sys

import mpmath
import numpy as np

mpmath.mp.dps = 40

DEG_A = 8
DEG_B = 11
B_EDGES = [1.0, 0.5, 0.25, 0.125, 0.0625, 0.0]


def bessel_diff(y):
    y = mpmath.mpf(y)
    return mpmath.besseli(0, y) * mpmath.besselk(0, y) - mpmath.besseli(1, y) * mpmath.besselk(1, y)


def q_of(y):
    y = mpmath.mpf(y)
    return mpmath.besseli(0, y) ** 2 + mpmath.besseli(1, y) ** 2


def cheb_points(a, b, n):
    t = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    return (a + b) / 2 + (b - a) / 2 * t


def fit_small():
    s = cheb_points(0.0, 1.0, 160)
    y = np.sqrt(s)
    P = np.array([float(bessel_diff(v) + mpmath.log(v) * q_of(v)) for v in y])
    Q = np.array([float(q_of(v)) for v in y])
    return (np.polynomial.polynomial.polyfit(s, P, DEG_A), np.polynomial.polynomial.polyfit(s, Q, DEG_A))


def fit_large():
    out = []
    for lo, hi in zip(B_EDGES[1:], B_EDGES[:-1]):
        mid, half = (lo + hi) / 2, (hi - lo) / 2
        t = np.cos(np.pi * (np.arange(120) + 0.5) / 120)
        u = np.maximum(mid + half * t, 1e-12)
        g = np.array([float(4 * mpmath.mpf(1 / v) ** 3 * bessel_diff(1 / v)) for v in u])
        out.append((mid, half, np.polynomial.polynomial.polyfit(t, g, DEG_B)))
    return out


def f32(x):
    return np.float32(x)


def horner2(c, x):
    """value and derivative by Horner, float32 rounding after each operation"""
    x = f32(x)
    p, d = f32(c[-1]), f32(0.0)
    for ck in c[-2::-1]:
        d = f32(f32(d * x) + p)
        p = f32(f32(p * x) + f32(ck))
    return p, d


def eval32(y, small, large):
    y = f32(y)
    if y <= 1.0:
        cP, cQ = small
        s = f32(y * y)
        P, dP = horner2(cP, s)
        Q, dQ = horner2(cQ, s)
        ly = f32(np.log(np.float32(y)))
        core = f32(P - f32(ly * Q))
        F = f32(s * core)
        # dF/dy = 2y [P + s P' - ln y (Q + s Q') - Q/2]
        dF = f32(f32(2.0) * y * f32(P + s * dP - ly * (Q + s * dQ) - f32(0.5) * Q))
        return float(F), float(dF)
    u = f32(f32(1.0) / y)
    k = min(int(np.floor(-np.log2(float(u)))), len(large) - 1) if u < 1.0 else 0
    mid, half, c = large[k]
    t = f32(f32(u - f32(mid)) * f32(1.0 / half))
    g, dg = horner2(c, t)
    F = f32(g * f32(f32(0.25) * u))
    # dF/dy = -(u^2/4) [ g + u dg/du ],  dg/du = dg/dt / half
    dF = f32(-f32(0.25) * u * u * f32(g + u * f32(dg * f32(1.0 / half))))
    return float(F), float(dF)


def check(small, large):
    worst_f = worst_d = 0.0
    for y in np.concatenate([np.geomspace(1e-4, 1.0, 300), np.geomspace(1.0, 2000.0, 600)]):
        y32 = float(np.float32(y))
        F, dF = eval32(y32, small, large)
        yy = mpmath.mpf(y32)
        ref = yy * yy * bessel_diff(yy)
        dref = mpmath.diff(lambda v: v * v * bessel_diff(v), yy)
        worst_f = max(worst_f, abs(F / float(ref) - 1))
        worst_d = max(worst_d, abs(dF - float(dref)) / abs(float(dref)) if dref != 0 else 0.0)
    return worst_f, worst_d


def main():
    small = fit_small()
    large = fit_large()
    wf, wd = check(small, large)
    w = sys.stdout.write
    w("// Generated by gen_disc_fit.py -- do not edit.\n")
    w("// Float32 fits of F(y) = y^2 [I0(y)K0(y) - I1(y)K1(y)] (Freeman disc, Eq. 9 reading).\n")
    w(f"// Worst relative error in float32 emulation: F {wf:.2e}, dF/dy {wd:.2e} (y in [1e-4, 2000]).\n")
    w("#pragma once\n\n")
    w(f"#define BANG_DISC_DEG_A {DEG_A}\n#define BANG_DISC_DEG_B {DEG_B}\n#define BANG_DISC_NPIECE_B {len(large)}\n\n")
    w("// y <= 1: F = s (P(s) - ln(y) Q(s)), s = y^2; coefficients of s^0 .. s^DEG_A\n")
    w("__constant__ float kDiscP[BANG_DISC_DEG_A + 1] = {" + ", ".join(f"{v:.9e}f" for v in small[0]) + "};\n")
    w("__constant__ float kDiscQ[BANG_DISC_DEG_A + 1] = {" + ", ".join(f"{v:.9e}f" for v in small[1]) + "};\n\n")
    w("// y >= 1: F = g(t) u / 4, u = 1/y, piece k covers u in [2^-(k+1), 2^-k] (last: [0, 1/16]),\n")
    w("// t = (u - mid_k) * invhalf_k; coefficients of t^0 .. t^DEG_B\n")
    w("__constant__ float kDiscMid[BANG_DISC_NPIECE_B] = {" + ", ".join(f"{m:.9e}f" for m, _, _ in large) + "};\n")
    w("__constant__ float kDiscInvHalf[BANG_DISC_NPIECE_B] = {" + ", ".join(f"{1.0 / h:.9e}f" for _, h, _ in large) + "};\n")
    w("__constant__ float kDiscG[BANG_DISC_NPIECE_B][BANG_DISC_DEG_B + 1] = {\n")
    for _, _, c in large:
        w("  {" + ", ".join(f"{v:.9e}f" for v in c) + "},\n")
    w("};\n")


if __name__ == "__main__":
    main()
