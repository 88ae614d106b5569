"""Generates bulge_fit.h: float32 fits of the projected profiles of the Hernquist (gamma = 1)
and Jaffe (gamma = 2) bulges, for the closed-form bulge option (bulge_kind 1 and 2).

With s = R / a the projected density and the projected pressure of a Dehnen bulge with
fixed gamma are universal functions of s:
  Sigma(R)           = M / a^2       * F_S(s)
  Sigma sigma_p^2(R) = G M^2 / a^3   * F_Q(s)
Hernquist: Sigma is Eq. 4 of the paper (with X(s) of Eq. 5) and sigma_p^2 is Eq. 6; Jaffe:
Eqs. B4 and B5.  Both closed forms cancel badly (near s = 1, and in sigma_p^2 at large s,
where the brace of Eq. 6 loses ~s^5 in relative size), so they are evaluated here with
mpmath at 80 digits, and checked against the defining projection integrals
  Sigma = 2 int_R^inf rho r dr / sqrt(r^2 - R^2),
  Sigma sigma_p^2 = 2 G int_R^inf rho M sqrt(r^2 - R^2) / r^2 dr
done by mpmath quadrature.

Representation: t = log2 s in [T0, T0 + N) is cut into N unit pieces; on piece k,
  log2 F(t) = E_k + p_k(u),  u = t - (T0 + k) in [0, 1),
with E_k an integer (so 2^E_k is exact in float32) and p_k a degree-DEG polynomial fitted
by least squares on Chebyshev points.  Outside [T0, T0 + N) the edge values hold (u clamped).
The slope d log2 F / d t = p_k'(u) (= R dln F / dR) serves the adjoint.  The script emulates
the float32 evaluation (Horner, one rounding per operation) and prints the worst relative
errors.  Run:  python gen_bulge_fit.py > bulge_fit.h
"""
import sys

import mpmath
import numpy as np

mpmath.mp.dps = 80

T0, N, DEG = -48, 80, 7
NODES = 28


def X_of(s):
    s = mpmath.mpf(s)
    if s < 1:
        return mpmath.acosh(1 / s) / mpmath.sqrt(1 - s * s)
    if s > 1:
        return mpmath.acos(1 / s) / mpmath.sqrt(s * s - 1)
    return mpmath.mpf(1)


def hernquist(s):
    """(F_S, F_Q) of the Hernquist bulge (Eqs. 4-6)."""
    s = mpmath.mpf(s)
    X = X_of(s)
    q = 1 - s * s
    FS = ((2 + s * s) * X - 3) / (2 * mpmath.pi * q * q)
    brace = ((-3 * s * s * X * (8 * s**6 - 28 * s**4 + 35 * s * s - 20) - 24 * s**6 + 68 * s**4 - 65 * s * s + 6)
             / (2 * q**3) - 6 * mpmath.pi * s)
    return FS, brace / (12 * mpmath.pi)


def jaffe(s):
    """(F_S, F_Q) of the Jaffe bulge (Eqs. B4-B5)."""
    s = mpmath.mpf(s)
    X = X_of(s)
    q = 1 - s * s
    FS = 1 / (4 * s) + (1 - (2 - s * s) * X) / (2 * mpmath.pi * q)
    br = (mpmath.pi / (2 * s) + 11 - mpmath.mpf(13) / 2 * mpmath.pi * s - 12 * s * s + 6 * mpmath.pi * s**3
          - X * (6 - 19 * s * s + 12 * s**4))
    return FS, br / (4 * mpmath.pi * q)


def by_integrals(s, gamma):
    """(F_S, F_Q) from the projection integrals of the Dehnen profile (a = M = G = 1)."""
    s = mpmath.mpf(s)
    g = mpmath.mpf(gamma)

    def rho(r):
        return (3 - g) / (4 * mpmath.pi) / (r**g * (1 + r) ** (4 - g))

    def mass(r):
        return (r / (1 + r)) ** (3 - g)

    # r = s cosh t: dr / sqrt(r^2 - s^2) = dt, sqrt(r^2 - s^2) = s sinh t
    FS = 2 * mpmath.quad(lambda t: rho(s * mpmath.cosh(t)) * s * mpmath.cosh(t), [0, 1, 5, 20, 60])
    FQ = 2 * mpmath.quad(lambda t: rho(s * mpmath.cosh(t)) * mass(s * mpmath.cosh(t)) * (s * mpmath.sinh(t)) ** 2
                         / (s * mpmath.cosh(t)) ** 2, [0, 1, 5, 20, 60])
    return FS, FQ


def fit(kind_fn):
    E = np.zeros((2, N), dtype=np.int64)
    C = np.zeros((2, N, DEG + 1))
    for k in range(N):
        x = 0.5 + 0.5 * np.cos(np.pi * (np.arange(NODES) + 0.5) / NODES)     # u in (0, 1)
        vals = [kind_fn(mpmath.mpf(2) ** (T0 + k + mpmath.mpf(float(u)))) for u in x]
        for f in range(2):
            l2 = np.array([float(mpmath.log(v[f], 2)) for v in vals])
            mid = float(mpmath.log(kind_fn(mpmath.mpf(2) ** (T0 + k + mpmath.mpf(0.5)))[f], 2))
            E[f, k] = int(round(mid))
            C[f, k] = np.polynomial.polynomial.polyfit(x, l2 - E[f, k], DEG)
    return E, C


def check(kind_fn, E, C):
    """Worst relative error of F and of the slope in float32 emulation (dense samples)."""
    Cf = C.astype(np.float32)
    worst = [0.0, 0.0, 0.0, 0.0]
    for k in range(N):
        for u in np.linspace(0.003, 0.997, 9):
            t = T0 + k + u
            ref = kind_fn(mpmath.mpf(2) ** mpmath.mpf(t))
            u32 = np.float32(u)
            for f in range(2):
                p = Cf[f, k, DEG]
                dp = np.float32(0.0)
                for i in range(DEG - 1, -1, -1):
                    dp = np.float32(dp * u32 + p)
                    p = np.float32(p * u32 + Cf[f, k, i])
                val = 2.0 ** float(p) * 2.0 ** int(E[f, k])
                worst[f] = max(worst[f], abs(val / float(ref[f]) - 1.0))
                h = mpmath.mpf("1e-20")
                rp = kind_fn(mpmath.mpf(2) ** (mpmath.mpf(t) + h))[f]
                slope_ref = float((mpmath.log(rp, 2) - mpmath.log(ref[f], 2)) / h)
                worst[2 + f] = max(worst[2 + f], abs(float(dp) - slope_ref) / max(1.0, abs(slope_ref)))
    return worst


def main():
    # the closed forms against the projection integrals
    dev = 0.0
    for fn, g in ((hernquist, 1), (jaffe, 2)):
        for s in ("1e-6", "0.01", "0.3", "0.999", "1.001", "2.5", "40", "3000"):
            a, b = fn(s), by_integrals(s, g)
            dev = max(dev, float(abs(a[0] / b[0] - 1)), float(abs(a[1] / b[1] - 1)))
    tables = {}
    errs = {}
    for name, fn in (("Hernquist", hernquist), ("Jaffe", jaffe)):
        E, C = fit(fn)
        tables[name] = (E, C)
        errs[name] = check(fn, E, C)
    out = sys.stdout
    out.write("// Generated by gen_bulge_fit.py -- do not edit.\n")
    out.write("// Float32 fits of the projected profiles of the Hernquist (Eqs. 4-6) and Jaffe (Eqs. B4-B5)\n")
    out.write("// bulges: Sigma = M a^-2 F_S(s), Sigma sigma_p^2 = G M^2 a^-3 F_Q(s), s = R / a;\n")
    out.write("// log2 F = E_k + p_k(u) on unit pieces of t = log2 s, u = t - (T0 + k).\n")
    out.write(f"// Closed forms vs projection integrals (mpmath): worst relative deviation {dev:.1e}.\n")
    for name in tables:
        w = errs[name]
        out.write(f"// {name}: worst relative error in float32 emulation F_S {w[0]:.2e}, F_Q {w[1]:.2e}; "
                  f"slopes {w[2]:.2e}, {w[3]:.2e} (t in [{T0}, {T0 + N}]).\n")
    out.write("#pragma once\n\n")
    out.write(f"#define BANG_BULGE_FIT_T0 {T0}\n#define BANG_BULGE_FIT_N {N}\n#define BANG_BULGE_FIT_DEG {DEG}\n\n")
    out.write("// [kind: 0 Hernquist, 1 Jaffe][function: 0 F_S, 1 F_Q][piece]: 2^E_k\n")
    out.write("static __constant__ float kBulgeFitScale[2][2][BANG_BULGE_FIT_N] = {\n")
    for name in tables:
        E, _ = tables[name]
        out.write("  {\n")
        for f in range(2):
            out.write("    {" + ", ".join(f"{2.0 ** int(e):.9e}f" for e in E[f]) + "},\n")
        out.write("  },\n")
    out.write("};\n\n")
    out.write("// [kind][function][piece][i]: coefficient of u^i of p_k\n")
    out.write("static __constant__ float kBulgeFitC[2][2][BANG_BULGE_FIT_N][BANG_BULGE_FIT_DEG + 1] = {\n")
    for name in tables:
        _, C = tables[name]
        out.write("  {\n")
        for f in range(2):
            out.write("    {\n")
            for k in range(N):
                out.write("      {" + ", ".join(f"{float(np.float32(c)):.9e}f" for c in C[f, k]) + "},\n")
            out.write("    },\n")
        out.write("  },\n")
    out.write("};\n")


if __name__ == "__main__":
    main()
