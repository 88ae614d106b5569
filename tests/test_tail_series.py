"""The upper-node series of the forward kernel's radial rule (bang_device.cuh, TailRule,
fill_tail_coeffs, bulge_projected_w), restated in float64 and checked against the plain
node-by-node sum it replaces.

For nodes k >= K of the rule r = R cosh t (t in [0, 16], n Gauss-Legendre nodes), a point's
q_k = 1 + w m_k (m_k = cosh t_k - 1) is expanded as (w m_k)^p (1 + 1/(w m_k))^p, so that
sum_{k>=K} W_k q_k^p = w^p sum_j binom(p, j) A_j w^-j with per-model A_j = sum W_k m_k^(p-j).
The kernels use two levels: the far level splits at KF (t ~ 3) with kFarTerms terms where
w m_KF >= kFarZ, the mid level at K (t ~ 5) with kTailTerms terms where w m_K >= kTailZ.
The header's constants are read from the source; the claim pinned here is the one its
comment makes: truncation below 1e-9 of the whole sum at both levels, for both projected
integrals (Sigma: p = g - 4, W = w_k cosh t_k cosh^-g t_k; Sigma sigma^2: p = 2g - 7,
W = w_k tanh^2 t_k cosh^(3-2g) t_k) over gamma in [0, 3) and every w each level serves,
with float32 coefficients and Horner as the kernels form them.
"""
import math
import os
import re

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "paper_2205_06819_gb300", "csrc", "bang_device.cuh")


def header_constants():
    """(K, terms, z) of the mid level, as the earlier single-level tests read them."""
    text = open(HEADER).read()
    K = {int(n): int(k) for n, k, _ in
         re.findall(r"struct TailRule<(\d+)> \{ static constexpr int K = (\d+), KF = (\d+);", text)}
    terms = int(re.search(r"constexpr int kTailTerms = (\d+);", text).group(1))
    z = float(re.search(r"constexpr float kTailZ = ([0-9.]+)f;", text).group(1))
    return K, terms, z


def levels():
    """[(name, n, K, terms, z)] of both series levels and both rules, read from the header."""
    text = open(HEADER).read()
    rules = re.findall(r"struct TailRule<(\d+)> \{ static constexpr int K = (\d+), KF = (\d+);", text)
    tm = int(re.search(r"constexpr int kTailTerms = (\d+);", text).group(1))
    zm = float(re.search(r"constexpr float kTailZ = ([0-9.]+)f;", text).group(1))
    tf = int(re.search(r"constexpr int kFarTerms = (\d+);", text).group(1))
    zf = float(re.search(r"constexpr float kFarZ = ([0-9.]+)f;", text).group(1))
    out = []
    for n, k, kf in rules:
        out.append(("mid", int(n), int(k), tm, zm))
        out.append(("far", int(n), int(kf), tf, zf))
    return out


def rule(n):
    x, wt = np.polynomial.legendre.leggauss(n)
    t = 8.0 * (x + 1.0)
    w = 8.0 * wt
    return t, w, np.cosh(t), 2.0 * np.sinh(0.5 * t) ** 2, np.tanh(t) ** 2


def series(W, m, p, K, terms, w):
    s, b = 0.0, 1.0
    for j in range(terms):
        if j:
            b *= (p - (j - 1)) / j
        s += b * np.sum(W[K:] * m[K:] ** (p - j)) * w ** (-j)
    return w ** p * s


LEVELS = levels()
LEVEL_IDS = [f"{name}{n}" for name, n, *_ in LEVELS]


@pytest.mark.parametrize("name,n,k,terms,z", LEVELS, ids=LEVEL_IDS)
def test_series_truncation_below_1e9_of_the_sum(name, n, k, terms, z):
    t, wk, c, m, th2 = rule(n)
    assert k % 2 == 0
    lo, hi, wcap = (4.5, 5.5, 0.25) if name == "mid" else (2.8, 3.4, 0.8)
    assert lo < t[k] < hi                              # the mid split near t = 5, the far one near 3
    wmin = z / m[k]
    assert wmin < wcap                                 # mid: all but the centre; far: R above ~2-3 a
    worst = 0.0
    for g in np.linspace(0.0, 2.999, 31):
        WS = wk * c * c ** -g
        WQ = wk * th2 * c ** (3 - 2 * g)
        for w in np.geomspace(wmin, 1.0 - 1e-6, 41):
            q = 1.0 + w * m
            fullS, fullQ = np.sum(WS * q ** (g - 4)), np.sum(WQ * q ** (2 * g - 7))
            headS, headQ = np.sum((WS * q ** (g - 4))[:k]), np.sum((WQ * q ** (2 * g - 7))[:k])
            eS = abs(headS + series(WS, m, g - 4, k, terms, w) - fullS) / fullS
            eQ = abs(headQ + series(WQ, m, 2 * g - 7, k, terms, w) - fullQ) / fullQ
            worst = max(worst, eS, eQ)
    assert worst < 1e-9, worst


def test_the_levels_nest():
    """Every point the mid level leaves to the far one is inside the far level's range:
    the far threshold in w lies above the mid one, and the far split below the mid split."""
    by = {(name, n): (k, z) for name, n, k, _, z in LEVELS}
    for n in (64, 128):
        (kf, zf), (km, zm) = by[("far", n)], by[("mid", n)]
        m = rule(n)[3]
        assert kf < km and zf / m[kf] > zm / m[km]


@pytest.mark.parametrize("name,n,k,terms,z", [lv for lv in LEVELS if lv[1] == 64], ids=["mid64", "far64"])
def test_a_shorter_series_or_a_looser_threshold_would_fail(name, n, k, terms, z):
    """The pin has teeth: a quarter of the terms, or the series used down to w m_K = z / 8,
    miss 1e-9 (at gamma = 2.5)."""
    t, wk, c, m, th2 = rule(n)
    g = 2.5
    WQ = wk * th2 * c ** (3 - 2 * g)

    def err(nterms, w):
        q = 1.0 + w * m
        full = np.sum(WQ * q ** (2 * g - 7))
        head = np.sum((WQ * q ** (2 * g - 7))[:k])
        return abs(head + series(WQ, m, 2 * g - 7, k, nterms, w) - full) / full

    assert err(terms // 4, z / m[k]) > 1e-9
    assert err(terms, z / 8 / m[k]) > 1e-9


def test_binomial_coefficients_by_the_product_formula():
    """binom(p, j) for real p as the kernel forms it: prod_{i<j} (p - i) / (i + 1)."""
    for p in (-4.0, -2.7, -7.0, -1.3):
        b = 1.0
        for j in range(8):
            if j:
                b *= (p - (j - 1)) / j
            ref = math.gamma(p + 1) / (math.gamma(j + 1) * math.gamma(p - j + 1)) if p != int(p) else \
                (-1) ** j * math.comb(int(-p) + j - 1, j)
            assert b == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("name,n,k,terms,z", LEVELS, ids=LEVEL_IDS)
def test_float32_coefficients_as_the_kernel_forms_them(name, n, k, terms, z):
    """The kernels form A_j in float32 (node terms W_k 2^(pc log2 c_k + p log2 m_k), powers
    of 1/m_k by multiplication) and evaluate the polynomial by float32 Horner: the upper
    nodes carry at most ~2e-4 (mid level) or ~1.5e-3 (far level) of either sum, so the sums
    stay within 1e-9."""
    f32 = np.float32
    t, wk, c, m64, th2 = rule(n)
    m = m64.astype(f32).astype(np.float64)                 # the kernels' float32 m_k
    WSf, WQf = f32(wk * c), f32(wk * th2)
    lcf, lmf = f32(np.log2(m + 1.0)), f32(np.log2(m))
    worst, share = 0.0, 0.0
    for g in np.linspace(0.0, 2.999, 16):
        g4, ng, g3 = f32(g - 4), f32(-g), f32(3 - 2 * g)
        pS, pQ = float(g4), 2.0 * float(g4) + 1.0

        def coef(Wf, pc, p):
            e = (Wf[k:] * np.exp2(f32(pc) * lcf[k:] + f32(p) * lmf[k:]).astype(f32)).astype(f32)
            r = (f32(1.0) / m[k:].astype(f32)).astype(f32)
            out = []
            for j in range(terms):
                out.append(float(np.sum(e, dtype=f32)))
                e = (e * r).astype(f32)
            return out
        AS, AQ = coef(WSf, ng, pS), coef(WQf, g3, pQ)
        WS = WSf.astype(float) * c ** float(ng)
        WQ = WQf.astype(float) * c ** float(g3)
        for w in np.geomspace(z / m[k], 1.0 - 1e-6, 25):
            q = 1.0 + w * m
            for W, A, p in ((WS, AS, pS), (WQ, AQ, pQ)):
                terms_full = W * q ** p
                full = terms_full.sum()
                share = max(share, terms_full[k:].sum() / full)
                b, cf = 1.0, []
                for j in range(terms):
                    if j:
                        b *= (p - (j - 1)) / j
                    cf.append(f32(f32(b) * f32(A[j])))
                u, P = f32(1.0 / w), cf[-1]
                for j in range(terms - 2, -1, -1):
                    P = f32(f32(P * u) + cf[j])
                worst = max(worst, abs(terms_full[:k].sum() + w ** p * float(P) - full) / full)
    assert share < (1e-3 if name == "mid" else 2e-3), share
    assert worst < 1e-9, worst


@pytest.mark.parametrize("name,n,k,terms,z", [lv for lv in LEVELS if lv[0] == "mid"], ids=["mid64", "mid128"])
def test_adjoint_sums_of_the_series(name, n, k, terms, z):
    """The adjoint's six sums over the upper nodes (bang_device.cuh, fill_tail_coeffs_adj):
    sum W q^p, w sum W q^p c / q (series in p - 1 with A_j + A_{j+1}) and
    sum W q^p log2(c / q) + log2 w sum W q^p (with A'_j and the derivative of the binomial
    coefficients), for both integrals, against the node-by-node sums: within 1e-9 of the
    sum (of Sigma, resp. Sigma sigma^2, for the log-weighted ones, which can cross zero)."""
    t, wk, c, m, th2 = rule(n)
    lcm = np.log2(c / m)

    def binom(p, j):
        b = 1.0
        for i in range(j):
            b *= (p - i) / (i + 1)
        return b

    worst = 0.0
    for g in np.linspace(0.0, 2.999, 16):
        for W, p in ((wk * c * c ** -g, g - 4), (wk * th2 * c ** (3 - 2 * g), 2 * g - 7)):
            A = [np.sum((W * m ** (p - j))[k:]) for j in range(terms + 1)]
            Ap = [np.sum((W * lcm * m ** (p - j))[k:]) for j in range(terms)]
            for w in np.geomspace(z / m[k], 1.0 - 1e-6, 25):
                q = 1.0 + w * m
                tt = W * q ** p
                uw = c / q
                lu = np.log2(c) - np.log2(q)
                lw = np.log2(w)
                sums = [tt.sum(), w * (tt * uw).sum(), (tt * lu).sum() + lw * tt.sum()]
                head = [tt[:k].sum(), w * (tt * uw)[:k].sum(), (tt * lu)[:k].sum() + lw * tt[:k].sum()]
                u = 1.0 / w
                ser = [sum(binom(p, j) * A[j] * u ** j for j in range(terms)),
                       sum(binom(p - 1, j) * (A[j] + A[j + 1]) * u ** j for j in range(terms)),
                       sum((binom(p, j) * Ap[j] - binom(p, j) * sum(1.0 / (p - i) for i in range(j)) / math.log(2)
                            * A[j]) * u ** j for j in range(terms))]
                for i in range(3):
                    worst = max(worst, abs(head[i] + w ** p * ser[i] - sums[i]) / abs(sums[0]))
    assert worst < 1e-9, worst
