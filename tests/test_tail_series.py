"""The upper-node series of the forward kernel's radial rule (bang_device.cuh, TailRule,
fill_tail_coeffs, bulge_projected_w), restated in float64 and checked against the plain
node-by-node sum it replaces.

For nodes k >= K of the rule r = R cosh t (t in [0, 16], n Gauss-Legendre nodes), a point's
q_k = 1 + w m_k (m_k = cosh t_k - 1) is expanded as (w m_k)^p (1 + 1/(w m_k))^p, so that
sum_{k>=K} W_k q_k^p = w^p sum_j binom(p, j) A_j w^-j with per-model A_j = sum W_k m_k^(p-j);
the kernel keeps kTailTerms terms and uses the series where w m_K >= kTailZ.  The header's
constants are read from the source; the claim pinned here is the one its comment makes:
truncation below 1e-9 of the whole sum, for both projected integrals (Sigma: p = g - 4,
W = w_k cosh t_k cosh^-g t_k; Sigma sigma^2: p = 2g - 7, W = w_k tanh^2 t_k cosh^(3-2g) t_k)
over gamma in [0, 3) and every w the series serves.
"""
import math
import os
import re

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "paper_2205_06819_gb300", "csrc", "bang_device.cuh")


def header_constants():
    text = open(HEADER).read()
    K = {int(n): int(k) for n, k in re.findall(r"struct TailRule<(\d+)> \{ static constexpr int K = (\d+);", text)}
    terms = int(re.search(r"constexpr int kTailTerms = (\d+);", text).group(1))
    z = float(re.search(r"constexpr float kTailZ = ([0-9.]+)f;", text).group(1))
    return K, terms, z


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


@pytest.mark.parametrize("n", [64, 128])
def test_series_truncation_below_1e9_of_the_sum(n):
    K, terms, z = header_constants()
    assert set(K) == {64, 128}
    t, wk, c, m, th2 = rule(n)
    k = K[n]
    assert k % 2 == 0 and 4.5 < t[k] < 5.5           # the split sits near t = 5
    wmin = z / m[k]
    assert wmin < 0.25                                # the series serves all but the centre
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


def test_a_shorter_series_or_a_looser_threshold_would_fail():
    """The pin has teeth: two terms, or the series used down to w m_K = 2, miss 1e-9."""
    K, terms, z = header_constants()
    t, wk, c, m, th2 = rule(64)
    k = K[64]
    g = 2.5
    WQ = wk * th2 * c ** (3 - 2 * g)

    def err(nterms, w):
        q = 1.0 + w * m
        full = np.sum(WQ * q ** (2 * g - 7))
        head = np.sum((WQ * q ** (2 * g - 7))[:k])
        return abs(head + series(WQ, m, 2 * g - 7, k, nterms, w) - full) / full

    assert err(2, z / m[k]) > 1e-9
    assert err(terms, 2.0 / m[k]) > 1e-9


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


@pytest.mark.parametrize("n", [64, 128])
def test_float32_coefficients_as_the_kernel_forms_them(n):
    """The kernels form A_j in float32 (node terms W_k 2^(pc log2 c_k + p log2 m_k), powers
    of 1/m_k by multiplication): the upper nodes carry at most ~2e-4 of either sum, so the
    float32 coefficients still leave the sums within 1e-9."""
    K, terms, z = header_constants()
    f32 = np.float32
    t, wk, c, m64, th2 = rule(n)
    k = K[n]
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
                b, s = 1.0, 0.0
                for j in range(terms):
                    if j:
                        b *= (p - (j - 1)) / j
                    s += b * A[j] * w ** (-j)
                worst = max(worst, abs(terms_full[:k].sum() + w ** p * s - full) / full)
    assert share < 1e-3, share
    assert worst < 1e-9, worst


@pytest.mark.parametrize("n", [64, 128])
def test_adjoint_sums_of_the_series(n):
    """The adjoint's six sums over the upper nodes (bang_device.cuh, fill_tail_coeffs_adj):
    sum W q^p, w sum W q^p c / q (series in p - 1 with A_j + A_{j+1}) and
    sum W q^p log2(c / q) + log2 w sum W q^p (with A'_j and the derivative of the binomial
    coefficients), for both integrals, against the node-by-node sums: within 1e-9 of the
    sum (of Sigma, resp. Sigma sigma^2, for the log-weighted ones, which can cross zero)."""
    K, terms, z = header_constants()
    t, wk, c, m, th2 = rule(n)
    k = K[n]
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
