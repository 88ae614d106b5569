"""Nested-sampling driver (Sec. 2.5; Skilling 2004) against closed forms: Gaussian and
two-mode Gaussian evidences and the posterior moments, the information H, the exact
evidence of a constant likelihood, the shrinkage schedule of batched removal (the prior
mass enclosed by L = u is known exactly), checkpoint / resume bit for bit, and the prior
transforms.  Runs on the CPU with analytic likelihoods."""
import math
import pickle

import numpy as np
import pytest
from scipy.special import ndtr

from paper_2205_06819_gb300.nested import BoxPrior, NestedResult, NestedSampler


def _gauss(center, s, logw=0.0):
    c = np.asarray(center, dtype=np.float64)

    def ll(th):
        return -0.5 * np.sum(((th - c) / s) ** 2, axis=1) + logw
    return ll


def _cube(D):
    return BoxPrior(np.array([[0.0, 1.0]] * D))


def _gauss_logz(D, s):
    """ln of the integral of exp(-|u - 1/2|^2 / 2 s^2) over the unit cube."""
    return D * math.log(s * math.sqrt(2 * math.pi) * (ndtr(0.5 / s) - ndtr(-0.5 / s)))


@pytest.mark.parametrize("batch", [1, 20, 100])
def test_gaussian_evidence_moments_information(batch):
    D, s = 4, 0.04
    N, seeds = (100, 1) if batch == 1 else (200, 3)      # one-at-a-time removal is slow in Python
    exact = _gauss_logz(D, s)
    zs = []
    for seed in range(seeds):
        r = NestedSampler(_gauss(np.full(D, 0.5), s), _cube(D), n_live=N, batch=batch, seed=seed).run()
        z = (r.logz - exact) / r.logz_err
        zs.append(z)
        assert abs(z) < 3.5, (seed, r.logz, exact, r.logz_err)
        m, c = r.mean_cov()
        assert np.all(np.abs(m - 0.5) < 0.25 * s)
        assert np.all(np.abs(np.sqrt(np.diag(c)) / s - 1.0) < 0.15)
        # H = E_post[ln L] - ln Z = -D/2 - ln Z for a Gaussian inside the cube
        assert abs(r.information - (-D / 2 - exact)) < 0.6
        assert abs(np.exp(r.log_weights).sum() - 1.0) < 1e-12
    assert abs(np.mean(zs)) < 2.0


def test_two_modes_evidence_and_mode_weight():
    D, s = 3, 0.03
    a, b = _gauss(np.full(D, 0.3), s), _gauss(np.full(D, 0.7), s, math.log(0.5))

    def ll(th):
        return np.logaddexp(a(th), b(th))
    exact = math.log(1.5) + D * math.log(s * math.sqrt(2 * math.pi))
    r = NestedSampler(ll, _cube(D), n_live=300, batch=30, seed=0).run()
    assert abs(r.logz - exact) < 3.5 * r.logz_err
    w = np.exp(r.log_weights)
    assert abs(w[r.samples[:, 0] > 0.5].sum() - 1.0 / 3.0) < 0.15


def test_near_constant_likelihood_gives_exact_evidence():
    """L = c + 1e-9 u: Z = c to 1e-9, because the prior-mass widths of the discarded points
    and the final live share telescope to 1 whatever the batch."""
    for n_live, batch in ((64, 1), (64, 7), (100, 60)):
        smp = NestedSampler(lambda th: -3.25 + 1e-9 * th[:, 0], _cube(2), n_live=n_live, batch=batch, seed=1)
        r = smp.run()
        assert r.n_dead > 3 * n_live
        assert abs(r.logz - (-3.25)) < 2e-9
        assert abs(r.information) < 1e-6


def test_plateau_stops_with_exact_evidence():
    """A constant likelihood: no point can rise above the contour, so the sampler stops and
    the live points carry the whole prior mass."""
    r = NestedSampler(lambda th: np.full(len(th), -3.25), _cube(2), n_live=50, batch=5, seed=1).run()
    assert r.n_dead == 0 and r.logz == pytest.approx(-3.25, abs=1e-13)


@pytest.mark.parametrize("batch", [1, 50])
def test_shrinkage_schedule(batch):
    """With L = u on [0, 1] the prior mass above L* is exactly 1 - L*.  After removing points
    in batches of K from N live points, ln X is assigned -sum 1/(N-k); the true ln(1 - L*) of
    the batch's last point scatters around it with variance (iterations) x sum 1/(N-k)^2."""
    N, seeds, removed = (50, 8, 400) if batch == 1 else (100, 8, 1000)
    per_it = sum(1.0 / (N - k) for k in range(batch))
    var_it = sum(1.0 / (N - k) ** 2 for k in range(batch))
    devs, wrong = [], []
    for seed in range(seeds):
        smp = NestedSampler(lambda th: th[:, 0].copy(), _cube(1), n_live=N, batch=batch, seed=seed, frac=1e-300,
                            slice_steps=4)
        while smp.it * batch < removed:
            smp.step()
        assert abs(smp.logx + smp.it * per_it) < 1e-9
        last = float(np.concatenate(smp.dead_l)[-1])
        sd = math.sqrt(smp.it * var_it)
        devs.append((math.log1p(-last) - smp.logx) / sd)
        wrong.append((math.log1p(-last) + smp.it * batch / N) / sd)   # a K/N-per-batch schedule
    assert max(abs(d) for d in devs) < 4.0
    assert abs(np.mean(devs)) < 3.0 / math.sqrt(seeds)
    if batch > 1:
        assert abs(np.mean(wrong)) > 5.0


def test_checkpoint_resume_is_bitwise(tmp_path):
    ll, prior = _gauss(np.full(3, 0.5), 0.05), _cube(3)
    full = NestedSampler(ll, prior, n_live=80, batch=8, seed=5).run()
    path = str(tmp_path / "ns.pkl")
    part = NestedSampler(ll, prior, n_live=80, batch=8, seed=5)
    part.run(checkpoint=path, every=5, max_iter=12)
    assert part.it == 12
    with open(path, "rb") as f:
        assert pickle.load(f)["it"] == 12
    resumed = NestedSampler.resume(path, ll, prior).run()
    assert resumed.logz == full.logz and resumed.n_like == full.n_like
    assert np.array_equal(resumed.samples, full.samples)
    assert np.array_equal(resumed.log_weights, full.log_weights)


def test_box_prior_transforms():
    box = np.array([[0.0, 2.0], [5.0, 5.0], [0.1, 10.0], [math.radians(30), math.radians(70)]])
    pr = BoxPrior(box, sin_slot=3, log_slots=(2,))
    assert pr.ndim == 3 and list(pr.free) == [0, 2, 3]
    u = np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [0.5, 0.5, 0.5]])
    th = pr(u)
    assert np.all(th[:, 1] == 5.0)
    assert np.allclose(th[:, 0], [0.0, 2.0, 1.0])
    assert np.allclose(th[:, 2], [0.1, 10.0, 1.0])                          # uniform in log10
    s0, s1 = math.sin(math.radians(30)), math.sin(math.radians(70))
    assert np.allclose(np.sin(th[:, 3]), [s0, s1, 0.5 * (s0 + s1)])        # uniform in sin i


def test_quantiles_and_equal_weight_resampling():
    x = np.arange(10, dtype=np.float64)[:, None]
    w = np.array([1, 1, 1, 1, 1, 1, 1, 1, 1, 11], dtype=np.float64)
    lw = np.log(w / w.sum())
    r = NestedResult(0.0, 0.0, 0.0, 0, 0, 0, x, lw, np.zeros(10))
    q = r.quantiles([0.5])
    assert 8.0 <= q[0, 0] <= 9.0                   # half the weight sits on the last row
    eq = r.equal_weight_samples(seed=3)
    counts = np.bincount(eq[:, 0].astype(int), minlength=10)
    assert counts.sum() == 10
    assert np.all(np.abs(counts - 10 * w / w.sum()) < 1.0)


def test_nan_is_outside_and_bad_arguments():
    def ll(th):
        out = -0.5 * np.sum(((th - 0.5) / 0.1) ** 2, axis=1)
        out[th[:, 0] < 0.2] = np.nan
        return out
    r = NestedSampler(ll, _cube(2), n_live=60, batch=6, seed=2).run()
    assert np.isfinite(r.logz)
    assert np.all(r.samples[np.exp(r.log_weights) > 1e-6, 0] >= 0.2)
    with pytest.raises(ValueError):
        NestedSampler(ll, _cube(2), n_live=10, batch=10)
    with pytest.raises(ValueError):
        NestedSampler(ll, BoxPrior(np.array([[1.0, 1.0]])), n_live=10, batch=2)


def test_model_selection_boxes():
    """The three models of the paper's evidence comparison (Sec. 3.1): the truth lies inside
    every box it can be expressed in, fixed slots sit at the truth, the two discs cannot
    swap, and the rotation-dominated model carries the paper's extra priors."""
    from paper_2205_06819_gb300 import fit, synth
    t = fit.truth_two_discs()
    S = fit.SLOT
    b2, b1, br = (fit.selection_box(m, t) for m in ("BD1D2", "BD", "BD_rot"))
    assert b2.shape == (19, 2) and b1.shape == (15, 2) and br.shape == (15, 2)
    for b in (b2, b1):
        P = b.shape[0]
        assert np.all((b[:, 0] <= t[:P]) & (t[:P] <= b[:, 1]))
    for s in ("x0", "y0", "PA", "inc", "gamma", "logM200", "c", "vsys"):
        assert b2[S[s], 0] == b2[S[s], 1] == t[S[s]]
    assert b2[S["logRd1"], 1] <= b2[S["logRd2"], 0]
    assert br[S["k1"], 0] == 0.7 and br[S["MLd1"], 0] == 2.5 and br[S["logMb"], 1] == 11.1
    assert BoxPrior(b2).ndim == 11 and BoxPrior(b1).ndim == 7
    g = fit.selection_box("BD1D2", t, free_geometry=True)
    assert BoxPrior(g).ndim == 13 and g[S["inc"], 0] == pytest.approx(30 * synth.DEG)


def test_speculative_slice_step_has_the_same_distribution():
    """One hit-and-run slice step from the same start, one position per call against four:
    the new points follow the same distribution (two-sample KS on the radius and the
    angle), all inside the contour."""
    from scipy.stats import ks_2samp
    D = 2

    def ll(th):
        return -np.sum((th - 0.5) ** 2, axis=1)
    lstar = -0.2 ** 2
    start = np.tile([0.55, 0.48], (20000, 1))
    out = {}
    for m in (1, 4):
        s = NestedSampler(ll, _cube(D), n_live=10, batch=5, seed=11 + m, slice_steps=1, speculate=m)
        u, lu = s._chains(start.copy(), ll(start), lstar, np.eye(D) * 0.15)
        assert np.all(lu > lstar) and np.allclose(lu, ll(u))
        out[m] = u
    rad = {m: np.hypot(out[m][:, 0] - 0.5, out[m][:, 1] - 0.5) for m in out}
    ang = {m: np.arctan2(out[m][:, 1] - 0.5, out[m][:, 0] - 0.5) for m in out}
    assert ks_2samp(rad[1], rad[4]).pvalue > 1e-3
    assert ks_2samp(ang[1], ang[4]).pvalue > 1e-3


@pytest.mark.parametrize("speculate", [3, 8])
def test_speculative_chains_keep_the_evidence_with_fewer_calls(speculate):
    D, s = 4, 0.04
    exact = _gauss_logz(D, s)
    calls = {1: 0, speculate: 0}
    zs = []
    for m in (1, speculate):
        for seed in range(3):
            base = _gauss(np.full(D, 0.5), s)

            def ll(th, m=m):
                calls[m] += 1
                return base(th)
            r = NestedSampler(ll, _cube(D), n_live=200, batch=20, seed=seed, speculate=m).run()
            if m == speculate:
                z = (r.logz - exact) / r.logz_err
                zs.append(z)
                assert abs(z) < 3.5, (seed, r.logz, exact, r.logz_err)
                mu, c = r.mean_cov()
                assert np.all(np.abs(mu - 0.5) < 0.25 * s)
                assert np.all(np.abs(np.sqrt(np.diag(c)) / s - 1.0) < 0.15)
    assert abs(np.mean(zs)) < 2.0
    assert calls[speculate] < 0.6 * calls[1]


def test_speculative_two_modes_and_checkpoint(tmp_path):
    D, s = 3, 0.03
    a, b = _gauss(np.full(D, 0.3), s), _gauss(np.full(D, 0.7), s, math.log(0.5))

    def ll(th):
        return np.logaddexp(a(th), b(th))
    exact = math.log(1.5) + D * math.log(s * math.sqrt(2 * math.pi))
    r = NestedSampler(ll, _cube(D), n_live=300, batch=30, seed=0, speculate=4).run()
    assert abs(r.logz - exact) < 3.5 * r.logz_err
    w = np.exp(r.log_weights)
    assert abs(w[r.samples[:, 0] > 0.5].sum() - 1.0 / 3.0) < 0.15
    # the setting travels with a checkpoint; resuming is bit for bit
    full = NestedSampler(ll, _cube(D), n_live=60, batch=6, seed=2, speculate=4).run()
    path = str(tmp_path / "spec.pkl")
    part = NestedSampler(ll, _cube(D), n_live=60, batch=6, seed=2, speculate=4)
    part.run(checkpoint=path, every=4, max_iter=8)
    resumed = NestedSampler.resume(path, ll, _cube(D)).run()
    assert resumed.logz == full.logz and np.array_equal(resumed.samples, full.samples)
    with pytest.raises(ValueError):
        NestedSampler(ll, _cube(D), n_live=60, batch=6, speculate=0)


def test_speculative_limits_and_edges():
    """Search limits that m does not divide (max_steps_out 3, max_shrink 5 with m = 4), a
    slice so thin that shrinking runs out (the chain keeps its point), and chains at the
    cube's edge: every returned point is inside the contour and its logL is its own."""
    D = 3

    def ll(th):
        return -np.sum(((th - 0.02) / 0.3) ** 2, axis=1)   # mode near a corner of the cube
    for m, steps_out, shrink in ((4, 3, 5), (3, 16, 64), (8, 1, 1)):
        s = NestedSampler(ll, _cube(D), n_live=20, batch=5, seed=m, slice_steps=3, speculate=m,
                          max_steps_out=steps_out, max_shrink=shrink)
        start = np.vstack([np.full(D, 0.02), np.full(D, 0.001), np.array([0.3, 0.02, 0.5])])
        lstar = float(ll(start).min()) - 0.5
        u, lu = s._chains(start.copy(), ll(start), lstar, np.eye(D) * 0.2)
        assert np.all((u >= 0.0) & (u <= 1.0))
        assert np.all(lu > lstar) and np.allclose(lu, ll(u))
    # a thin slice: the contour sits just below the start's logL, shrinking is cut off
    s = NestedSampler(ll, _cube(D), n_live=20, batch=5, seed=1, slice_steps=1, speculate=4, max_shrink=2)
    start = np.full((4, D), 0.02)
    lstar = float(ll(start[:1])[0]) - 1e-12
    u, lu = s._chains(start.copy(), ll(start), lstar, np.eye(D) * 0.5)
    assert np.all(lu > lstar)


def test_call_size_buckets():
    """gpu_loglike pads a call to a bucket size: never smaller than the call, a multiple of
    4, at most 1/3 (1/4 from 60 on) larger than the bucket below, and few sizes in all (the
    library keeps 32 plans)."""
    from paper_2205_06819_gb300.nested import _bucket
    sizes = sorted({_bucket(n) for n in range(1, 3001)})
    assert all(_bucket(n) >= n for n in range(1, 5000))
    assert all(b % 4 == 0 for b in sizes) and sizes[0] == 16
    assert all(b1 <= b0 * 4 // 3 + 4 for b0, b1 in zip(sizes, sizes[1:]))
    assert len(sizes) <= 24
