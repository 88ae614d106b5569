"""Full-size parity of the workloads, in the launch shapes bench.py times.

single and batched: chi^2 and every map element of the first, middle and last rows.

uneven: 64 galaxies with spaxel grids drawn from {32x32, 48x64, 78x73, 96x96, 128x128}, 4x4
oversampling, Gaussian PSF FWHM U[1.5, 3.5]", 64 rows each: the 4096 rows in one
persistent launch after the autotuner has chosen its shape for that batch (as bench.py
does).  Checked against the float64 oracle: the first and last rows and one row of every
grid size, chi^2 and every element of the four maps.

largest: 128x128 spaxels, 7x7 oversampling, Moffat PSF (beta 3, FWHM 2.5"), two discs, 128
radial nodes: the 4096-row batch in one tuned launch; six rows (first, last and four
spread over the batch) checked for chi^2 and every map element, with the largest error of
each map printed (run with -s); the gradient of two rows from the 1024-row gradient launch
bench.py times for this workload, against the oracle's dual-number gradient.

Bars: chi^2 within 1e-5 relative; maps within 2e-5 relative (B, sigma, M/L) and 2e-5 of the
map's largest |v| (velocity); the gradient bar of bang_testdata.assert_grad_close.  The
data are the oracle's noise-free maps at each galaxy's seeded true parameters plus noise,
the rows the seeded batches of synth.workload.
"""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2205_06819_gb300 import synth  # noqa: E402

from bang_testdata import Dataset, assert_grad_close, grad_errors  # noqa: E402

CHI2_RTOL = 1e-5
MAP_RTOL = 2e-5


@pytest.fixture(scope="module")
def Model():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2205_06819_gb300 import build as b
    oracle.build()
    b.build()
    from paper_2205_06819_gb300.model import Model
    return Model


def workload_data(name):
    """The workload's galaxies as test datasets (oracle maps + noise), its rows and gal_idx."""
    wl = synth.workload(name)
    wid = synth.workload_id(name)
    box = synth.prior_box(wl.n_discs, wl.gamma_fixed)
    dss = []
    for g, spec in enumerate(wl.galaxies):
        tt = synth.draw_theta_true(box, synth.dataset_seed(wid, g))
        dss.append(Dataset(spec, tt, n_discs=wl.n_discs, n_quad=wl.n_quad, seed=synth.dataset_seed(wid, g)))
    theta = np.concatenate([synth.draw_theta_batch(box, d.theta_true, wl.rows_per_galaxy, synth.batch_seed(wid) + 7 * g)
                            for g, d in enumerate(dss)]).astype(np.float32)
    gal_idx = np.repeat(np.arange(len(dss), dtype=np.int32), wl.rows_per_galaxy)
    return wl, dss, theta, gal_idx


def map_errors(got, ref):
    """Largest error of each map: B, sigma, M/L relative per element; v over the map's largest |v|."""
    out = {}
    for c, name in enumerate(["B", "v", "sigma", "ML"]):
        if name == "v":
            out[name] = float(np.abs(got[c] - ref[c]).max() / np.abs(ref[c]).max())
        else:
            out[name] = float((np.abs(got[c] - ref[c]) / np.abs(ref[c])).max())
    return out


def check_rows(Model, wl, dss, theta, gal_idx, pick, label):
    """The whole batch in one tuned launch (logL, then the maps of every row), the picked
    rows against the oracle.  Returns the largest errors."""
    multi = len(dss) > 1
    m = Model([d.model_galaxy() for d in dss], n_discs=wl.n_discs, n_quad=wl.n_quad)
    gi = gal_idx if multi else None
    B = theta.shape[0]
    m.tune(B, gi)
    t = torch.from_numpy(theta).cuda()
    logL = m.loglike(t, gi).cpu().numpy()
    maps = m.maps(t, gi)
    worst = {"chi2": 0.0, "B": 0.0, "v": 0.0, "sigma": 0.0, "ML": 0.0}
    import oracle
    for b in pick:
        d = dss[gal_idx[b]]
        ref_l, ref_chi2 = d.oracle_loglike(theta[b:b + 1])
        assert np.isfinite(ref_l[0]) and np.isfinite(logL[b]), (label, b)
        chi = -2.0 * (logL[b] + oracle.norm_const(d.og))
        rel = abs(chi - ref_chi2[0]) / ref_chi2[0]
        worst["chi2"] = max(worst["chi2"], float(rel))
        assert rel < CHI2_RTOL, (label, b, rel)
        me = map_errors(maps[b].cpu().numpy(), d.oracle_maps(theta[b]))
        for k, v in me.items():
            worst[k] = max(worst[k], v)
        assert max(me.values()) < MAP_RTOL, (label, b, me)
    del maps
    return m, worst


@pytest.mark.parametrize("name", ["single", "batched"])
def test_single_and_batched_workloads_maps(Model, name):
    """The single-row workload (30x30, os 3, gamma = 1) and the batched one (80x80, os 5, 1024
    rows): chi^2 and every map element of the first, middle and last rows."""
    wl, dss, theta, gal_idx = workload_data(name)
    B = theta.shape[0]
    pick = sorted({0, B // 2, B - 1})
    m, worst = check_rows(Model, wl, dss, theta, gal_idx, pick, name)
    m.close()
    print(json.dumps({"workload": name, "rows": int(B), "rows_checked": pick, "max_rel_chi2": worst["chi2"],
                      "max_map_err": {k: worst[k] for k in ("B", "v", "sigma", "ML")}}))


def test_uneven_workload_full_size(Model):
    wl, dss, theta, gal_idx = workload_data("uneven")
    sizes = {}
    for b in range(theta.shape[0]):
        s = dss[gal_idx[b]].spec
        sizes.setdefault((s.nx, s.ny), b)
    assert len(sizes) == 5
    pick = sorted({0, theta.shape[0] - 1, *sizes.values()})
    m, worst = check_rows(Model, wl, dss, theta, gal_idx, pick, "uneven")
    m.close()
    print(json.dumps({"workload": "uneven", "rows": int(theta.shape[0]), "rows_checked": [int(b) for b in pick],
                      "max_rel_chi2": worst["chi2"],
                      "max_map_err": {k: worst[k] for k in ("B", "v", "sigma", "ML")}}))


def test_largest_workload_full_size(Model):
    wl, dss, theta, gal_idx = workload_data("largest")
    B = theta.shape[0]
    pick = [0, 1, 1000, 2047, 3000, B - 1]
    m, worst = check_rows(Model, wl, dss, theta, gal_idx, pick, "largest")
    # the gradient launch bench.py times for this workload: the first 1024 rows
    import oracle
    Bg = 1024
    tg = torch.from_numpy(theta[:Bg]).cuda()
    m.tune(Bg, grad=True)
    lg, g = m.loglike_grad(tg)
    g = g.cpu().numpy()
    ds = dss[0]
    rows = [0, Bg - 1]                     # a posterior-like row and a prior draw
    _, gref = oracle.loglike_grad(ds.og, theta[rows].astype(np.float64), n_discs=2, n_quad=128)
    gerr = grad_errors(g[rows], gref)
    print(json.dumps({"workload": "largest", "rows": int(B), "rows_checked": pick, "max_rel_chi2": worst["chi2"],
                      "max_map_err": {k: worst[k] for k in ("B", "v", "sigma", "ML")},
                      "grad_rows": rows, "grad_err_over_norm": max(e[0] for e in gerr),
                      "grad_err_component_relative": max(e[1] for e in gerr)}))
    assert_grad_close(g[rows], gref, "largest")
    m.close()
