"""bench.py's algorithmic operation counts and peaks (the roofline denominators): the
per-point SFU and FP32 counts of the forward and gradient paths as documented, the
row-subset counts, and the roofline arithmetic from the measured per-SM rates."""
import math
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from paper_2205_06819_gb300 import synth  # noqa: E402


def test_padded_points_and_sfu_count_of_the_batched_workload():
    wl = synth.workload("batched")
    assert bench.points_per_eval(wl.galaxies[0]) == 430 * 430          # 80 x 5 + 2 x 15
    # forward: per node below the series split one lg2 and one ex2; the series one reciprocal
    # and two ex2; per point 13 half-rate and 4 ex2 (one disc)
    per_eval = bench.algorithmic_sfu_ops(wl) / wl.batch
    assert per_eval == 430 * 430 * (18 + 14 + 18 + 6)
    ops, cyc = bench.sfu_work(wl)
    assert cyc / wl.batch == pytest.approx(430 * 430 * ((18 + 14) / 16 + (18 + 6) / 32), rel=1e-12)


def test_series_split_matches_the_kernel_header():
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2205_06819_gb300",
                            "csrc", "bang_device.cuh")).read()
    rules = re.findall(r"struct TailRule<(\d+)> \{ static constexpr int K = (\d+), KF = (\d+);", hdr)
    assert {int(n): int(kf) for n, _, kf in rules} == bench.TAIL_SPLIT
    assert {int(n): int(k) for n, k, _ in rules} == bench.MID_SPLIT
    assert int(re.search(r"constexpr int kTailTerms = (\d+);", hdr).group(1)) == bench.MID_TERMS
    assert int(re.search(r"constexpr int kFarTerms = (\d+);", hdr).group(1)) == bench.FAR_TERMS


def test_sfu_count_of_the_gradient_step():
    """logL + gradient = the forward seed pass plus the adjoint: per node below the split one
    lg2 and two ex2 (q^(g-4) and u/w), the series one reciprocal and two ex2, per point 18
    half-rate and 4 ex2 (one disc); two discs add half a half-rate and one ex2 per point to
    each pass."""
    wl = synth.workload("adjoint")
    ops, cyc = bench.sfu_work(wl, grad=True)
    fwd = 430 * 430 * ((18 + 14) / 16 + (18 + 6) / 32)
    adj = 430 * 430 * ((24 + 19) / 16 + (48 + 6) / 32)
    assert cyc / wl.batch == pytest.approx(fwd + adj, rel=1e-12)
    assert ops / wl.batch == 430 * 430 * (18 + 14 + 18 + 6 + 24 + 19 + 48 + 6)
    assert bench.sfu_ops_per_point(128, 2, True) == {"half": 48 + 19.5, "full": 96 + 7}
    assert bench.sfu_ops_per_point_node_by_node(128, 2, True) == {"half": 128 + 18.5, "full": 256 + 5}
    assert bench.sfu_ops_per_point(128, 2, False) == {"half": 36 + 14.5, "full": 36 + 7}


def test_fp32_count_of_the_batched_and_largest_workloads():
    wl = synth.workload("batched")
    L = 5 + 2 * 15
    psf = 4.0 * ((5 * 80 + 30) * 80 + 80 * 80) * L
    expect = 430 * 430 * (6 * 18 + 28 + 200) + psf + 40 * 6400
    assert bench.algorithmic_fp32_ops(wl) / wl.batch == pytest.approx(expect, rel=1e-12)
    big = synth.workload("largest")                                   # Moffat: two-dimensional taps
    h = int(math.floor(3.0 * 2.5 / 2.35482 / (1.0 / 7)))
    L = 7 + 2 * h
    expect = (7 * 128 + 2 * h) ** 2 * (6 * 36 + 28 + 200) + 4.0 * 128 * 128 * L * L + 40 * 128 * 128
    assert bench.algorithmic_fp32_ops(big) / big.batch == pytest.approx(expect, rel=1e-12)


def test_row_subsets_of_an_uneven_batch():
    wl = synth.workload("uneven")
    gi = [0] * 3 + [5] * 2
    per = [bench.points_per_eval(g) for g in wl.galaxies]
    assert bench.algorithmic_sfu_ops(wl, gi, 5) == (3 * per[0] + 2 * per[5]) * (18 + 14 + 18 + 6)


def test_roofline_block_arithmetic():
    """frac = the SFU time of the step's operations at the per-SM issue rates over the
    measured time; peak = operations over that time."""
    wl = synth.workload("batched")
    t_sfu = 1024 * 430 * 430 * ((18 + 14) / 16 + (18 + 6) / 32) / (152 * 2070e6)
    r = bench.roofline_block(wl, 2.0 * t_sfu, mhz=2070.0, sms=152)
    assert r["sfu_frac"] == pytest.approx(0.5, rel=1e-12)
    assert r["frac"] == pytest.approx(max(r["sfu_frac"], r["fp32"]["frac"]), rel=1e-12)
    ops = 1024 * 430 * 430 * 56
    assert r["peak"] == pytest.approx(ops / t_sfu / 1e9, rel=1e-12)
    assert r["achieved"] == pytest.approx(r["peak"] / 2, rel=1e-12)
    assert r["sfu_sm_cycles_per_point"] == pytest.approx((18 + 14) / 16 + (18 + 6) / 32, rel=1e-12)
    nbn = 1024 * 430 * 430 * ((64 + 13) / 16 + (64 + 4) / 32) / (152 * 2070e6)
    assert r["node_by_node_sfu_frac"] == pytest.approx(nbn / (2.0 * t_sfu), rel=1e-12)
    g = bench.roofline_block(synth.workload("adjoint"), 1e-3, grad=True, mhz=2070.0, sms=152)
    assert g["frac"] > 0 and g["fp32"]["frac"] > 0


def test_cpu_baseline_parity_sample():
    """The cpu_baseline leg compares the oracle's chi^2 of the rows it timed with the logL it
    is given: the oracle's own logL passes, one perturbed by 1e-4 of chi^2 fails."""
    import numpy as np
    import oracle
    oracle.build()
    spec = synth.GalaxySpec(12, 10, 2, 2.0)
    box = synth.prior_box(1)
    th = synth.draw_theta_true(box, 3)
    og = oracle.Galaxy(spec.nx, spec.ny, spec.oversample, spec.psf_fwhm_arcsec, spec.kpc_per_arcsec)
    data, err, mask = synth.noisy_data(oracle.maps(og, th), seed=4)
    theta = synth.draw_theta_batch(box, th, 3, seed=5).astype(np.float32)

    class Gal:
        nx, ny, oversample, psf_fwhm_arcsec, kpc_per_arcsec = spec.nx, spec.ny, spec.oversample, 2.0, \
            spec.kpc_per_arcsec
        psf_kind, moffat_beta = 0, 3.0

    Gal.data, Gal.err, Gal.mask = data, err, mask

    class WL:
        n_discs, n_quad = 1, 64

    og2 = oracle.Galaxy(spec.nx, spec.ny, spec.oversample, 2.0, spec.kpc_per_arcsec, data=data.astype(np.float64),
                        err=err.astype(np.float64), mask=mask)
    logL, chi2 = oracle.loglike(og2, theta.astype(np.float64))
    ok = bench.cpu_oracle_sample(WL, Gal, theta, 0.05, logL)
    assert ok["parity"]["rows"] >= 1 and ok["parity"]["pass"]
    assert ok["parity"]["max_rel_chi2_err"] < 1e-12
    bad = bench.cpu_oracle_sample(WL, Gal, theta, 0.05, logL + 0.5e-4 * chi2)
    assert not bad["parity"]["pass"]


def test_list_workloads_prints_the_five_configurations():
    """``bench.py --list-workloads`` prints each workload as plain data (no GPU needed)."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                                       "bench.py"), "--list-workloads"],
                         capture_output=True, text=True, check=True).stdout.strip().splitlines()
    rows = [json.loads(line) for line in out]
    assert [r["workload"] for r in rows] == list(synth.WORKLOADS)
    by = {r["workload"]: r for r in rows}
    assert by["batched"]["rows"] == 1024 and by["batched"]["padded_fine_points_per_row"] == 430 * 430
    assert by["adjoint"]["gradient"] and by["adjoint"]["rows"] == 256
    assert by["largest"]["n_discs"] == 2 and by["largest"]["n_quad"] == 128 and by["largest"]["rows"] == 4096
    assert by["largest"]["padded_fine_points_per_row"] == 940 * 940
    assert by["uneven"]["rows"] == 64 * 64 and sum(g["count"] for g in by["uneven"]["galaxies"]) == 64
    assert by["single"]["rows"] == 1 and by["single"]["gamma_fixed"] == 1.0
