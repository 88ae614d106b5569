"""Nested sampling on the CUDA likelihood: the synthetic analogue of the paper's evidence
comparison (Sec. 3.1).  Data come from a bulge + inner disc + outer disc galaxy (oracle
maps plus the Sec. 3.1 noise model); the evidence must prefer the two-disc model by a wide
margin, the two-disc posterior must cover the truth, and the best sample's logL must match
the oracle."""
import numpy as np
import pytest

from bang_testdata import Dataset
from paper_2205_06819_gb300 import fit, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def selection():
    spec = synth.GalaxySpec(24, 24, 3, 2.5)
    truth = fit.truth_two_discs()
    ds = Dataset(spec, truth, n_discs=2, seed=11)
    out = {}
    for name in ("BD1D2", "BD"):
        out[name] = fit.run_model(name, spec, ds.data, ds.err, truth, n_live=100, batch=20, seed=3)
    return ds, truth, out


def test_evidence_prefers_two_discs(selection):
    _, _, out = selection
    (r2, row2), (r1, row1) = out["BD1D2"], out["BD"]
    print({k: (v[1]["logZ"], v[1]["logZ_err"], v[1]["n_like"], round(v[1]["evals_per_s"])) for k, v in out.items()})
    assert np.isfinite(r2.logz) and np.isfinite(r1.logz)
    assert r2.logz - r1.logz > 10.0 + 5 * (r2.logz_err + r1.logz_err)


def test_two_disc_posterior_covers_truth(selection):
    _, truth, out = selection
    r2, _ = out["BD1D2"]
    prior_free = np.flatnonzero(fit.selection_box("BD1D2", truth)[:, 1] > fit.selection_box("BD1D2", truth)[:, 0])
    q = r2.quantiles([0.16, 0.5, 0.84])
    for j in prior_free:
        half = max(0.5 * (q[2, j] - q[0, j]), 1e-3 * abs(truth[j]) + 1e-4)
        assert abs(q[1, j] - truth[j]) < 5.0 * half, (synth.PARAM_NAMES_2[j], q[:, j], truth[j])


def test_best_sample_matches_oracle(selection):
    import oracle
    ds, _, out = selection
    r2, _ = out["BD1D2"]
    best = r2.samples[np.argmax(r2.log_l)][None, :].astype(np.float32)
    norm = oracle.norm_const(ds.og)
    chi2_gpu = -2.0 * (r2.log_l.max() + norm)
    chi2_or = -2.0 * (ds.oracle_loglike(best)[0] + norm)
    assert abs(chi2_gpu - chi2_or) <= 1e-5 * chi2_or, (chi2_gpu, chi2_or)


def test_padded_calls_return_the_rows_own_values():
    """gpu_loglike pads each call to a bucket size with copies of its first row: the values
    returned are the call's own rows, equal to an unpadded call of the bucket's size."""
    from paper_2205_06819_gb300.model import Model
    from paper_2205_06819_gb300.nested import _bucket, gpu_loglike
    import torch
    spec = synth.GalaxySpec(16, 14, 3, 2.5)
    truth = fit.truth_two_discs()
    ds = Dataset(spec, truth, n_discs=2, seed=21)
    m = Model([ds.model_galaxy()], n_discs=2)
    try:
        box = fit.selection_box("BD1D2", truth)
        rng = np.random.default_rng(4)
        th = box[:, 0] + rng.random((37, box.shape[0])) * (box[:, 1] - box[:, 0])
        got = gpu_loglike(m)(th)
        nb = _bucket(37)
        assert got.shape == (37,) and nb == 48
        full = np.concatenate([th, np.repeat(th[:1], nb - 37, axis=0)]).astype(np.float32)
        ref = m.loglike(torch.from_numpy(full)).numpy()
        assert np.array_equal(got, ref[:37]) and np.isfinite(got).all()
    finally:
        m.close()
