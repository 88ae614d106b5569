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
