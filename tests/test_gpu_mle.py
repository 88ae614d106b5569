"""A gradient-based method on the shared likelihood: L-BFGS through the LogLike autograd
function (the adjoint) climbs from a start 5% of the prior range off to the maximum of the
likelihood; the maximum beats the truth's logL (noisy data) and lies within a few percent
of the prior range of the truth."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2205_06819_gb300 import fit, synth  # noqa: E402

from bang_testdata import Dataset  # noqa: E402


def test_lbfgs_on_the_adjoint_finds_the_maximum():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_06819_gb300 import build as b
    b.build()
    from paper_2205_06819_gb300.model import Model
    truth = fit.truth_two_discs()
    ds = Dataset(synth.GalaxySpec(24, 20, 3, 2.5), truth, n_discs=2, seed=91)
    m = Model(ds.model_galaxy(), n_discs=2)
    box = fit.selection_box("BD1D2", truth)
    free = np.flatnonzero(box[:, 1] > box[:, 0])
    lo, hi = box[free, 0], box[free, 1]
    start = truth.copy()
    start[free] += 0.05 * (hi - lo) * np.random.default_rng(3).choice([-1.0, 1.0], size=free.size)
    start[free] = np.clip(start[free], lo, hi)
    l_start = float(m.loglike(torch.from_numpy(start.astype(np.float32)[None]).cuda())[0])
    l_truth = float(m.loglike(torch.from_numpy(truth.astype(np.float32)[None]).cuda())[0])
    th, l_best = fit.max_likelihood(m, start, free, lo, hi, iters=80)
    assert l_best > l_start and l_best >= l_truth - 1.0
    assert np.all(np.abs(th[free] - truth[free]) <= 0.02 * (hi - lo)), (th[free] - truth[free]) / (hi - lo)
