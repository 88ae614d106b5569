"""GPU parity of the hand-written adjoint (d logL / d theta) through the C ABI.

References: the FP64 oracle's forward-mode dual-number gradient of the same discrete
likelihood, and Richardson-extrapolated central differences of the oracle's logL with
h = 1e-4 * max(|theta_p|, 1).  Tolerance: per row, the gradient vector within 1e-4 of the
oracle's in relative Euclidean norm, every component within 5e-5 of that norm, and every
component of at least 5% of the norm within 1e-4 of its own size (bang_testdata.GRAD_RTOL).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2205_06819_gb300 import synth  # noqa: E402

from bang_testdata import Dataset, assert_grad_close, theta_batch  # noqa: E402

GRAD_RTOL = 1e-4
CHI2_RTOL = 1e-5

TH1 = np.array([0.05, -0.08, 0.4, 0.95, 10.2, math.log10(0.9), 1.3, 10.4, math.log10(2.8), 0.55,
                3.5, 2.0, 12.4, 9.0, 15.0])
TH2 = np.concatenate([TH1, [10.1, math.log10(4.0), 0.8, 2.5]])


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


def oracle_grad(ds, theta32):
    import oracle
    th = np.asarray(theta32, np.float32).astype(np.float64)
    return oracle.loglike_grad(ds.og, th, n_discs=ds.n_discs, n_quad=ds.n_quad)


def run(Model, ds, theta):
    m = Model(ds.model_galaxy(), n_discs=ds.n_discs, n_quad=ds.n_quad)
    logL, grad = m.loglike_grad(torch.from_numpy(theta).cuda())
    logL2 = m.loglike(torch.from_numpy(theta).cuda())
    return m, logL.cpu().numpy(), grad.cpu().numpy(), logL2.cpu().numpy()


def test_gradient_matches_oracle_ragged_grid(Model):
    ds = Dataset(synth.GalaxySpec(17, 13, 3, 2.2), TH1, seed=41)
    theta = theta_batch(1, TH1, 10, seed=42)
    _, logL, grad, logL2 = run(Model, ds, theta)
    np.testing.assert_allclose(logL, logL2, rtol=1e-12)
    ref_logL, ref_grad = oracle_grad(ds, theta)
    chi = -2 * (logL + __import__("oracle").norm_const(ds.og))
    chi_ref = -2 * (ref_logL + __import__("oracle").norm_const(ds.og))
    assert (np.abs(chi - chi_ref) / chi_ref).max() < CHI2_RTOL
    assert_grad_close(grad, ref_grad, "ragged")


def test_gradient_matches_oracle_finite_differences(Model):
    import oracle
    ds = Dataset(synth.GalaxySpec(9, 8, 2, 1.8), TH1, seed=43)
    theta = theta_batch(1, TH1, 2, seed=44)
    _, _, grad, _ = run(Model, ds, theta)
    for b in range(theta.shape[0]):
        th = theta[b].astype(np.float64)
        fd = np.zeros(th.size)
        for p in range(th.size):
            def central(h):
                tp, tm = th.copy(), th.copy()
                tp[p] += h
                tm[p] -= h
                return (oracle.loglike(ds.og, tp)[0][0] - oracle.loglike(ds.og, tm)[0][0]) / (2 * h)
            h = 1e-4 * max(abs(th[p]), 1.0)
            fd[p] = (4 * central(h / 2) - central(h)) / 3
        # differences of float64 logL values: their noise bounds small components, so the
        # bar here is the norm one (the dual-number gradient takes the per-component bar)
        nrm = np.linalg.norm(fd)
        assert np.abs(grad[b] - fd).max() <= GRAD_RTOL * nrm, ("fd", b, np.abs(grad[b] - fd) / nrm)


def test_gradient_moffat_two_discs_128_nodes(Model):
    ds = Dataset(synth.GalaxySpec(12, 10, 3, 2.5, psf_kind=1, moffat_beta=3.0), TH2, n_discs=2, n_quad=128, seed=45)
    theta = theta_batch(2, TH2, 6, seed=46)
    _, _, grad, _ = run(Model, ds, theta)
    _, ref = oracle_grad(ds, theta)
    assert_grad_close(grad, ref, "moffat")


def test_gradient_edge_parameters_and_domain(Model):
    ds = Dataset(synth.GalaxySpec(11, 9, 2, 1.6), TH1, seed=47)
    rows = np.repeat(TH1[None], 7, 0).astype(np.float32)
    rows[0, 6] = 0.0
    rows[1, 6] = 2.9
    rows[2, 9] = 1.0
    rows[3, 3] = 0.0
    rows[4, 3] = 1.6      # out of domain
    rows[5, 13] = -2.0    # out of domain
    rows[6, [0, 1]] = 0.0
    _, logL, grad, _ = run(Model, ds, rows)
    assert np.all(np.isneginf(logL[[4, 5]])) and np.all(grad[[4, 5]] == 0)
    ok = [0, 1, 2, 3, 6]
    _, ref = oracle_grad(ds, rows[ok])
    assert_grad_close(grad[ok], ref, "edge")


def test_uneven_batch_gradient(Model):
    specs = [synth.GalaxySpec(7, 9, 3, 1.5), synth.GalaxySpec(14, 11, 3, 2.9)]
    dss = [Dataset(s, TH1, seed=50 + k) for k, s in enumerate(specs)]
    thetas = [theta_batch(1, TH1, 3, seed=60 + k) for k in range(2)]
    gal_idx = np.array([0, 1, 0, 1, 0, 1], dtype=np.int32)
    theta = np.empty((6, 15), np.float32)
    theta[gal_idx == 0] = thetas[0]
    theta[gal_idx == 1] = thetas[1]
    m = Model([d.model_galaxy() for d in dss])
    _, grad = m.loglike_grad(torch.from_numpy(theta).cuda(), gal_idx=gal_idx)
    grad = grad.cpu().numpy()
    for k, ds in enumerate(dss):
        _, ref = oracle_grad(ds, theta[gal_idx == k])
        assert_grad_close(grad[gal_idx == k], ref, f"uneven{k}")


def test_autograd_function(Model):
    from paper_2205_06819_gb300.model import LogLike
    ds = Dataset(synth.GalaxySpec(8, 7, 2, 1.5), TH1, seed=71)
    m = Model(ds.model_galaxy())
    theta = torch.from_numpy(theta_batch(1, TH1, 4, seed=72)).cuda().requires_grad_(True)
    w = torch.tensor([1.0, -2.0, 0.5, 3.0], dtype=torch.float64, device="cuda")
    (LogLike.apply(theta, m) * w).sum().backward()
    _, g = m.loglike_grad(theta.detach())
    torch.testing.assert_close(theta.grad, g * w.float()[:, None], rtol=1e-6, atol=0)


def test_host_buffers(Model):
    ds = Dataset(synth.GalaxySpec(8, 6, 2, 1.5), TH1, seed=73)
    m = Model(ds.model_galaxy())
    theta = theta_batch(1, TH1, 3, seed=74)
    l_dev, g_dev = m.loglike_grad(torch.from_numpy(theta).cuda())
    l_host, g_host = m.loglike_grad(torch.from_numpy(theta))
    np.testing.assert_array_equal(l_dev.cpu().numpy(), l_host.numpy())
    np.testing.assert_allclose(g_dev.cpu().numpy(), g_host.numpy(), rtol=1e-6)


def test_full_size_adjoint_workload_sampled_rows(Model):
    """The 256-row 80x80 (os 5) adjoint workload in one call; two rows against the oracle."""
    wl = synth.workload("adjoint")
    wid = synth.workload_id("adjoint")
    box = synth.prior_box(1)
    tt = synth.draw_theta_true(box, synth.dataset_seed(wid))
    ds = Dataset(wl.galaxies[0], tt, seed=synth.dataset_seed(wid))
    theta = synth.draw_theta_batch(box, tt, wl.batch, synth.batch_seed(wid)).astype(np.float32)
    m = Model(ds.model_galaxy())
    m.tune(wl.batch, grad=True)                    # the launch shape bench.py times
    logL, grad = m.loglike_grad(torch.from_numpy(theta).cuda())
    grad = grad.cpu().numpy()
    pick = np.array([0, 255])
    ref_l, ref = oracle_grad(ds, theta[pick])
    import json
    import oracle
    from bang_testdata import grad_errors
    chi = -2.0 * (logL.cpu().numpy()[pick] + oracle.norm_const(ds.og))
    chi_ref = -2.0 * (ref_l + oracle.norm_const(ds.og))
    ge = grad_errors(grad[pick], ref)
    print(json.dumps({"workload": "adjoint", "rows": int(wl.batch), "rows_checked": pick.tolist(),
                      "max_rel_chi2": float((np.abs(chi - chi_ref) / chi_ref).max()),
                      "grad_err_over_norm": max(e[0] for e in ge), "grad_err_component_relative": max(e[1] for e in ge)}))
    assert (np.abs(chi - chi_ref) / chi_ref).max() < CHI2_RTOL
    assert_grad_close(grad[pick], ref, "full")
