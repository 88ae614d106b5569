"""The float64 check path (bang_loglike_fp64) against the float64 oracle: the same discrete
model computed in float64 on both sides, so chi^2 agrees to near float64 rounding (bar
1e-11 relative; measured 1e-14) and not just to the float32 bar of the fused kernels
(1e-5).  Cases: the single-row workload (30x30, os 3, gamma = 1), two discs with a
Hernquist halo, a Moffat PSF and 128 nodes, the circular window with centre sampling,
masked spaxels; rows outside the domain; host and device buffers; unsupported options."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2205_06819_gb300 import synth  # noqa: E402

from bang_testdata import Dataset, theta_batch  # noqa: E402

FP64_RTOL = 1e-11


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2205_06819_gb300 import build as b
    oracle.build()
    b.build()
    from paper_2205_06819_gb300.model import Model
    return Model


def oracle_chi2(ds, theta64):
    import oracle
    _, chi2 = oracle.loglike(ds.og, theta64, n_discs=ds.n_discs, n_quad=ds.n_quad, halo_kind=ds.halo_kind)
    return chi2


def gpu_chi2(ds, logL):
    import oracle
    return -2.0 * (np.asarray(logL, dtype=np.float64) + oracle.norm_const(ds.og))


CASES = [
    # (spec, n_discs, n_quad, halo_kind, psf_mode, gamma_fixed, masked)
    (synth.GalaxySpec(30, 30, 3, 2.5), 1, 64, 0, 0, 1.0, False),
    (synth.GalaxySpec(16, 14, 3, 2.4, psf_kind=1, moffat_beta=3.0), 2, 128, 1, 0, None, False),
    (synth.GalaxySpec(18, 15, 3, 2.2), 1, 64, 0, 3, None, True),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fp64_path_matches_the_oracle(lib, case):
    spec, nd, nq, halo, psf_mode, gfix, masked = CASES[case]
    box = synth.prior_box(nd, gfix, halo)
    th = synth.draw_theta_true(box, 70 + case)
    mask = None
    if masked:
        mask = np.ones((4, spec.ny, spec.nx), np.uint8)
        mask[:, :3, :4] = 0
        mask[2, 7, :] = 0
    ds = Dataset(spec, th, n_discs=nd, n_quad=nq, seed=80 + case, halo_kind=halo, psf_mode=psf_mode, mask=mask)
    theta = theta_batch(nd, th, 4, seed=90 + case, gamma_fixed=gfix, halo_kind=halo).astype(np.float64)
    theta[0] = th                                     # the true parameters: chi^2 ~ N_spax
    m = lib(ds.model_galaxy(), n_discs=nd, n_quad=nq, halo_kind=halo, psf_mode=psf_mode)
    got = m.loglike_fp64(torch.from_numpy(theta).cuda()).cpu().numpy()
    ref = oracle_chi2(ds, theta)
    rel = np.abs(gpu_chi2(ds, got) - ref) / ref
    assert rel.max() < FP64_RTOL, rel
    # the float32 path agrees with both to its own bar
    got32 = m.loglike(torch.from_numpy(theta.astype(np.float32)).cuda()).cpu().numpy()
    ref32 = oracle_chi2(ds, theta.astype(np.float32).astype(np.float64))
    assert (np.abs(gpu_chi2(ds, got32) - ref32) / ref32).max() < 1e-5
    m.close()


def test_domain_buffers_and_options(lib):
    spec = synth.GalaxySpec(12, 10, 2, 2.0)
    box = synth.prior_box(1)
    th = synth.draw_theta_true(box, 5)
    ds = Dataset(spec, th, seed=6)
    theta = theta_batch(1, th, 3, seed=7).astype(np.float64)
    theta[1, 3] = 2.0                                 # inclination beyond pi/2: outside the domain
    m = lib(ds.model_galaxy())
    host = m.loglike_fp64(torch.from_numpy(theta))
    dev = m.loglike_fp64(torch.from_numpy(theta).cuda()).cpu()
    assert torch.equal(host, dev)
    assert host[1].item() == -np.inf and np.isfinite(host[[0, 2]].numpy()).all()
    ref = oracle_chi2(ds, theta[[0, 2]])
    assert (np.abs(gpu_chi2(ds, host[[0, 2]].numpy()) - ref) / ref).max() < FP64_RTOL
    with pytest.raises(ValueError):
        m.loglike_fp64(torch.from_numpy(theta.astype(np.float32)))
    m.close()
    for kw in ({"psf_mode": 4}, {"bulge_kind": 1}):
        m2 = lib(ds.model_galaxy(), **kw)
        with pytest.raises(Exception, match="UNSUPPORTED"):
            m2.loglike_fp64(torch.from_numpy(theta))
        m2.close()
