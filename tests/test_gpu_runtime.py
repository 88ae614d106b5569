"""Runtime behaviour of the library: calls on a caller's stream, several host threads on one
model, CUDA-graph replay when the caller's buffers change, and several live models with one
destroyed in between.  Every result must equal the plain single-threaded call."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2205_06819_gb300 import synth  # noqa: E402

from bang_testdata import Dataset, theta_batch  # noqa: E402


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_06819_gb300 import build as b
    b.build()
    from paper_2205_06819_gb300.model import Model
    box = synth.prior_box(1)
    th = synth.draw_theta_true(box, 5)
    ds = Dataset(synth.GalaxySpec(24, 20, 3, 2.2), th, seed=6)
    return Model, ds, th


def test_caller_stream(env):
    Model, ds, th = env
    m = Model(ds.model_galaxy())
    theta = torch.from_numpy(theta_batch(1, th, 64, seed=7)).cuda()
    ref = m.loglike(theta).cpu().numpy()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        t2 = theta * 1.0                    # produced on the side stream
        out = m.loglike(t2)
        after = out * 2.0                   # consumed on the side stream
    s.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    np.testing.assert_array_equal(after.cpu().numpy(), 2.0 * ref)


def test_threads_share_a_model(env):
    Model, ds, th = env
    m = Model(ds.model_galaxy())
    thetas = [torch.from_numpy(theta_batch(1, th, 32 + 8 * k, seed=20 + k)).cuda() for k in range(4)]
    refs = [m.loglike(t).cpu().numpy() for t in thetas]
    grads = [m.loglike_grad(t)[1].cpu().numpy() for t in thetas]
    errors = []

    def work(k):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for _ in range(5):
                    got = m.loglike(thetas[k])
                    _, g = m.loglike_grad(thetas[k])
                    s.synchronize()
                    if not np.array_equal(got.cpu().numpy(), refs[k]):
                        errors.append((k, "logL"))
                    if not np.array_equal(g.cpu().numpy(), grads[k]):
                        errors.append((k, "grad"))
        except Exception as e:  # noqa: BLE001
            errors.append((k, repr(e)))

    ts = [threading.Thread(target=work, args=(k,)) for k in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors


def test_graph_replay_follows_the_callers_buffers(env):
    Model, ds, th = env
    m = Model(ds.model_galaxy())
    a = torch.from_numpy(theta_batch(1, th, 48, seed=31)).cuda()
    b = torch.from_numpy(theta_batch(1, th, 48, seed=32)).cuda()
    out1, out2 = torch.empty(48, dtype=torch.float64, device="cuda"), torch.empty(48, dtype=torch.float64, device="cuda")
    ra = m.loglike(a, out=out1).cpu().numpy().copy()
    rb = m.loglike(b, out=out2).cpu().numpy().copy()
    assert not np.array_equal(ra, rb)
    np.testing.assert_array_equal(m.loglike(a, out=out2).cpu().numpy(), ra)
    a.copy_(b)                              # same buffer, new values: the replay must see them
    np.testing.assert_array_equal(m.loglike(a, out=out1).cpu().numpy(), rb)


def test_several_models_and_destroy(env):
    Model, ds, th = env
    theta = torch.from_numpy(theta_batch(1, th, 40, seed=41)).cuda()
    m1 = Model(ds.model_galaxy())
    ref = m1.loglike(theta).cpu().numpy()
    m2 = Model(ds.model_galaxy(), bulge_table=1024)
    m3 = Model(ds.model_galaxy(), psf_mode=4)
    r3 = m3.loglike(theta).cpu().numpy()
    m2.loglike(theta)
    m2.close()
    np.testing.assert_array_equal(m1.loglike(theta).cpu().numpy(), ref)
    np.testing.assert_array_equal(m3.loglike(theta).cpu().numpy(), r3)
    m1.close()
    np.testing.assert_array_equal(m3.loglike(theta).cpu().numpy(), r3)
    m3.close()


def test_gradient_is_bitwise_reproducible(env):
    """Every adjoint work item writes its own partial sums, summed per row in item order: no
    atomics, so repeated calls give the same bits (what a checkpointed sampler relies on)."""
    Model, ds, th = env
    m = Model(ds.model_galaxy(), n_discs=1)
    t = torch.from_numpy(theta_batch(1, th, 96, seed=51)).cuda()
    l0, g0 = m.loglike_grad(t)
    for _ in range(4):
        l1, g1 = m.loglike_grad(t)
        assert torch.equal(l0, l1) and torch.equal(g0, g1)
