"""The learned warm start: trained on renders only, the network predicts the
optics far better than the training prior, and the inverse solve started
from its estimates reaches 1% median dn and T error in fewer steps than the
plain solve from the same perturbed guesses."""
import numpy as np
import pytest

from paper_2606_21381_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    from paper_2606_21381_gb300 import cnn
    from paper_2606_21381_gb300.render import Renderer
    r = Renderer(512, 512)
    net = cnn.WarmStartNet(torch.device("cuda"), seed=0)
    res = cnn.train(net, cnn.TrainConfig(samples=100_000), r)
    ev = cnn.calibrate(net, r)
    assert r.sync_status() == 0
    return net, r, res, ev


def test_training_reduces_the_loss(trained):
    _, _, res, _ = trained
    assert np.all(np.isfinite(res.losses))
    assert res.losses[-50:, 0].mean() < 0.5 * res.losses[:10, 0].mean()


def test_network_beats_the_prior_on_held_out_renders(trained):
    _, _, _, ev = trained
    for key in ("defocus", "NA", "shear"):
        assert ev[key] < 0.5 * ev[key + "_prior"], key
    assert ev["opd"] < 0.8 * ev["opd_prior"]
    assert ev["recall"] > 0.5 and ev["false_pos"] < 0.1


def test_warm_start_reaches_one_percent_in_fewer_steps(trained):
    from paper_2606_21381_gb300 import cnn, inverse
    net, _, _, _ = trained
    soa, o = scenes.inverse_512()
    o = dict(o, defocus=0.8, shear_px=1.0)
    r = inverse.Renderer(512, 512)
    target = r.render(torch.from_numpy(soa).cuda(), None, o)
    plain, warm = [], []
    for seed in (7, 9, 10):
        s0, o0 = inverse.perturb(soa, o, np.random.default_rng(seed))
        sw, ow = cnn.warm_start(net, target, s0, o0)
        # fixed particle properties and poses are the guess's
        assert np.array_equal(sw[[0, 1, 2, 3, 4, 7, 8]], s0[[0, 1, 2, 3, 4, 7, 8]])
        cfg = inverse.SolveConfig(steps=300, record_every=5)
        a = inverse.time_to_error(inverse.solve(target, s0, o0, r, cfg, truth=soa).history)
        b = inverse.time_to_error(inverse.solve(target, sw, ow, r, cfg, truth=soa).history)
        assert a is not None and b is not None
        plain.append(a[0])
        warm.append(b[0])
    assert sum(warm) < 0.85 * sum(plain), (plain, warm)


def test_graphed_training_follows_the_eager_loop():
    """The training step replayed as a CUDA graph (device-side step count,
    learning rate and bias corrections) takes the path of the eager loop:
    same renders, same losses up to float rounding, same weights."""
    from paper_2606_21381_gb300 import cnn
    from paper_2606_21381_gb300.render import Renderer
    r = Renderer(512, 512)
    out = {}
    for graph in (False, True):
        net = cnn.WarmStartNet(torch.device("cuda"), seed=3)
        res = cnn.train(net, cnn.TrainConfig(samples=64 * 12, graph=graph, seed=4), r)
        out[graph] = (res.losses, [w.clone() for w in net.w])
    assert r.sync_status() == 0 and cnn.sync_status() == 0
    la, lb = out[False][0], out[True][0]
    assert la.shape == lb.shape == (12, 4)
    assert np.allclose(la, lb, rtol=1e-2, atol=1e-5)
    # Adam steps a weight by about lr whatever its gradient's size, so a
    # rounding-level gradient can flip single entries: compare norms
    for wa, wb in zip(out[False][1], out[True][1]):
        assert float(torch.linalg.norm(wa - wb)) <= 2e-3 * float(torch.linalg.norm(wa)) + 1e-6
