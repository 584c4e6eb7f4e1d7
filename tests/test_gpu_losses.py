"""The image losses of inverse rendering on the GPU (osog_loss_target +
osog_image_loss, through the C ABI) against the FP64 oracle: the low-pass
misfit of the coarse-to-fine solve and the log-amplitude spectral loss of
Eq. 8, values and image gradients, within 1e-3 relative."""
import numpy as np
import pytest

import oracle
from paper_2606_21381_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS_REL = 1e-4  # float32 spectra carry ~1e-7 of their largest amplitude as noise
TOL = 1e-3


def renders(H, W, modes, seed):
    """A rendered target and a render of the same scene with perturbed
    particles (the two images an inverse-rendering step compares)."""
    from paper_2606_21381_gb300.render import Renderer
    rng = np.random.default_rng(seed)
    soa = scenes.draw_particles(rng, 40, H, W, mu=(0.002, 0.02))
    o = scenes.optics(H, W, modes=modes, defocus=0.6)
    r = Renderer(H, W)
    t = r.render(torch.from_numpy(soa).cuda(), None, o)
    soa2 = soa.copy()
    soa2[6] *= 1.15
    soa2[0] += 0.4
    x = r.render(torch.from_numpy(soa2).cuda(), None, o)
    return r, x.contiguous(), t.contiguous(), o


def assert_close(got, want, what):
    assert abs(got - want) <= TOL * abs(want), (what, got, want)


@pytest.mark.parametrize("H,W,modes,cut", [(128, 256, 5, 0.45), (256, 256, 2, 1.3),
                                           (64, 128, 7, 0.2)])
def test_losses_and_gradients_match_the_oracle(H, W, modes, cut):
    r, x, t, o = renders(H, W, modes, seed=H + modes)
    table = r.loss_target(t)
    cutoff = torch.tensor([cut], dtype=torch.float32, device="cuda")
    K = x.shape[0]
    scale = 1.0 / x.numel()
    for sw in (0.0, 0.7):
        loss, grad = r.image_loss(x, table, o["dx"], cutoff, misfit_scale=scale,
                                  spectral_weight=sw, eps_rel=EPS_REL)
        assert r.sync_status() == 0
        xd, td = x.double().cpu().numpy(), t.double().cpu().numpy()
        m, gm = oracle.lowpass_misfit(xd, td, o["dx"], cut, scale)
        sp, gs = oracle.spectral_loss(xd, td, EPS_REL)
        loss = loss.cpu().numpy()
        assert_close(loss[0], m, "misfit")
        if sw:
            assert_close(loss[1], sp, "spectral")
        else:
            assert loss[1] == 0.0
        want = gm + sw * gs
        err = np.abs(grad.double().cpu().numpy() - want).max()
        assert err <= TOL * np.abs(want).max(), (sw, err, np.abs(want).max())
    assert K == bin(modes).count("1")


def test_cutoff_is_read_on_the_device_and_results_are_bitwise_repeatable():
    r, x, t, o = renders(128, 128, 1, seed=3)
    table = r.loss_target(t)
    cutoff = torch.tensor([0.3], dtype=torch.float32, device="cuda")
    a, ga = r.image_loss(x, table, o["dx"], cutoff, misfit_scale=1.0, spectral_weight=0.2,
                         eps_rel=EPS_REL)
    a, ga = a.clone(), ga.clone()
    b, gb = r.image_loss(x, table, o["dx"], cutoff, misfit_scale=1.0, spectral_weight=0.2,
                         eps_rel=EPS_REL)
    assert torch.equal(a, b) and torch.equal(ga, gb)
    cutoff.fill_(0.9)  # a device-side update, no new host argument
    c, _ = r.image_loss(x, table, o["dx"], cutoff, misfit_scale=1.0, spectral_weight=0.2,
                        eps_rel=EPS_REL)
    xd, td = x.double().cpu().numpy(), t.double().cpu().numpy()
    assert_close(float(c[0]), oracle.lowpass_misfit(xd, td, o["dx"], 0.9, 1.0)[0], "misfit")
    assert float(c[0]) > float(a[0])
    assert r.sync_status() == 0


def test_identical_images_give_zero_losses():
    r, x, t, o = renders(64, 64, 3, seed=5)
    table = r.loss_target(t)
    cutoff = torch.tensor([0.5], dtype=torch.float32, device="cuda")
    loss, grad = r.image_loss(t, table, o["dx"], cutoff, misfit_scale=1.0, spectral_weight=1.0,
                              eps_rel=EPS_REL)
    assert float(loss[0]) <= 1e-10 and float(loss[1]) <= 1e-10
    assert float(grad.abs().max()) <= 1e-6
