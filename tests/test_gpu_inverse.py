"""Inverse rendering on the 512^2 scene (200 particles, brightfield + DIC):
recover dn, thickness, centres, angles, defocus and shear from guesses
perturbed by 20%, with the adjoint and the NA curriculum."""
import numpy as np
import pytest

from paper_2606_21381_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_inverse_solve_recovers_parameters():
    from paper_2606_21381_gb300 import inverse
    from paper_2606_21381_gb300.render import Renderer
    soa, o = scenes.inverse_512()
    o = dict(o, defocus=0.8, shear_px=1.0)
    r = Renderer(512, 512)
    target = r.render(torch.from_numpy(soa).cuda(), None, o)
    s0, o0 = inverse.perturb(soa, o, np.random.default_rng(7))
    e0 = inverse.errors(s0, soa, [o0["defocus"], o0["shear_px"]], o)
    res = inverse.solve(target, s0, o0, r, inverse.SolveConfig(steps=400))
    assert r.sync_status() == 0
    e = inverse.errors(res.soa, soa, res.optics_params, o)
    assert e0["dn_rel_median"] > 0.05 and e0["centre_px_median"] > 0.3
    assert e["dn_rel_median"] < 0.005 and e["T_rel_median"] < 0.005
    assert e["frac_dn_T_within_1pct"] > 0.8
    assert e["centre_px_median"] < 0.02 and e["theta_rad_median"] < 0.01
    assert e["defocus_abs"] < 0.02 and e["shear_rel"] < 0.01
    assert res.losses[-1] < 1e-2 * res.losses[0]
    # fixed particles (a, b, mu, kind) are untouched
    assert np.array_equal(res.soa[[3, 4, 7, 8]], s0[[3, 4, 7, 8]])


def test_solve_with_the_spectral_loss_term():
    # Eq. 8's log-amplitude term added to the misfit: the solve still
    # recovers the particles (the term is shift-invariant, so it only helps
    # alongside the pixel misfit)
    from paper_2606_21381_gb300 import inverse
    from paper_2606_21381_gb300.render import Renderer
    soa, o = scenes.inverse_512()
    o = dict(o, defocus=0.8, shear_px=1.0)
    r = Renderer(512, 512)
    target = r.render(torch.from_numpy(soa).cuda(), None, o)
    s0, o0 = inverse.perturb(soa, o, np.random.default_rng(8))
    res = inverse.solve(target, s0, o0, r, inverse.SolveConfig(steps=300, spectral_weight=1e-5))
    e = inverse.errors(res.soa, soa, res.optics_params, o)
    assert e["dn_rel_median"] < 0.01 and e["T_rel_median"] < 0.01
    assert res.losses[-1] < 1e-2 * res.losses[0]
    x0 = torch.from_numpy(s0).cuda()
    x1 = torch.from_numpy(res.soa).cuda()
    assert float(inverse.spectral_loss(r.render(x1, None, o), target)) < \
        0.1 * float(inverse.spectral_loss(r.render(x0, None, o0), target))
