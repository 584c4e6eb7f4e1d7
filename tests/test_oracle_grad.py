"""Pins of the oracle's analytic adjoint against central finite differences
of the oracle's forward model, for every particle field, both particle
kinds, all three modalities and the optics scalars."""
import math

import numpy as np
import pytest

import oracle
from paper_2606_21381_gb300 import scenes

OPT_KEYS = ("defocus", "shear_px", "shear_angle", "bias_phase")


def loss(soa, n, o, w):
    return float(np.sum(w * oracle.render(soa, n, o)["images"]))


def fd_field(soa, n, o, w, f, p, h):
    """Central difference in field f of particle p; the step is taken
    between two float32 values so the particle tensor stays exact."""
    x = float(soa[f, p])
    xp, xm = np.float32(x + h), np.float32(x - h)
    a, b = soa.copy(), soa.copy()
    a[f, p], b[f, p] = xp, xm
    return (loss(a, n, o, w) - loss(b, n, o, w)) / (float(xp) - float(xm))


def scene(seed, kinds):
    rng = np.random.default_rng(seed)
    n = len(kinds)
    soa = scenes.draw_particles(rng, n, 64, 64, mu=(0.005, 0.03), size_scale=1.3)
    soa[8] = kinds
    soa[0] = rng.uniform(14, 50, n)
    soa[1] = rng.uniform(14, 50, n)
    return soa


@pytest.mark.parametrize("modes", [1, 2, 4])
def test_particle_gradient_matches_central_differences(modes):
    soa = scene(7 + modes, [0, 1, 0, 1])
    n = soa.shape[1]
    o = oracle.make_optics(64, 64, modes=modes, defocus=0.9, NA=0.5, shear_angle=0.6)
    rng = np.random.default_rng(modes)
    w = rng.standard_normal((1, 64, 64))
    g, _ = oracle.render_grad(soa, n, o, w)
    assert np.all(g[8] == 0.0)
    # small steps: prisms are piecewise linear, and a step that straddles a
    # kink (plateau edge, wall diagonal) of one pixel would bias the difference
    steps = {0: 1e-4, 1: 1e-4, 2: 1e-5, 3: 1e-4, 4: 1e-4, 5: 1e-5, 6: 2e-5, 7: 2e-5}
    for p in range(n):
        for f, h in steps.items():
            fd = fd_field(soa, n, o, w, f, p, h)
            scale = max(np.abs(g[f]).max(), 1e-12)
            assert abs(g[f, p] - fd) <= 2e-3 * scale + 1e-3 * abs(fd), (p, f, g[f, p], fd)


def test_optics_gradient_matches_central_differences():
    soa = scene(3, [0, 1, 1])
    o = oracle.make_optics(64, 64, modes=7, defocus=0.7, NA=0.5, shear_px=1.3,
                           shear_angle=0.4, bias_phase=0.9)
    rng = np.random.default_rng(5)
    w = rng.standard_normal((3, 64, 64))
    _, gopt = oracle.render_grad(soa, 3, o, w)
    for k, key in enumerate(OPT_KEYS):
        h = 1e-5
        a, b = dict(o), dict(o)
        a[key] += h
        b[key] -= h
        fd = (loss(soa, 3, a, w) - loss(soa, 3, b, w)) / (2 * h)
        assert abs(gopt[k] - fd) <= 1e-5 * max(1.0, abs(fd)), (key, gopt[k], fd)
    assert abs(gopt[0]) > 1e-3 and abs(gopt[2]) > 1e-4


def test_gradient_of_background_only_loss_is_zero_without_particles():
    o = oracle.make_optics(32, 32, modes=1)
    g, gopt = oracle.render_grad(np.zeros((9, 1), np.float32), 0, o, np.ones((1, 32, 32)))
    assert g.shape == (9, 0)
    assert abs(gopt[0]) < 1e-9  # a uniform field is unchanged by defocus
