"""Pins of the oracle's literal (incoherent) reading of Eq. 5: uniform
field, all-pass pupil (the sheared interferogram itself, by circular
shifts), energy conservation of the unit-sum PSF, and the defocus-sign
symmetry of an intensity PSF."""
import math

import numpy as np

import oracle


def opt(**kw):
    return oracle.make_optics(32, 32, **dict(dict(modes=4, NA=0.4, shear_px=2.0, shear_angle=0.0,
                                                  bias_phase=math.pi / 5), **kw))


def rand_field(seed, H=32, W=32):
    rng = np.random.default_rng(seed)
    return np.exp(-0.2 * rng.random((H, W))) * np.exp(1j * rng.uniform(-1, 1, (H, W)))


def interferogram(E, o):
    """|U(r + ds) e^{i theta} - U(r - ds) e^{-i theta}|^2 for a whole-pixel
    shear along x or y by circular shifts."""
    d = o["shear_px"] / 2
    assert d == int(d)
    ax = 1 if abs(math.cos(o["shear_angle"])) > 0.5 else 0
    s = int(round(d * (math.cos(o["shear_angle"]) if ax == 1 else math.sin(o["shear_angle"]))))
    th = o["bias_phase"]
    fwd = np.roll(E, -s, axis=ax)  # U(r + ds)
    bwd = np.roll(E, s, axis=ax)   # U(r - ds)
    return np.abs(fwd * np.exp(1j * th) - bwd * np.exp(-1j * th)) ** 2


def test_uniform_field_gives_the_bias_background():
    o = opt(defocus=1.3)
    out = oracle.dic_incoherent(o, np.ones((32, 32), dtype=complex))
    np.testing.assert_allclose(out, 4 * math.sin(o["bias_phase"]) ** 2, rtol=0, atol=1e-12)


def test_all_pass_pupil_leaves_the_interferogram():
    # NA 0.8 at dx 0.5, lambda 0.55 covers every DFT frequency; in focus the
    # PSF is a delta and I equals the sheared interferogram
    for angle in (0.0, math.pi / 2, math.pi):
        o = opt(NA=0.8, defocus=0.0, shear_angle=angle)
        E = rand_field(1)
        np.testing.assert_allclose(oracle.dic_incoherent(o, E), interferogram(E, o),
                                   rtol=0, atol=1e-11)


def test_unit_sum_psf_conserves_energy():
    o = opt(NA=0.35, defocus=0.9)
    E = rand_field(2)
    out = oracle.dic_incoherent(o, E)
    J = interferogram(E, o)
    assert abs(out.sum() - J.sum()) <= 1e-10 * J.sum()
    assert np.abs(out - J).max() > 1e-3  # the PSF does blur


def test_defocus_sign_does_not_change_the_intensity_psf():
    # P(-dz) = conj P(dz) gives |h_{-dz}(r)|^2 = |h_dz(-r)|^2, the same PSF
    # for a pupil symmetric under q -> -q (NA below the Nyquist row)
    E = rand_field(3)
    a = oracle.dic_incoherent(opt(NA=0.3, defocus=1.5), E)
    b = oracle.dic_incoherent(opt(NA=0.3, defocus=-1.5), E)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
    c = oracle.dic_incoherent(opt(NA=0.3, defocus=0.0), E)
    assert np.abs(a - c).max() > 1e-3
