"""Pins of the oracle's image losses of inverse rendering (Sec. IV.B): the
log-amplitude spectral loss of Eq. 8 and the low-pass misfit of the
coarse-to-fine solve, with their image gradients.

Each check compares the oracle with something other than itself: closed
forms (a scaled image, Parseval, the DC-only filter), an invariant (circular
shifts leave amplitude spectra unchanged), numpy's FFT as a library special
case, and central differences for the gradients."""
import numpy as np

import oracle


def images(seed, K=2, H=16, W=32):
    rng = np.random.default_rng(seed)
    return rng.random((K, H, W)) + 0.5


def test_spectral_loss_zero_for_identical_and_for_circular_shifts():
    t = images(0)
    assert oracle.spectral_loss(t, t)[0] == 0.0
    shifted = np.roll(t, shift=(3, -5), axis=(1, 2))
    v, g = oracle.spectral_loss(shifted, t)
    assert v < 1e-24
    assert np.abs(g).max() < 1e-10


def test_spectral_loss_of_a_scaled_image_is_log_scale_squared():
    """|F(c I)| = c |F(I)|, so every frequency contributes (log c)^2 when the
    guard eps is negligible against every amplitude."""
    t = images(1)
    amp = np.abs(np.fft.fft2(t))
    assert amp.min() > 1e-6 * amp.max()
    for c in (0.5, 1.7, 3.0):
        v, _ = oracle.spectral_loss(c * t, t, eps_rel=1e-12)
        assert abs(v - np.log(c) ** 2) < 1e-5 * max(1.0, np.log(c) ** 2)


def test_spectral_loss_matches_numpy_fft_on_a_small_case():
    t, x = images(2, K=1, H=8, W=8), images(3, K=1, H=8, W=8)
    bt, bx = np.abs(np.fft.fft2(t[0])), np.abs(np.fft.fft2(x[0]))
    e = 1e-3 * bt.max()
    want = np.mean((np.log(bx + e) - np.log(bt + e)) ** 2)
    assert abs(oracle.spectral_loss(x, t, eps_rel=1e-3)[0] - want) < 1e-13


def test_spectral_loss_gradient_matches_central_differences():
    t = images(4, K=2, H=8, W=16)
    x = t + 0.2 * images(5, K=2, H=8, W=16)
    v, g = oracle.spectral_loss(x, t, eps_rel=1e-4)
    h = 1e-6
    for idx in [(0, 0, 0), (0, 3, 7), (1, 7, 15), (1, 4, 2)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (oracle.spectral_loss(xp, t, eps_rel=1e-4)[0] -
              oracle.spectral_loss(xm, t, eps_rel=1e-4)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max())


def test_lowpass_misfit_passing_everything_is_the_pixel_misfit():
    """A cut-off beyond the grid's corner frequency keeps every frequency:
    by Parseval the misfit is scale * sum (I - T)^2 and its gradient
    2 scale (I - T)."""
    t, x = images(6), images(7)
    dx = 0.5
    v, g = oracle.lowpass_misfit(x, t, dx, cutoff=10.0, scale=0.3)
    assert abs(v - 0.3 * np.sum((x - t) ** 2)) < 1e-12 * v
    assert np.abs(g - 0.6 * (x - t)).max() < 1e-12


def test_lowpass_misfit_keeping_only_the_mean():
    """A cut-off below the first nonzero frequency keeps the DC term alone:
    L = scale (sum (I - T))^2 / (H W) per image, gradient 2 scale
    sum (I - T) / (H W) at every pixel of that image."""
    t, x = images(8), images(9)
    K, H, W = t.shape
    dx = 0.5
    cut = 0.5 / (max(H, W) * dx)
    v, g = oracle.lowpass_misfit(x, t, dx, cutoff=cut, scale=2.0)
    s = (x - t).sum(axis=(1, 2))
    assert abs(v - 2.0 * np.sum(s ** 2) / (H * W)) < 1e-12 * abs(v)
    for k in range(K):
        assert np.abs(g[k] - 4.0 * s[k] / (H * W)).max() < 1e-12


def test_lowpass_misfit_gradient_matches_central_differences():
    t, x = images(10), images(11)
    v, g = oracle.lowpass_misfit(x, t, 0.5, cutoff=0.35, scale=1.0)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 9, 30), (0, 15, 3)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (oracle.lowpass_misfit(xp, t, 0.5, 0.35)[0] - oracle.lowpass_misfit(xm, t, 0.5, 0.35)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max())
