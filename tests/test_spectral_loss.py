"""The spectral loss of Eq. 8 (log-amplitude FFT misfit) on the CPU: zero
for identical images and for circular shifts, positive otherwise, and its
autograd gradient matches central differences."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_21381_gb300.inverse import spectral_loss  # noqa: E402


def test_zero_for_shifts_positive_otherwise():
    g = torch.Generator().manual_seed(0)
    a = torch.rand((2, 32, 48), generator=g, dtype=torch.float64) + 0.5
    assert float(spectral_loss(a, a)) == 0.0
    shifted = torch.roll(a, shifts=(5, -7), dims=(1, 2))
    assert float(spectral_loss(a, shifted)) < 1e-20
    blurred = 0.5 * (a + torch.roll(a, 1, dims=2))
    assert float(spectral_loss(a, blurred)) > 1e-3


def test_gradient_matches_central_differences():
    g = torch.Generator().manual_seed(1)
    t = torch.rand((1, 16, 16), generator=g, dtype=torch.float64) + 0.5
    x = (t + 0.1 * torch.rand((1, 16, 16), generator=g, dtype=torch.float64)).requires_grad_(True)
    (gx,) = torch.autograd.grad(spectral_loss(x, t), x)
    h = 1e-6
    for idx in [(0, 0, 0), (0, 3, 7), (0, 15, 9)]:
        xp, xm = x.detach().clone(), x.detach().clone()
        xp[idx] += h
        xm[idx] -= h
        fd = (float(spectral_loss(xp, t)) - float(spectral_loss(xm, t))) / (2 * h)
        assert abs(fd - float(gx[idx])) <= 1e-6 * max(1.0, abs(fd))


def test_frequency_domain_misfit_equals_the_filtered_one():
    # the solve's curriculum misfit, evaluated by Parseval on the rfft
    # half-plane, equals the spatial sum of squared low-passed differences
    from paper_2606_21381_gb300.inverse import SpectralMisfit, filtered, lowpass_mask
    g = torch.Generator().manual_seed(3)
    for H, W in ((32, 48), (64, 64), (16, 30)):
        t = torch.rand((2, H, W), generator=g, dtype=torch.float64)
        x = t + 0.3 * torch.rand((2, H, W), generator=g, dtype=torch.float64)
        norm = float(t.numel())
        mis = SpectralMisfit(t, 0.5, norm)
        for na in (0.1, 0.25, 0.4):
            mask = lowpass_mask(H, W, 0.5, 0.55, na, "cpu").double()
            want = ((filtered(x, mask) - filtered(t, mask)) ** 2).sum() / norm
            got = mis(x, 2.0 * na / 0.55)
            assert abs(float(got) - float(want)) <= 1e-9 * max(1e-12, float(want)), (H, W, na)
