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
