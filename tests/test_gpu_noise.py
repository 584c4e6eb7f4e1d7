"""osog_sensor_noise against the FP64 oracle (same Philox streams, same
Poisson decisions), reproducibility independent of the launch, in-place
use and argument checks."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _img(n, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 2.0, n).astype(np.float32)
    x[::97] = -0.1  # clipped to zero photons
    x[::89] = 0.0
    return x


@pytest.mark.parametrize("g,sigma", [(0.5, 0.0), (20.0, 3.0), (5000.0, 2.0), (3e6, 40.0)])
def test_matches_the_oracle(g, sigma):
    from paper_2606_21381_gb300.noise import sensor_noise
    x = _img(512 * 512)
    want = oracle.sensor_noise(x, g, sigma, 12345)
    got = sensor_noise(torch.from_numpy(x).cuda(), g, sigma, 12345).cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=2e-7, atol=1e-9)


def test_draw_depends_only_on_seed_and_index():
    from paper_2606_21381_gb300.noise import sensor_noise
    x = torch.from_numpy(_img(3 * 2048 * 2048 + 17, 1)).cuda()
    a = sensor_noise(x, 1000.0, 1.5, 7)
    b = sensor_noise(x, 1000.0, 1.5, 7)
    assert torch.equal(a, b)
    part = sensor_noise(x[:100_003].contiguous(), 1000.0, 1.5, 7)
    assert torch.equal(part, a[:100_003])
    assert not torch.equal(sensor_noise(x, 1000.0, 1.5, 8), a)
    idx = np.array([0, 5, 12_582_911, 12_582_928])
    xs = x.cpu().numpy()
    for i in idx:
        lam = 1000.0 * max(float(xs[i]), 0.0)
        want = (oracle.poisson(lam, 7, int(i)) + 1.5 * oracle.normal(7, int(i))) / 1000.0
        assert abs(float(a[i]) - want) <= 2e-7 * abs(want) + 1e-9


def test_in_place_and_argument_checks():
    from paper_2606_21381_gb300._lib import OsogError
    from paper_2606_21381_gb300.noise import sensor_noise
    x = torch.from_numpy(_img(10_000, 2)).cuda()
    want = sensor_noise(x, 50.0, 1.0, 3)
    y = x.clone()
    sensor_noise(y, 50.0, 1.0, 3, out=y)
    assert torch.equal(y, want)
    for g, s in ((0.0, 1.0), (-1.0, 1.0), (10.0, -1.0), (10.0, float("nan"))):
        with pytest.raises(OsogError):
            sensor_noise(x, g, s, 3)
