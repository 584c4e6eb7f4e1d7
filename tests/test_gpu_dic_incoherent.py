"""The literal (incoherent) reading of Eq. 5 through
osog_render_dic_incoherent against the FP64 oracle: square and non-square
canvases, defocus, an all-pass pupil, and the empty field."""
import math

import numpy as np
import pytest

import oracle
from paper_2606_21381_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-4  # of the empty-field background 4 sin^2(theta)


def _case(H, W, n, seed, **kw):
    rng = np.random.default_rng(seed)
    soa = scenes.draw_particles(rng, n, H, W, mu=(0.0, 0.02))
    o = scenes.optics(H, W, **dict(dict(modes=scenes.MODE_DIC, NA=0.5, shear_px=1.0), **kw))
    return soa, o


@pytest.mark.parametrize("H,W,n,kw", [
    (256, 256, 64, dict(defocus=0.7)),
    (128, 256, 40, dict(defocus=-1.2, shear_angle=0.3, bias_phase=1.1)),
    (256, 256, 64, dict(NA=0.8, defocus=0.0, shear_px=2.0, shear_angle=0.0)),
])
def test_matches_the_oracle(H, W, n, kw):
    from paper_2606_21381_gb300.render import Renderer
    soa, o = _case(H, W, n, 31 + H + n, **kw)
    want = oracle.render_dic_incoherent(soa, n, o)
    r = Renderer(H, W)
    got = r.render_dic_incoherent(torch.from_numpy(soa).cuda(), None, o).cpu().numpy()
    assert r.sync_status() == 0
    bg = 4 * math.sin(o["bias_phase"]) ** 2
    assert np.abs(want - bg).max() > 0.05 * bg  # contrast
    assert np.abs(got - want).max() <= TOL * bg


def test_empty_field_is_the_bias_background():
    from paper_2606_21381_gb300.render import Renderer
    r = Renderer(128, 128)
    o = scenes.optics(128, 128, modes=scenes.MODE_DIC, NA=0.45, defocus=1.0)
    img = r.render_dic_incoherent(torch.zeros((9, 1), device="cuda"), 0, o).cpu().numpy()
    assert r.sync_status() == 0
    np.testing.assert_allclose(img, 4 * math.sin(o["bias_phase"]) ** 2, rtol=0, atol=1e-5)


def test_bound_optics_scalars_in_the_incoherent_dic():
    """The incoherent DIC reads defocus, shear and bias from a bound device
    array like every other entry point of the plan."""
    from paper_2606_21381_gb300.autograd import OPTICS_PARAMS
    from paper_2606_21381_gb300.render import Renderer
    r = Renderer(128, 128)
    rng = np.random.default_rng(21)
    soa = scenes.draw_particles(rng, 20, 128, 128, mu=(0.0, 0.02))
    x = torch.from_numpy(np.ascontiguousarray(soa)).cuda()
    base = scenes.optics(128, 128, modes=4, NA=0.5)
    want = dict(base, defocus=0.4, shear_px=1.2, shear_angle=0.7, bias_phase=0.6)
    ref = r.render_dic_incoherent(x, None, want)
    params = torch.tensor([want[k] for k in OPTICS_PARAMS], dtype=torch.float32, device="cuda")
    r.bind_optics_params(params)
    try:
        got = r.render_dic_incoherent(x, None, base)
    finally:
        r.bind_optics_params(None)
    assert r.sync_status() == 0
    scale = float(ref.abs().max())
    assert float((got - ref).abs().max()) <= 1e-5 * scale
