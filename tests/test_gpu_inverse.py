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
    # the particles outside the 1% set trade dn against T: the phase fixes the
    # product dn T, T alone is seen only through the absorption contrast mu T,
    # which is weakest for the smallest particles
    rel = lambda row: np.abs(res.soa[row] - soa[row]) / np.abs(soa[row])
    dnT = np.abs(res.soa[5] * res.soa[6] - soa[5] * soa[6]) / np.abs(soa[5] * soa[6])
    miss = (rel(6) > 0.01) | (rel(5) > 0.01)
    assert miss.any()
    assert np.median(dnT[miss]) < 0.5 * np.median(rel(6)[miss])
    size = soa[3] * soa[4]
    assert np.median(size[miss]) < np.median(size[~miss])


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
    assert float(inverse.spectral_loss(r.render(x1, None, o), target, r)) < \
        0.1 * float(inverse.spectral_loss(r.render(x0, None, o0), target, r))


def _scene_and_guess(seed):
    from paper_2606_21381_gb300 import inverse
    from paper_2606_21381_gb300.render import Renderer
    soa, o = scenes.inverse_512()
    o = dict(o, defocus=0.8, shear_px=1.0)
    r = Renderer(512, 512)
    target = r.render(torch.from_numpy(soa).cuda(), None, o)
    s0, o0 = inverse.perturb(soa, o, np.random.default_rng(seed))
    return soa, o, r, target, s0, o0


def test_graph_replays_equal_the_eager_device_steps():
    """The captured solve step replayed as a CUDA graph gives bit for bit
    what the same step launched eagerly gives."""
    from paper_2606_21381_gb300 import inverse
    soa, o, r, target, s0, o0 = _scene_and_guess(9)
    out = {}
    for mode in ("graph", "device"):
        res = inverse.solve(target, s0, o0, r, inverse.SolveConfig(steps=12, mode=mode))
        assert r.sync_status() == 0
        out[mode] = res
    assert np.array_equal(out["graph"].soa, out["device"].soa)
    assert np.array_equal(out["graph"].optics_params, out["device"].optics_params)
    assert out["graph"].losses == out["device"].losses
    assert out["graph"].losses[-1] < out["graph"].losses[0]


def test_autograd_loop_agrees_with_the_device_step():
    """The autograd loop (optics on the host, float64 Adam on them) and the
    device-resident step take the same path within float rounding."""
    from paper_2606_21381_gb300 import inverse
    soa, o, r, target, s0, o0 = _scene_and_guess(10)
    a = inverse.solve(target, s0, o0, r, inverse.SolveConfig(steps=30, mode="autograd"))
    d = inverse.solve(target, s0, o0, r, inverse.SolveConfig(steps=30, mode="graph"))
    assert r.sync_status() == 0
    # Adam moves a parameter whose gradient is near zero by about +-lr per
    # step whatever its size, so rounding can flip single particles' early
    # steps: compare medians over the particles and the losses
    for row in (0, 1, 2, 5, 6):
        moved = np.median(np.abs(a.soa[row] - s0[row]))
        diff = np.median(np.abs(a.soa[row] - d.soa[row]))
        assert diff <= 0.05 * moved + 1e-7, (row, diff, moved)
    assert np.allclose(a.optics_params, d.optics_params, rtol=1e-2, atol=1e-4)
    assert abs(a.losses[-1] - d.losses[-1]) <= 0.05 * a.losses[-1]
    assert abs(a.losses[0] - d.losses[0]) <= 1e-4 * a.losses[0]


def test_bound_optics_scalars_match_the_struct():
    """Defocus, shear and bias read from a bound device array give the images
    and gradients of the same values given in the optics struct."""
    from paper_2606_21381_gb300.autograd import OPTICS_PARAMS
    soa, o, r, target, s0, o0 = _scene_and_guess(11)
    x = torch.from_numpy(soa).cuda()
    want = dict(o, defocus=0.6, shear_px=1.3, shear_angle=0.5, bias_phase=0.9)
    gI = torch.randn((2, 512, 512), device="cuda")
    img_s = r.render(x, None, want)
    g_s = r.backward(x, None, want, gI)
    params = torch.tensor([want[k] for k in OPTICS_PARAMS], dtype=torch.float32, device="cuda")
    r.bind_optics_params(params)
    try:
        img_b = r.render(x, None, o)          # the struct's four scalars are ignored
        g_b = r.backward(x, None, o, gI)
        params[0] = 0.0                       # read when the kernels run
        img_0 = r.render(x, None, o)
    finally:
        r.bind_optics_params(None)
    img_0s = r.render(x, None, dict(want, defocus=0.0))
    assert r.sync_status() == 0
    scale = float(img_s.abs().max())
    assert float((img_b - img_s).abs().max()) <= 1e-5 * scale
    assert float((img_0 - img_0s).abs().max()) <= 1e-5 * scale
    assert float((img_0 - img_s).abs().max()) > 1e-3 * scale
    for a, b in zip(g_b, g_s):
        assert float((a - b).abs().max()) <= 1e-3 * float(b.abs().max())
    # unbound again: the struct's values apply
    assert torch.equal(r.render(x, None, want), img_s)


def test_graphed_solve_with_fixed_optics():
    """With the optics fixed the bound scalars never move, and the particles
    still converge (the guess's optics are the true ones here)."""
    from paper_2606_21381_gb300 import inverse
    soa, o, r, target, s0, _ = _scene_and_guess(12)
    res = inverse.solve(target, s0, o, r, inverse.SolveConfig(steps=200), fixed_optics=True)
    assert r.sync_status() == 0
    want = np.array([o[k] for k in ("defocus", "shear_px", "shear_angle", "bias_phase")])
    assert np.allclose(res.optics_params, want, rtol=0, atol=1e-6)
    assert res.losses[-1] < 1e-2 * res.losses[0]
    e = inverse.errors(res.soa, soa)
    assert e["dn_rel_median"] < 0.01


def test_resumed_solve_equals_an_uninterrupted_one(tmp_path):
    """A solve checkpointed halfway (saved to disk and loaded back) and
    resumed ends bitwise where the uninterrupted solve ends: the state holds
    everything the step carries (particles, optics scalars, Adam moments,
    the step counter that drives the curriculum, the losses)."""
    from paper_2606_21381_gb300 import inverse
    from paper_2606_21381_gb300.render import Renderer
    rng = np.random.default_rng(17)
    soa = scenes.draw_particles(rng, 40, 256, 256, mu=(0.005, 0.02))
    o = scenes.optics(256, 256, modes=5, defocus=0.6, NA=0.45)
    r = Renderer(256, 256)
    target = r.render(torch.from_numpy(soa).cuda(), None, o)
    s0, o0 = inverse.perturb(soa, o, rng)
    cfg = inverse.SolveConfig(steps=40, checkpoint_every=20)
    saved = []
    full = inverse.solve(target, s0, o0, r, cfg, on_checkpoint=saved.append)
    assert [s.step for s in saved] == [20, 40]
    path = str(tmp_path / "solve_state.pt")
    saved[0].save(path)
    resumed = inverse.solve(target, s0, o0, r, cfg, resume=inverse.SolveState.load(path))
    assert r.sync_status() == 0
    assert np.array_equal(full.soa, resumed.soa)
    assert np.array_equal(full.optics_params, resumed.optics_params)
    assert full.losses == resumed.losses
    assert not np.array_equal(full.soa, s0)  # the solve did move
