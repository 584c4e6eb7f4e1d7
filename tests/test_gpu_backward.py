"""GPU adjoint (osog_render_backward, through the C ABI) against the FP64
oracle adjoint, plus central differences of the GPU forward.

Bar: relative error <= 1e-3 per parameter, with a floor of 1e-3 of the
largest gradient of the same field (the same group of parameters).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_21381_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("cx", "cy", "theta", "a", "b", "T", "dn", "mu")
_renderers = {}


def renderer(H, W):
    from paper_2606_21381_gb300.render import Renderer
    if (H, W) not in _renderers:
        _renderers[(H, W)] = Renderer(H, W)
    return _renderers[(H, W)]


def gpu_grad(soa, o, gI):
    r = renderer(o["H"], o["W"])
    gs, go = r.backward(torch.from_numpy(np.ascontiguousarray(soa)).cuda(), None, o,
                        torch.from_numpy(np.ascontiguousarray(gI, dtype=np.float32)).cuda())
    assert r.sync_status() == 0
    return gs.cpu().numpy().astype(np.float64), go.cpu().numpy().astype(np.float64)


def assert_grads_close(g, ref, tol=1e-3):
    for f, name in enumerate(FIELDS):
        scale = np.abs(ref[f]).max()
        if scale == 0.0:
            assert np.abs(g[f]).max() == 0.0, name
            continue
        err = np.abs(g[f] - ref[f])
        bound = tol * np.maximum(np.abs(ref[f]), scale)
        bad = np.nonzero(err > bound)[0]
        assert bad.size == 0, (name, bad[:5], g[f, bad[:5]], ref[f, bad[:5]])
    assert np.all(g[8] == 0.0)


def assert_optics_close(go, ref, modes, tol=1e-3):
    n = 4 if modes & 4 else 1
    for k in range(n):
        assert abs(go[k] - ref[k]) <= tol * max(abs(ref[k]), 1e-3 * np.abs(ref[:n]).max()), \
            (k, go[k], ref[k])
    for k in range(n, 4):
        assert go[k] == 0.0


@pytest.mark.parametrize("H,W,modes", [(128, 128, 7), (64, 256, 3), (256, 64, 4)])
def test_backward_matches_oracle_adjoint(H, W, modes):
    rng = np.random.default_rng(H + W + modes)
    n = 40
    soa = scenes.draw_particles(rng, n, H, W, mu=(0.002, 0.03), size_scale=1.2)
    o = scenes.optics(H, W, modes=modes, defocus=0.8, NA=0.5, shear_angle=0.5,
                      shear_px=1.2, bias_phase=0.7)
    K = bin(modes).count("1")
    gI = rng.standard_normal((K, H, W))
    ref, ref_o = oracle.render_grad(soa, n, oracle.make_optics(**o), gI)
    g, go = gpu_grad(soa, o, gI.astype(np.float32).astype(np.float64))
    assert_grads_close(g, ref)
    assert_optics_close(go, ref_o, modes)


def test_backward_inverse_workload_512():
    """The inverse-rendering scene: 512^2, 200 particles, brightfield + DIC."""
    soa, o = scenes.inverse_512()
    n = soa.shape[1]
    rng = np.random.default_rng(11)
    gI = rng.standard_normal((2, 512, 512)).astype(np.float32).astype(np.float64)
    ref, ref_o = oracle.render_grad(soa, n, oracle.make_optics(**o), gI)
    g, go = gpu_grad(soa, o, gI)
    assert_grads_close(g, ref)
    assert_optics_close(go, ref_o, o["modes"])


def test_backward_is_bitwise_deterministic_and_skips_invalid_particles():
    soa, o = scenes.inverse_512()
    soa = soa.copy()
    soa[5, 17] = np.nan  # an invalid particle: skipped, zero gradient
    rng = np.random.default_rng(2)
    gI = rng.standard_normal((2, 512, 512)).astype(np.float32)
    r = renderer(512, 512)
    dev = torch.from_numpy(soa).cuda()
    a = r.backward(dev, None, o, torch.from_numpy(gI).cuda())
    assert r.sync_status() == 5
    b = r.backward(dev, None, o, torch.from_numpy(gI).cuda())
    r.sync_status()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert torch.all(a[0][:, 17] == 0)


def test_autograd_function_uses_the_adjoint():
    from paper_2606_21381_gb300.autograd import render
    soa, o = scenes.inverse_512(n=50)
    r = renderer(512, 512)
    x = torch.from_numpy(soa).cuda().requires_grad_(True)
    p = torch.tensor([0.3, 1.0, math.pi / 4, math.pi / 4], dtype=torch.float64, requires_grad=True)
    img = render(x, o, r, p)
    w = torch.randn_like(img)
    (img * w).sum().backward()
    o2 = dict(o, defocus=0.3)
    gs, go = r.backward(x.detach(), None, o2, w.contiguous())
    assert torch.equal(x.grad, gs)
    assert torch.allclose(p.grad, go.double().cpu())


def test_central_differences_of_gpu_forward_on_one_percent_of_parameters():
    """1% of the unknowns of the inverse problem plus the optics scalars:
    GPU adjoint vs central differences of the GPU forward.

    Float32 FFT rounding changes at every output pixel whenever any input
    changes, so the loss weights are confined to windows around the probed
    particles (the difference noise then scales with the window area, not the
    canvas).  The image is smooth in dn and mu, in an ellipsoid's T (its
    profile scales with T; a prism's plateau edge moves with T) and in the
    optics scalars, so those are probed.  Centre and angle move the footprint
    edge, where an ellipsoid's sqrt profile has unbounded slope: any step that
    float32 resolves lets a pixel centre cross the rim, so those are checked
    against the FP64 oracle adjoint instead (itself pinned by FP64 central
    differences with tiny steps)."""
    soa, o = scenes.inverse_512()
    n = soa.shape[1]
    r = renderer(512, 512)
    rng = np.random.default_rng(4)
    ell = np.nonzero(soa[8] == 0)[0]
    picks = [(5, int(p)) for p in rng.choice(ell, 4, replace=False)]
    picks += [(int(f), int(p)) for f, p in zip(rng.choice([6, 7], 6), rng.integers(0, n, 6))]
    wnp = np.zeros((2, 512, 512), np.float32)
    for _, p in picks:
        x0, y0 = int(soa[0, p]), int(soa[1, p])
        ys, xs = slice(max(y0 - 24, 0), y0 + 24), slice(max(x0 - 24, 0), x0 + 24)
        wnp[:, ys, xs] = rng.standard_normal(wnp[:, ys, xs].shape)
    w = torch.from_numpy(wnp).cuda()

    def loss(s_np, oo):
        img = r.render(torch.from_numpy(s_np).cuda(), None, oo)
        return float((img.double() * w.double()).sum())

    g, go = gpu_grad(soa, o, wnp.astype(np.float64))
    steps = {5: 2e-2, 6: 2e-3, 7: 2e-3}
    for f, p in picks:
        a, b = soa.copy(), soa.copy()
        a[f, p] += steps[f]
        b[f, p] -= steps[f]
        fd = (loss(a, o) - loss(b, o)) / (float(a[f, p]) - float(b[f, p]))
        assert abs(g[f, p] - fd) <= 2e-2 * max(abs(fd), 0.02 * np.abs(g[f]).max()), (f, p, g[f, p], fd)
    for k, key in enumerate(("defocus", "shear_px", "shear_angle", "bias_phase")):
        h = 1e-2
        a, b = dict(o), dict(o)
        a[key] += h
        b[key] -= h
        fd = (loss(soa, a) - loss(soa, b)) / (2 * h)
        assert abs(go[k] - fd) <= 2e-2 * max(abs(fd), 0.02 * np.abs(go).max()), (key, go[k], fd)


def _inverse_scene():
    soa, o = scenes.inverse_512()
    x = torch.from_numpy(soa).cuda()
    gI = torch.from_numpy(np.random.default_rng(3).standard_normal((2, 512, 512))
                          .astype(np.float32)).cuda()
    return x, o, gI


def test_kept_forward_state_gives_the_same_image_and_gradients():
    """osog_render_keep + osog_render_backward_kept reproduce osog_render and
    osog_render_backward bit for bit (the same kernels on the same state)."""
    r = renderer(512, 512)
    x, o, gI = _inverse_scene()
    img = r.render(x, None, o)
    img_k, ws = r.render_keep(x, None, o)
    g_k = r.backward_kept(x, None, o, gI, ws)
    g = r.backward(x, None, o, gI)
    assert r.sync_status() == 0
    assert torch.equal(img, img_k)
    assert torch.equal(g[0], g_k[0]) and torch.equal(g[1], g_k[1])
    # and on a canvas of another size, with a ragged particle count (n < ld)
    r2 = renderer(128, 128)
    rng = np.random.default_rng(4)
    soa = scenes.draw_particles(rng, 37, 128, 128, mu=(0.002, 0.03))
    o2 = scenes.optics(128, 128, modes=7, defocus=0.8, NA=0.5, shear_px=1.2)
    x2 = torch.from_numpy(np.ascontiguousarray(soa)).cuda()
    gI2 = torch.randn((3, 128, 128), device="cuda")
    img_k, ws = r2.render_keep(x2, 30, o2)
    g_k = r2.backward_kept(x2, 30, o2, gI2, ws)
    g = r2.backward(x2, 30, o2, gI2)
    assert r2.sync_status() == 0
    assert torch.equal(r2.render(x2, 30, o2), img_k)
    assert torch.equal(g[0], g_k[0]) and torch.equal(g[1], g_k[1])
    assert torch.all(g_k[0][:, 30:] == 0)


def test_kept_state_is_checked_and_consumed():
    import ctypes
    from paper_2606_21381_gb300._lib import OsogError, optics_struct
    r = renderer(512, 512)
    x, o, gI = _inverse_scene()
    _, ws = r.render_keep(x, None, o)
    with pytest.raises(OsogError):  # other optics than the kept forward's
        r.backward_kept(x, None, dict(o, defocus=o["defocus"] + 0.1), gI, ws)
    with pytest.raises(OsogError):  # another particle count
        r.backward_kept(x, x.shape[1] - 1, o, gI, ws)
    with pytest.raises(OsogError):  # another workspace
        r.backward_kept(x, None, o, gI, torch.empty_like(ws))
    r.backward_kept(x, None, o, gI, ws)
    with pytest.raises(OsogError):  # the adjoint consumed the state
        r.backward_kept(x, None, o, gI, ws)
    # another call writing the same workspace drops the state
    _, ws = r.render_keep(x, None, o, ws=ws)
    img = torch.empty((2, 512, 512), device="cuda")
    oo = optics_struct(o)
    assert r._L.osog_render(r.plan, ctypes.c_void_p(x.data_ptr()), x.shape[1], x.shape[1],
                            ctypes.byref(oo), ctypes.c_void_p(img.data_ptr()),
                            ctypes.c_void_p(ws.data_ptr()), ws.numel(), None) == 0
    with pytest.raises(OsogError):
        r.backward_kept(x, None, o, gI, ws)
    assert r.sync_status() == 0


def test_kept_state_on_a_non_square_canvas_with_three_modalities():
    r = renderer(64, 256)
    rng = np.random.default_rng(12)
    soa = scenes.draw_particles(rng, 25, 64, 256, mu=(0.002, 0.03))
    o = scenes.optics(64, 256, modes=7, defocus=-0.6, NA=0.5, shear_px=0.8, bias_phase=0.4)
    x = torch.from_numpy(np.ascontiguousarray(soa)).cuda()
    gI = torch.randn((3, 64, 256), device="cuda")
    img_k, ws = r.render_keep(x, None, o)
    g_k = r.backward_kept(x, None, o, gI, ws)
    g = r.backward(x, None, o, gI)
    assert r.sync_status() == 0
    assert torch.equal(r.render(x, None, o), img_k)
    assert torch.equal(g[0], g_k[0]) and torch.equal(g[1], g_k[1])


def test_more_live_differentiable_renders_than_the_plan_remembers():
    """A loss over 65 differentiable renders of one renderer: the plan keeps
    the forward states of its last 64 workspaces, so the oldest render's
    adjoint finds its state dropped and recomputes the forward.  Every
    gradient equals the one osog_render_backward gives for that render."""
    from paper_2606_21381_gb300.autograd import render
    r = renderer(128, 128)
    rng = np.random.default_rng(31)
    soa = scenes.draw_particles(rng, 20, 128, 128, mu=(0.002, 0.02))
    o = scenes.optics(128, 128, modes=1, defocus=0.4)
    base = torch.from_numpy(np.ascontiguousarray(soa)).cuda()
    xs = [(base + 0.01 * i * (torch.arange(9, device="cuda") < 2).float()[:, None])
          .requires_grad_(True) for i in range(65)]
    ws = [torch.randn((1, 128, 128), device="cuda") for _ in range(65)]
    loss = sum((render(x, o, r) * w).sum() for x, w in zip(xs, ws))
    loss.backward()
    assert r.sync_status() == 0
    for x, w in zip(xs, ws):
        gs, _ = r.backward(x.detach(), None, o, w)
        assert torch.equal(x.grad, gs)
