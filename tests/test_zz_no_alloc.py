"""osog_render_noalloc: the render for callers that cannot allocate device
memory (no plan, no workspace; scratch in the library's static device
arrays).  Its images must match osog_render's within the parity tolerance
on consecutive calls that reuse the same static scratch.

This file is collected last on purpose: it must pass in a fresh process
(where its first call performs the per-device set-up) as well as after
every other test.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2606_21381_gb300 import _lib, scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

I_TOL = 2e-4  # of the mean background intensity, as in the parity tests


def background(optics):
    return [4 * math.sin(optics["bias_phase"]) ** 2 if bit == 4 else 1.0
            for bit in (1, 2, 4) if optics["modes"] & bit]


def noalloc(soa_dev, optics, K):
    L = _lib.lib()
    out = torch.full((K, optics["H"], optics["W"]), float("nan"), device="cuda")
    o = _lib.optics_struct(optics)
    rc = L.osog_render_noalloc(ctypes.c_void_p(soa_dev.data_ptr()), soa_dev.shape[1],
                               soa_dev.shape[1], ctypes.byref(o),
                               ctypes.c_void_p(out.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out


def test_noalloc_matches_render_on_consecutive_calls():
    from paper_2606_21381_gb300.render import Renderer

    soa_a, o_a = scenes.plain_256(seed=0)                      # brightfield + oblique
    rng = np.random.default_rng(21)
    soa_b = scenes.draw_particles(rng, 900, 256, 256, mu=(0.0, 0.02))
    o_b = scenes.optics(256, 256, modes=7, defocus=-0.7)       # all three modalities
    r = Renderer(256, 256)
    for soa, o in ((soa_a, o_a), (soa_b, o_b), (soa_a, o_a)):
        dev = torch.from_numpy(soa).cuda()
        K = bin(o["modes"]).count("1")
        rc, got = noalloc(dev, o, K)
        assert rc == 0
        want = r.render(dev, None, o)
        torch.cuda.synchronize()
        assert r.sync_status() == 0
        got, want = got.cpu().numpy(), want.cpu().numpy()
        assert np.all(np.isfinite(got))
        for k, bg in enumerate(background(o)):
            assert np.abs(got[k].astype(np.float64) - want[k]).max() <= I_TOL * bg


def test_noalloc_rejects_renders_beyond_its_static_scratch():
    o = scenes.optics(2048, 2048, modes=1)
    dev = torch.zeros((9, 16), device="cuda")
    rc, _ = noalloc(dev, o, 1)
    assert rc == 3  # OSOG_ERR_WORKSPACE: needs more than the 8 MiB static scratch
    o = scenes.optics(256, 256, modes=7)
    dev = torch.zeros((9, 70000), device="cuda")
    rc, _ = noalloc(dev, o, 3)
    assert rc == 3
