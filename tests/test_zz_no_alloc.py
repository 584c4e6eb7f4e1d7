"""osog_render_noalloc: the render for callers that cannot allocate device
memory, because their host application owns all of it (plugins, real-time
loops that may not block on an allocator).  It takes no plan and no
workspace; its scratch lives in the library's static device arrays.

Checked here: its images equal the FP64 oracle's element by element within
the parity tolerance on consecutive calls that reuse the same static
scratch; the calls leave the device's allocated and free memory unchanged;
its device-side errors (an invalid particle, more particle-band pairs than
the scratch holds) reach the caller through osog_noalloc_sync_status and are
cleared by the read.

This file is collected last on purpose: it must pass in a fresh process
(where its first call performs the per-device set-up) as well as after
every other test.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2606_21381_gb300 import _lib, scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

I_TOL = 2e-4  # of the mean background intensity, as in the parity tests
OK, BIN_OVERFLOW, WORKSPACE, INVALID_PARTICLE = 0, 4, 3, 8


def background(optics):
    return [4 * math.sin(optics["bias_phase"]) ** 2 if bit == 4 else 1.0
            for bit in (1, 2, 4) if optics["modes"] & bit]


def stream_ptr():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def noalloc(soa_dev, optics, out):
    o = _lib.optics_struct(optics)
    return _lib.lib().osog_render_noalloc(ctypes.c_void_p(soa_dev.data_ptr()), soa_dev.shape[1],
                                          soa_dev.shape[1], ctypes.byref(o),
                                          ctypes.c_void_p(out.data_ptr()), stream_ptr())


def sync_status():
    return _lib.lib().osog_noalloc_sync_status(stream_ptr())


def n_modes(o):
    return bin(o["modes"]).count("1")


def test_noalloc_matches_the_oracle_on_consecutive_calls():
    soa_a, o_a = scenes.plain_256(seed=0)                      # brightfield + oblique
    rng = np.random.default_rng(21)
    soa_b = scenes.draw_particles(rng, 900, 256, 256, mu=(0.0, 0.02))
    o_b = scenes.optics(256, 256, modes=7, defocus=-0.7)       # all three modalities
    cases = [(soa_a, o_a), (soa_b, o_b), (soa_a, o_a)]
    inputs = [torch.from_numpy(s).cuda() for s, _ in cases]
    outs = [torch.full((n_modes(o), o["H"], o["W"]), float("nan"), device="cuda")
            for _, o in cases]
    torch.cuda.synchronize()
    for i, ((soa, o), dev, out) in enumerate(zip(cases, inputs, outs)):
        alloc0 = torch.cuda.memory_allocated()
        free0 = torch.cuda.mem_get_info()[0]
        assert noalloc(dev, o, out) == OK
        assert sync_status() == OK
        if i > 0:  # the first call on a device may load the library's module
            assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_allocated() == alloc0
        want = oracle.render(soa, soa.shape[1], oracle.make_optics(**o))["images"]
        got = out.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        for k, bg in enumerate(background(o)):
            assert np.abs(got[k] - want[k]).max() <= I_TOL * bg, (i, k)


def test_noalloc_reports_device_errors_through_its_status_read():
    soa, o = scenes.plain_256(seed=0)
    bad = soa.copy()
    bad[3, 5] = -1.0                                           # a <= 0: invalid particle
    dev = torch.from_numpy(bad).cuda()
    out = torch.empty((n_modes(o), 256, 256), device="cuda")
    assert noalloc(dev, o, out) == OK                          # found on the device
    assert sync_status() == INVALID_PARTICLE
    assert sync_status() == OK                                 # the read cleared it
    # the rest of the scene still renders: only particle 5 is skipped
    keep = np.delete(soa, 5, axis=1)
    want = oracle.render(keep, keep.shape[1], oracle.make_optics(**o))["images"]
    got = out.cpu().numpy().astype(np.float64)
    assert np.abs(got - want).max() <= I_TOL


def test_noalloc_bin_overflow_is_reported_and_the_scratch_recovers():
    # 24,000 particles 600 px tall on a 512^2 canvas (32 bands of 16 rows):
    # 768,000 particle-band pairs, more than the ~325,000 slots the static
    # scratch has left after the scene's other regions
    n = 24000
    rng = np.random.default_rng(5)
    soa = np.zeros((9, n), np.float32)
    soa[0] = rng.uniform(0, 512, n)
    soa[1] = rng.uniform(200, 312, n)
    soa[3] = 0.7                                               # a: 0.7 px wide
    soa[4] = 300.0                                             # b: 300 px tall (theta = 0)
    soa[5] = 1.0
    soa[6] = 0.01
    o = scenes.optics(512, 512, modes=1)
    out = torch.empty((1, 512, 512), device="cuda")
    assert noalloc(torch.from_numpy(soa).cuda(), o, out) == OK
    assert sync_status() == BIN_OVERFLOW
    # the next scene renders correctly from the same scratch
    soa_a, o_a = scenes.plain_256(seed=0)
    out_a = torch.empty((n_modes(o_a), 256, 256), device="cuda")
    assert noalloc(torch.from_numpy(soa_a).cuda(), o_a, out_a) == OK
    assert sync_status() == OK
    want = oracle.render(soa_a, soa_a.shape[1], oracle.make_optics(**o_a))["images"]
    assert np.abs(out_a.cpu().numpy().astype(np.float64) - want).max() <= I_TOL


def test_noalloc_rejects_renders_beyond_its_static_scratch():
    # outputs of the full size, so that nothing is written out of bounds
    # even if a render were accepted
    o = scenes.optics(2048, 2048, modes=1)
    dev = torch.zeros((9, 16), device="cuda")
    out = torch.empty((1, 2048, 2048), device="cuda")
    assert noalloc(dev, o, out) == WORKSPACE   # G and Q alone need 64 MiB
    o = scenes.optics(256, 256, modes=7)
    dev = torch.zeros((9, 100000), device="cuda")  # records alone exceed the 6 MiB left
    out = torch.empty((3, 256, 256), device="cuda")
    assert noalloc(dev, o, out) == WORKSPACE
    assert sync_status() == OK
