"""Every bounded device wait can run out, and when it does the launch still
ends, the error reaches the host as OSOG_ERR_TIMEOUT, and the next call
works.  The waits are made to run out by targets that nothing reaches (a
failure-detection form that neither faults nor hangs the GPU):

- the persistent batched launch: each column item waits for one more
  finished strip than its scene has (osog_tuning_t.test_wait_extra) with a
  short poll limit (osog_tuning_t.wait_polls);
- the column pass's wait for the bulk copy of its column block (square
  canvases of 1024 or more): the barrier expects 16 bytes more than the
  copy delivers (the same test_wait_extra), with a short poll limit;
- the tcgen05 convolutions: every CTA also waits, for a few polls, on a
  barrier that nothing arrives on (osog_conv_test_wait_limit); the kernel
  still waits for its own tensor-core work and releases its tensor memory,
  which the next convolution (it allocates the same tensor memory) shows.
"""
import numpy as np
import pytest

from paper_2606_21381_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT = 6


def test_persistent_launch_wait_runs_out_and_the_next_launch_is_correct():
    from paper_2606_21381_gb300.render import Renderer
    rng = np.random.default_rng(8)
    soas = [scenes.draw_particles(rng, int(c), 256, 256, mu=(0, 0.02)) for c in (300, 50, 420)]
    optics = [scenes.optics(256, 256, modes=3, defocus=d) for d in (0.3, -0.5, 1.1)]
    soa_all, offs = scenes.concat(soas)
    dev = torch.from_numpy(soa_all).cuda()
    r = Renderer(256, 256)
    base = r.batch(dev, offs, optics, tuning={"use_graph": 0, "persistent": -1}).clone()
    assert r.sync_status() == 0
    r.batch(dev, offs, optics, tuning={"use_graph": 0, "persistent": 1, "wait_polls": 2000,
                                       "test_wait_extra": 1})
    torch.cuda.synchronize()   # the launch ended
    assert r.sync_status() == TIMEOUT
    assert r.sync_status() == 0  # read and cleared
    again = r.batch(dev, offs, optics, tuning={"use_graph": 0, "persistent": 1}).clone()
    assert r.sync_status() == 0
    assert torch.equal(again, base)


def test_column_bulk_copy_wait_runs_out_and_the_next_launch_is_correct():
    from paper_2606_21381_gb300.render import Renderer
    rng = np.random.default_rng(10)
    soas = [scenes.draw_particles(rng, int(c), 1024, 1024, mu=(0, 0.02)) for c in (900, 400)]
    optics = [scenes.optics(1024, 1024, modes=1, defocus=d) for d in (0.4, -0.8)]
    soa_all, offs = scenes.concat(soas)
    dev = torch.from_numpy(soa_all).cuda()
    r = Renderer(1024, 1024)
    three = {"use_graph": 0, "persistent": -1}
    base = r.batch(dev, offs, optics, tuning=three).clone()
    assert r.sync_status() == 0
    r.batch(dev, offs, optics, tuning=dict(three, wait_polls=2000, test_wait_extra=1))
    torch.cuda.synchronize()   # the launch ended
    assert r.sync_status() == TIMEOUT
    assert r.sync_status() == 0
    again = r.batch(dev, offs, optics, tuning=three).clone()
    assert r.sync_status() == 0
    assert torch.equal(again, base)


def test_convolution_wait_runs_out_and_tensor_memory_is_released():
    from oracle import cnn_reference as ref
    from paper_2606_21381_gb300 import _lib, cnn
    dev = torch.device("cuda")
    rng = np.random.default_rng(9)
    N, H, W, C, K = 1, 40, 40, 40, 128   # reductions of 360: the tcgen05 path
    x = rng.standard_normal((N, H, W, C))
    w = rng.standard_normal((K, 3, 3, C)) / np.sqrt(9 * C)
    b = rng.standard_normal(K).astype(np.float32)
    xt = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16)
    wt = torch.from_numpy(w.astype(np.float32)).to(torch.bfloat16)
    xd, wd, bd = xt.to(dev), wt.to(dev), torch.from_numpy(b).to(dev)
    want = ref.conv_forward(xt.double().numpy(), wt.double().numpy(), b.astype(np.float64), 1, 1,
                            True)
    cnn.use_tcgen05(True)
    assert cnn.sync_status() == 0
    L = _lib.lib()
    try:
        assert L.osog_conv_test_wait_limit(64) == 0
        y, y32 = cnn.conv2d(xd, wd, bd, 1, 1, True, want_f32=True)
        dy = torch.ones_like(y)
        cnn.conv2d_backward_filter(dy, xd, w.shape, 1, 1)   # the tcgen05 filter gradient too
        assert cnn.sync_status() == TIMEOUT
    finally:
        assert L.osog_conv_test_wait_limit(0) == 0
    # the results of the launch whose probe wait ran out are still valid
    assert np.abs(y32.cpu().numpy() - want).max() <= 1e-5 * np.abs(want).max()
    # and the next launches allocate the tensor memory again and finish
    y2, y32b = cnn.conv2d(xd, wd, bd, 1, 1, True, want_f32=True)
    cnn.conv2d_backward_filter(dy, xd, w.shape, 1, 1)
    assert cnn.sync_status() == 0
    assert torch.equal(y32, y32b)
