"""The warm-start network's convolution kernels against the float64 CPU
reference: forward, data gradient (with the ReLU mask), filter and bias
gradients on ragged shapes, bitwise determinism, and the whole network's
parameter gradients."""
import numpy as np
import pytest
import torch

from oracle import cnn_reference as ref

pytestmark = pytest.mark.gpu

# N, H, W, C, K, R, S, stride, pad: tails in every GEMM dimension
SHAPES = [
    (2, 17, 23, 8, 32, 3, 3, 1, 1),
    (2, 33, 31, 8, 24, 3, 3, 2, 1),
    (1, 40, 40, 40, 72, 3, 3, 2, 1),
    (3, 16, 16, 128, 64, 3, 3, 1, 1),
    (2, 9, 13, 32, 8, 1, 1, 1, 0),
    (1, 66, 70, 64, 128, 3, 3, 1, 1),
    (1, 30, 30, 16, 16, 3, 3, 2, 0),
    (2, 15, 17, 16, 8, 1, 1, 2, 0),   # stride 2, 1 x 1: two parity classes see no tap
    (1, 21, 19, 8, 16, 5, 5, 2, 2),
    (1, 64, 64, 32, 64, 3, 3, 2, 1),  # the network's second layer at small size
]


def _bf16(a, dev):
    """(bf16 device tensor, the same values as float64 numpy)."""
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.to(dev), t.to(torch.float64).numpy()


def _inputs(shape, seed):
    N, H, W, C, K, R, S, stride, pad = shape
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((N, H, W, C))
    w = rng.standard_normal((K, R, S, C)) / np.sqrt(R * S * C)
    b = rng.standard_normal(K).astype(np.float32)
    P = (H + 2 * pad - R) // stride + 1
    Q = (W + 2 * pad - S) // stride + 1
    dy = rng.standard_normal((N, P, Q, K))
    return x, w, b, dy


@pytest.fixture(scope="module", params=["tcgen05", "mma_sync"])
def cnn(request):
    """The convolution module with the forward / data-gradient engine set to
    the tcgen05 tensor cores or the warp-level MMA (every test runs on both)."""
    from paper_2606_21381_gb300 import cnn as m
    m.use_tcgen05(request.param == "tcgen05")
    yield m
    assert m.sync_status() == 0
    m.use_tcgen05(True)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("relu", [False, True])
def test_conv_forward_matches_reference(cnn, shape, relu):
    dev = torch.device("cuda")
    x, w, b, _ = _inputs(shape, 1)
    xd, x64 = _bf16(x, dev)
    wd, w64 = _bf16(w, dev)
    bd = torch.from_numpy(b).to(dev)
    y, y32 = cnn.conv2d(xd, wd, bd, shape[7], shape[8], relu, want_f32=True)
    want = ref.conv_forward(x64, w64, b.astype(np.float64), shape[7], shape[8], relu)
    assert cnn.sync_status() == 0
    got32 = y32.cpu().numpy().astype(np.float64)
    scale = np.abs(want).max()
    assert np.abs(got32 - want).max() <= 1e-5 * scale
    # the bf16 output is the fp32 value rounded to nearest
    got = y.to(torch.float32).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 1e-5 * scale)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("masked", [False, True])
def test_conv_backward_data_matches_reference(cnn, shape, masked):
    dev = torch.device("cuda")
    x, w, b, dy = _inputs(shape, 2)
    xd, x64 = _bf16(x, dev)
    wd, w64 = _bf16(w, dev)
    dyd, dy64 = _bf16(dy, dev)
    dx = cnn.conv2d_backward_data(dyd, wd, tuple(xd.shape), shape[7], shape[8],
                                  x_act=xd if masked else None)
    want, _, _ = ref.conv_grads(x64, w64, b.astype(np.float64), shape[7], shape[8], dy64)
    if masked:
        want = want * (x64 > 0)
    assert cnn.sync_status() == 0
    got = dx.to(torch.float32).cpu().numpy().astype(np.float64)
    scale = np.abs(want).max()
    assert np.all(np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 1e-5 * scale)


@pytest.mark.parametrize("shape", SHAPES)
def test_conv_backward_filter_matches_reference(cnn, shape):
    dev = torch.device("cuda")
    x, w, b, dy = _inputs(shape, 3)
    xd, x64 = _bf16(x, dev)
    _, w64 = _bf16(w, dev)
    dyd, dy64 = _bf16(dy, dev)
    dw, db = cnn.conv2d_backward_filter(dyd, xd, w.shape, shape[7], shape[8])
    _, want_w, want_b = ref.conv_grads(x64, w64, b.astype(np.float64), shape[7], shape[8], dy64)
    got_w = dw.cpu().numpy().astype(np.float64)
    assert np.abs(got_w - want_w).max() <= 1e-5 * np.abs(want_w).max() * np.sqrt(dy.size / dy.shape[-1])
    assert np.abs(db.cpu().numpy() - want_b).max() <= 1e-5 * np.abs(dy64).sum(axis=(0, 1, 2)).max()


def test_filter_gradient_spans_several_pixel_splits(cnn):
    # 2 x 64 x 64 output pixels = 4 splits of 2048 plus a ragged tail
    shape = (2, 65, 66, 8, 16, 3, 3, 1, 1)
    test_conv_backward_filter_matches_reference(cnn, shape)


def test_kernels_are_bitwise_deterministic(cnn):
    dev = torch.device("cuda")
    shape = (4, 64, 64, 32, 64, 3, 3, 1, 1)
    x, w, b, dy = _inputs(shape, 4)
    xd, _ = _bf16(x, dev)
    wd, _ = _bf16(w, dev)
    dyd, _ = _bf16(dy, dev)
    bd = torch.from_numpy(b).to(dev)
    outs = []
    for _ in range(2):
        y = cnn.conv2d(xd, wd, bd, 1, 1, True)
        dx = cnn.conv2d_backward_data(dyd, wd, tuple(xd.shape), 1, 1, x_act=xd)
        dw, db = cnn.conv2d_backward_filter(dyd, xd, w.shape, 1, 1)
        outs.append([t.clone() for t in (y, dx, dw, db)])
    for a, c in zip(*outs):
        assert torch.equal(a, c)


def test_relu_backward(cnn):
    dev = torch.device("cuda")
    rng = np.random.default_rng(5)
    dyd, dy64 = _bf16(rng.standard_normal(1000), dev)
    actd, act64 = _bf16(rng.standard_normal(1000), dev)
    got = cnn.relu_backward(dyd, actd).to(torch.float32).cpu().numpy()
    assert np.array_equal(got, np.where(act64 > 0, dy64, 0.0).astype(np.float32))


def _reference_network_grads(net, x64, dout64):
    """float64 CPU autograd through the same network, with activations
    rounded to bf16 where the kernels store them."""
    import torch.nn.functional as F
    ws = [torch.from_numpy(w.to(torch.bfloat16).to(torch.float64).cpu().numpy()).permute(0, 3, 1, 2)
          .contiguous().requires_grad_(True) for w in net.w]
    bs = [b.cpu().double().clone().requires_grad_(True) for b in net.b]
    a = torch.from_numpy(x64).permute(0, 3, 1, 2)
    for i, (_, _, _, stride, pad) in enumerate(net.specs):
        z = F.conv2d(a, ws[i], bs[i], stride=stride, padding=pad)
        if i < len(net.specs) - 1:
            a = torch.clamp(z, min=0.0)
            a = a + (a.to(torch.bfloat16).to(torch.float64) - a).detach()
        else:
            out = z
    (out * torch.from_numpy(dout64).permute(0, 3, 1, 2)).sum().backward()
    return [w.grad.permute(0, 2, 3, 1).numpy() for w in ws], [b.grad.numpy() for b in bs], \
        out.detach().permute(0, 2, 3, 1).numpy()


def test_network_gradients_match_reference(cnn):
    dev = torch.device("cuda")
    net = cnn.WarmStartNet(dev, seed=1)
    rng = np.random.default_rng(6)
    x = np.zeros((2, 64, 64, 8))
    x[..., :2] = rng.standard_normal((2, 64, 64, 2))
    xd, x64 = _bf16(x, dev)
    out, acts = net.forward(xd)
    dout = rng.standard_normal(tuple(out.shape)).astype(np.float32)
    doutd, dout64 = _bf16(dout, dev)
    grads = net.backward(doutd.to(torch.float32), acts)
    want_w, want_b, want_out = _reference_network_grads(net, x64, dout64)
    got_out = out.cpu().numpy()
    assert np.abs(got_out - want_out).max() <= 2e-2 * np.abs(want_out).max()
    for i, ((dw, db), ww, wb) in enumerate(zip(grads, want_w, want_b)):
        gw = dw.cpu().numpy().astype(np.float64)
        if i == 0:  # padding channels are zero in the input
            gw, ww = gw[..., :2], ww[..., :2]
        cos = (gw * ww).sum() / np.sqrt((gw * gw).sum() * (ww * ww).sum())
        assert cos > 0.999, (i, cos)
        assert np.linalg.norm(gw - ww) <= 3e-2 * np.linalg.norm(ww), i
        gb = db.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(gb - wb) <= 3e-2 * np.linalg.norm(wb) + 1e-6, i
