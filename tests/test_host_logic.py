"""Host-side logic of the learned warm start and the solver that runs on
the CPU: the multi-tensor Adam equals the per-tensor formula, the loss
selects the same channels as list indexing would, and an unknown solve
mode is refused before any device work."""
import pytest

torch = pytest.importorskip("torch")


def test_multi_tensor_adam_matches_the_per_tensor_formula():
    from paper_2606_21381_gb300.cnn import Adam
    g = torch.Generator().manual_seed(0)
    ps = [torch.randn(5, 3, generator=g), torch.randn(7, generator=g)]
    qs = [p.clone() for p in ps]
    opt = Adam(ps, lr=1e-2)
    m = [torch.zeros_like(p) for p in qs]
    v = [torch.zeros_like(p) for p in qs]
    for t in range(1, 8):
        gs = [torch.randn(p.shape, generator=g) for p in ps]
        opt.step(gs, lr=1e-2 * (1 + 0.1 * t))
        c1, c2 = 1 - 0.9 ** t, 1 - 0.999 ** t
        for q, gr, mm, vv in zip(qs, gs, m, v):
            mm.mul_(0.9).add_(gr, alpha=0.1)
            vv.mul_(0.999).addcmul_(gr, gr, value=0.001)
            q.sub_(1e-2 * (1 + 0.1 * t) * (mm / c1) / (torch.sqrt(vv / c2) + 1e-8))
    for a, b in zip(ps, qs):
        assert torch.allclose(a, b, rtol=1e-6, atol=1e-7)


def test_loss_channels_by_slices_equal_list_indexing():
    from paper_2606_21381_gb300 import cnn
    g = torch.Generator().manual_seed(1)
    out = torch.randn(3, 16, 16, cnn.OUT_CHANNELS, generator=g)
    tgt = torch.rand(3, 16, 16, cnn.OUT_CHANNELS, generator=g)
    mask = torch.rand(3, 16, 16, generator=g) > 0.6
    loss, grad, parts = cnn.loss_and_grad(out, tgt, mask)
    o = out.clone().requires_grad_(True)
    heat = torch.nn.functional.binary_cross_entropy_with_logits(o[..., cnn.CH_HEAT],
                                                                tgt[..., cnn.CH_HEAT])
    m = mask.float()
    reg_ch = [cnn.CH_T, cnn.CH_DN, cnn.CH_OPD]
    reg = (((o[..., reg_ch] - tgt[..., reg_ch]) ** 2).sum(-1) * m).sum() / m.sum().clamp(min=1.0)
    glob_ch = [cnn.CH_DEFOCUS, cnn.CH_NA, cnn.CH_SHEAR, cnn.CH_MEAN_DN]
    gm = o[..., glob_ch].mean(dim=(1, 2))
    glob = ((gm - tgt[:, 0, 0, glob_ch]) ** 2).sum(-1).mean()
    (heat + reg + glob).backward()
    assert torch.allclose(loss, (heat + reg + glob).detach(), rtol=1e-6)
    assert torch.allclose(grad, o.grad, rtol=1e-5, atol=1e-8)
    assert torch.allclose(parts, torch.stack([heat, reg, glob]).detach(), rtol=1e-6)


def test_unknown_solve_mode_is_refused():
    from paper_2606_21381_gb300 import inverse
    with pytest.raises(ValueError):
        inverse.solve(torch.zeros(1, 32, 32), None, {}, None, inverse.SolveConfig(mode="nope"))
