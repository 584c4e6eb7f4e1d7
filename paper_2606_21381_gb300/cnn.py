"""Learned warm start of the inverse solve: a small BF16 convolutional
network with FP32 accumulation that reads a brightfield + DIC image and
predicts the global optics (defocus, NA, shear, mean dn) and, on a grid of
8 x 8 pixel cells, where particle centres are and their thickness and dn.
Its predictions replace the perturbed starting values of the gradient-based
recovery (the paper's differentiable calibration, Sec. IV.B); the plain
curriculum solve stays the fallback and the judge of the error.

Every convolution, its data gradient and its filter gradient run in
libosog's implicit-GEMM tensor-core kernels (``osog_cnn.h``); the network is
trained only on images the renderer produces on the fly.  The loss on the
head outputs, the input packing and Adam are small elementwise torch
operations on device tensors.
"""
from __future__ import annotations

import ctypes
import math
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib, scenes
from ._lib import check

CELL = 8                # pixels per output cell (three stride-2 layers)
IN_CHANNELS = 8         # BF, DIC, zero padding to the kernels' multiple of 8
OUT_CHANNELS = 8
# (C_in, C_out, stride) of the six 3 x 3 layers, then the 1 x 1 head
LAYERS = ((IN_CHANNELS, 32, 2), (32, 64, 2), (64, 128, 2), (128, 128, 1), (128, 64, 1),
          (64, 32, 1))
# head output channels
CH_HEAT, CH_T, CH_DN, CH_DEFOCUS, CH_NA, CH_SHEAR, CH_MEAN_DN, CH_OPD = range(8)
# target normalisation: (value - centre) / scale
NORM = {"T": (1.75, 1.25), "dn": (0.0325, 0.0275), "defocus": (0.0, 2.0), "NA": (0.45, 0.15),
        "shear": (1.0, 0.5), "opd": (0.06, 0.06)}
INPUT_SCALE = 2.0


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(dev) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def conv_shape(x: torch.Tensor, w: torch.Tensor, stride: int, pad: int) -> _lib.ConvShape:
    N, H, W, C = x.shape
    K, R, S, C2 = w.shape
    if C != C2:
        raise ValueError(f"input has {C} channels, filters {C2}")
    return _lib.ConvShape(N, H, W, C, K, R, S, stride, pad)


def _out_hw(s: _lib.ConvShape) -> tuple[int, int]:
    L = _lib.lib()
    P, Q = L.osog_conv_out_h(ctypes.byref(s)), L.osog_conv_out_w(ctypes.byref(s))
    if P <= 0 or Q <= 0:
        raise ValueError(f"invalid convolution shape {[getattr(s, f) for f, _ in s._fields_]}")
    return P, Q


def _require(t: torch.Tensor, dtype, name: str):
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")


def conv2d(x, w, bias, stride: int, pad: int, relu: bool, want_f32: bool = False):
    """NHWC bf16 y = act(conv(x, w) + bias) (and its fp32 copy if asked)."""
    _require(x, torch.bfloat16, "x")
    _require(w, torch.bfloat16, "w")
    _require(bias, torch.float32, "bias")
    s = conv_shape(x, w, stride, pad)
    P, Q = _out_hw(s)
    y = torch.empty((s.N, P, Q, s.K), dtype=torch.bfloat16, device=x.device)
    y32 = torch.empty((s.N, P, Q, s.K), dtype=torch.float32, device=x.device) if want_f32 else None
    check(_lib.lib().osog_conv2d_forward(ctypes.byref(s), _ptr(x), _ptr(w), _ptr(bias), int(relu),
                                         _ptr(y), _ptr(y32), _stream(x.device)), "osog_conv2d_forward")
    return (y, y32) if want_f32 else y


def conv2d_backward_data(dy, w, x_shape, stride: int, pad: int, x_act=None):
    """dx (bf16 NHWC of x_shape), times (x_act > 0) when x_act is given."""
    _require(dy, torch.bfloat16, "dy")
    _require(w, torch.bfloat16, "w")
    if x_act is not None:
        _require(x_act, torch.bfloat16, "x_act")
    N, H, W, C = x_shape
    K, R, S, _ = w.shape
    s = _lib.ConvShape(N, H, W, C, K, R, S, stride, pad)
    P, Q = _out_hw(s)
    if tuple(dy.shape) != (N, P, Q, K):
        raise ValueError(f"dy has shape {tuple(dy.shape)}, expected {(N, P, Q, K)}")
    dx = torch.empty((N, H, W, C), dtype=torch.bfloat16, device=dy.device)
    w_t = torch.empty_like(w)
    check(_lib.lib().osog_conv2d_backward_data(ctypes.byref(s), _ptr(dy), _ptr(w), _ptr(x_act),
                                               _ptr(dx), _ptr(w_t), _stream(dy.device)),
          "osog_conv2d_backward_data")
    return dx


def conv2d_backward_filter(dy, x, w_shape, stride: int, pad: int, ws=None):
    """(dw fp32 [K][R][S][C], dbias fp32 [K])."""
    _require(dy, torch.bfloat16, "dy")
    _require(x, torch.bfloat16, "x")
    K, R, S, C = w_shape
    N, H, W, _ = x.shape
    s = _lib.ConvShape(N, H, W, C, K, R, S, stride, pad)
    P, Q = _out_hw(s)
    if tuple(dy.shape) != (N, P, Q, K):
        raise ValueError(f"dy has shape {tuple(dy.shape)}, expected {(N, P, Q, K)}")
    L = _lib.lib()
    need = L.osog_conv2d_backward_filter_workspace(ctypes.byref(s))
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 16), dtype=torch.uint8, device=dy.device)
    dw = torch.empty((K, R, S, C), dtype=torch.float32, device=dy.device)
    db = torch.empty((K,), dtype=torch.float32, device=dy.device)
    check(L.osog_conv2d_backward_filter(ctypes.byref(s), _ptr(dy), _ptr(x), _ptr(dw), _ptr(db),
                                        _ptr(ws), ws.numel(), _stream(dy.device)),
          "osog_conv2d_backward_filter")
    return dw, db


def use_tcgen05(enable: bool) -> None:
    """Engine of the forward and data-gradient convolutions (process-wide):
    tcgen05 tensor cores (default) or the warp-level MMA."""
    _lib.lib().osog_conv_use_tcgen05(1 if enable else 0)


def sync_status(device=None) -> int:
    """Synchronise and return (and clear) a latched convolution error."""
    dev = torch.device(device or "cuda")
    return int(_lib.lib().osog_conv_sync_status(_stream(dev)))


def relu_backward(dy, act):
    _require(dy, torch.bfloat16, "dy")
    _require(act, torch.bfloat16, "act")
    out = torch.empty_like(dy)
    check(_lib.lib().osog_relu_backward(_ptr(dy), _ptr(act), _ptr(out), dy.numel(),
                                        _stream(dy.device)), "osog_relu_backward")
    return out


# ------------------------------------------------------------------ network
class WarmStartNet:
    """Six 3 x 3 convolutions (32-64-128-128-64-32 channels; the first three
    with stride 2) with ReLU, then a 1 x 1 head to OUT_CHANNELS per 8 x 8
    pixel cell.  Master weights are fp32; the kernels read bf16 copies."""

    def __init__(self, device="cuda", seed: int = 0):
        self.device = torch.device(device)
        g = torch.Generator().manual_seed(seed)
        self.specs = [(cin, cout, 3, stride, 1) for cin, cout, stride in LAYERS]
        self.specs.append((LAYERS[-1][1], OUT_CHANNELS, 1, 1, 0))
        self.w, self.b = [], []
        for i, (cin, cout, k, _, _) in enumerate(self.specs):
            fan_in = (2 if i == 0 else cin) * k * k
            std = math.sqrt((1.0 if i == len(self.specs) - 1 else 2.0) / fan_in)
            w = torch.randn(cout, k, k, cin, generator=g) * std
            if i == 0:
                w[..., 2:] = 0.0  # padding channels carry no signal
            self.w.append(w.to(self.device))
            self.b.append(torch.zeros(cout, device=self.device))
        self.sigma = None   # held-out RMS errors, set by calibrate()
        self.refresh()

    def refresh(self) -> None:
        """Round the master weights to the bf16 copies the kernels read (in
        place once they exist, so that a captured CUDA graph keeps reading
        the current values)."""
        wb = getattr(self, "wb", None)
        if wb is not None and len(wb) == len(self.w) and all(
                a.shape == b.shape and a.device == b.device for a, b in zip(wb, self.w)):
            for a, b in zip(wb, self.w):
                a.copy_(b)
        else:
            self.wb = [w.to(torch.bfloat16).contiguous() for w in self.w]

    def parameters(self) -> list[torch.Tensor]:
        return self.w + self.b

    def forward(self, x: torch.Tensor):
        """x: bf16 NHWC [N][H][W][8] -> (fp32 head output [N][H/8][W/8][8],
        activations kept for the backward pass)."""
        acts = [x]
        last = len(self.specs) - 1
        for i, (_, _, _, stride, pad) in enumerate(self.specs):
            if i < last:
                acts.append(conv2d(acts[-1], self.wb[i], self.b[i], stride, pad, relu=True))
            else:
                _, out = conv2d(acts[-1], self.wb[i], self.b[i], stride, pad, relu=False,
                                want_f32=True)
        return out, acts

    def backward(self, dout: torch.Tensor, acts) -> list[tuple[torch.Tensor, torch.Tensor]]:
        """Gradients (dw, db) of every layer from dL/d(head output)."""
        dy = dout.to(torch.bfloat16).contiguous()
        grads = [None] * len(self.specs)
        for i in reversed(range(len(self.specs))):
            _, _, _, stride, pad = self.specs[i]
            grads[i] = conv2d_backward_filter(dy, acts[i], tuple(self.w[i].shape), stride, pad)
            if i > 0:  # through this layer and the ReLU that produced its input
                dy = conv2d_backward_data(dy, self.wb[i], tuple(acts[i].shape), stride, pad,
                                          x_act=acts[i])
        return grads

    def state_dict(self) -> dict:
        return {"w": [w.cpu() for w in self.w], "b": [b.cpu() for b in self.b],
                "sigma": self.sigma}

    def load_state_dict(self, d: dict) -> None:
        self.w = [w.to(self.device) for w in d["w"]]
        self.b = [b.to(self.device) for b in d["b"]]
        self.sigma = d.get("sigma")
        self.refresh()


class Adam:
    def __init__(self, params, lr=1e-3, betas=(0.9, 0.999), eps=1e-8):
        self.p, self.lr, self.betas, self.eps, self.t = params, lr, betas, eps, 0
        self.m = [torch.zeros_like(p) for p in params]
        self.v = [torch.zeros_like(p) for p in params]

    @torch.no_grad()
    def step(self, grads, lr=None) -> None:
        """p -= lr (m / c1) / (sqrt(v / c2) + eps) on all parameters at once
        (multi-tensor operations: a few launches instead of a few per
        tensor)."""
        self.t += 1
        b1, b2 = self.betas
        lr = self.lr if lr is None else lr
        c1, c2 = 1 - b1 ** self.t, 1 - b2 ** self.t
        torch._foreach_mul_(self.m, b1)
        torch._foreach_add_(self.m, grads, alpha=1 - b1)
        torch._foreach_mul_(self.v, b2)
        torch._foreach_addcmul_(self.v, grads, grads, value=1 - b2)
        den = torch._foreach_div(self.v, c2)
        torch._foreach_sqrt_(den)
        torch._foreach_add_(den, self.eps)
        upd = torch._foreach_div(self.m, den)
        torch._foreach_mul_(upd, lr / c1)
        torch._foreach_sub_(self.p, upd)


# ------------------------------------------------------------------ data
def pack_input(images: torch.Tensor, crop: int | None = None) -> torch.Tensor:
    """(S, 2, H, W) brightfield + DIC images -> bf16 NHWC network input of
    the crops (S (H/crop) (W/crop), crop, crop, 8): each channel minus its
    crop mean, times INPUT_SCALE, zero padding channels."""
    S, K, H, W = images.shape
    if K != 2:
        raise ValueError("the network reads brightfield + DIC (2 modalities)")
    c = crop or H
    if H % c or W % c:
        raise ValueError("the crop must tile the image")
    x = images.reshape(S, K, H // c, c, W // c, c).permute(0, 2, 4, 3, 5, 1)
    x = x.reshape(-1, c, c, K)
    x = (x - x.mean(dim=(1, 2), keepdim=True)) * INPUT_SCALE
    out = torch.zeros((x.shape[0], c, c, IN_CHANNELS), dtype=torch.bfloat16, device=images.device)
    out[..., :K] = x
    return out


def _norm(key, v):
    c, s = NORM[key]
    return (v - c) / s


def _denorm(key, v):
    c, s = NORM[key]
    return v * s + c


def random_optics(rng: np.random.Generator, size: int) -> dict:
    """Training optics: brightfield + DIC, defocus U(-2, 2) um, NA U(0.3,
    0.6), shear length U(0.5, 1.5) px."""
    return scenes.optics(size, size, modes=scenes.MODE_BF | scenes.MODE_DIC,
                         NA=float(rng.uniform(0.3, 0.6)), defocus=float(rng.uniform(-2.0, 2.0)),
                         shear_px=float(rng.uniform(0.5, 1.5)))


def random_scene(rng: np.random.Generator, size: int) -> np.ndarray:
    """Particles with the batched workload's distributions: count
    log-uniform in [1e3, 4e4] per 2048^2 (scaled by area), dn U(0.005,
    0.06), absorption U(0, 0.02)."""
    count = int(round(math.exp(rng.uniform(math.log(1e3), math.log(4e4))) * (size / 2048.0) ** 2))
    return scenes.draw_particles(rng, max(count, 1), size, size, dn=(0.005, 0.06), mu=(0.0, 0.02))


def cell_targets(soas, optics_list, size: int, crop: int):
    """Per crop and cell: target [N][crop/8][crop/8][8] (heat, T, dn, 4
    global values, dn T) and the mask of cells holding a particle centre
    (the largest dn T wins a shared cell)."""
    per = size // crop
    g = crop // CELL
    n_crops = len(soas) * per * per
    tgt = np.zeros((n_crops, g, g, OUT_CHANNELS), dtype=np.float32)
    mask = np.zeros((n_crops, g, g), dtype=bool)
    soa = np.concatenate(soas, axis=1)
    scene = np.repeat(np.arange(len(soas)), [a.shape[1] for a in soas])
    cx, cy, T, dn = soa[0], soa[1], soa[5], soa[6]
    opd = dn * T
    ix = np.clip(cx.astype(np.int64), 0, size - 1)
    iy = np.clip(cy.astype(np.int64), 0, size - 1)
    crop_id = scene * per * per + (iy // crop) * per + (ix // crop)
    order = np.argsort(opd, kind="stable")  # later (larger) entries win a cell
    ci, gi, gj = crop_id[order], ((iy % crop) // CELL)[order], ((ix % crop) // CELL)[order]
    mask[ci, gi, gj] = True
    tgt[ci, gi, gj, CH_HEAT] = 1.0
    tgt[ci, gi, gj, CH_T] = _norm("T", T[order])
    tgt[ci, gi, gj, CH_DN] = _norm("dn", dn[order])
    tgt[ci, gi, gj, CH_OPD] = _norm("opd", opd[order])
    cnt = np.bincount(crop_id, minlength=n_crops)
    sums = np.bincount(crop_id, weights=dn, minlength=n_crops)
    scene_mean = np.array([a[6].mean() for a in soas])
    mean_dn = np.where(cnt > 0, sums / np.maximum(cnt, 1), np.repeat(scene_mean, per * per))
    tgt[..., CH_MEAN_DN] = _norm("dn", mean_dn)[:, None, None]
    rep = lambda v: np.repeat(np.asarray(v, dtype=np.float64), per * per)[:, None, None]
    tgt[..., CH_DEFOCUS] = _norm("defocus", rep([o["defocus"] for o in optics_list]))
    tgt[..., CH_NA] = _norm("NA", rep([o["NA"] for o in optics_list]))
    tgt[..., CH_SHEAR] = _norm("shear", rep([o["shear_px"] for o in optics_list]))
    return tgt, mask


class _PinnedStaging:
    """Host-to-device copies through two reused pinned buffers per array
    kind, so the host can run ahead without page-locking memory each step;
    a slot is refilled only after its previous copy has finished."""

    def __init__(self):
        self.bufs, self.events, self.turn = {}, {}, 0

    def next_turn(self) -> None:
        self.turn ^= 1

    def to_device(self, key: str, a: np.ndarray, dev) -> torch.Tensor:
        src = torch.from_numpy(np.ascontiguousarray(a))
        k = (key, self.turn)
        buf = self.bufs.get(k)
        if buf is None or buf.numel() < src.numel() or buf.dtype != src.dtype:
            buf = torch.empty(max(src.numel(), 1), dtype=src.dtype, pin_memory=True)
            self.bufs[k] = buf
            self.events.pop(k, None)
        ev = self.events.get(k)
        if ev is not None:
            ev.synchronize()
        view = buf[:src.numel()].view(src.shape)
        view.copy_(src)
        out = view.to(dev, non_blocking=True)
        e = torch.cuda.Event()
        e.record(torch.cuda.current_stream(dev))
        self.events[k] = e
        return out


class RenderStream:
    """Batches of training crops rendered on the fly: each batch draws
    `scenes_per_batch` random scenes with random optics, renders them in one
    batched call and cuts them into crop x crop windows."""

    def __init__(self, renderer, scenes_per_batch: int = 16, crop: int = 256, seed: int = 0):
        if renderer.H != renderer.W or renderer.H % crop:
            raise ValueError("the canvas must be square and tiled by the crop")
        self.r, self.S, self.crop = renderer, scenes_per_batch, crop
        self.size = renderer.H
        self.rng = np.random.default_rng(seed)
        self.staging = _PinnedStaging()

    @property
    def crops_per_batch(self) -> int:
        return self.S * (self.size // self.crop) ** 2

    def next(self):
        soas = [random_scene(self.rng, self.size) for _ in range(self.S)]
        optics_list = [random_optics(self.rng, self.size) for _ in range(self.S)]
        soa_all, offsets = scenes.concat(soas)
        dev = self.r.device
        st = self.staging
        st.next_turn()
        # direct launches: the counts change every batch, so a cached graph
        # would be captured anew each time
        imgs = self.r.batch(st.to_device("soa", soa_all, dev), offsets, optics_list,
                            tuning={"use_graph": 0})
        x = pack_input(imgs, self.crop)
        tgt, mask = cell_targets(soas, optics_list, self.size, self.crop)
        return x, st.to_device("tgt", tgt, dev), st.to_device("mask", mask, dev)


# ------------------------------------------------------------------ training
def loss_and_grad(out: torch.Tensor, tgt: torch.Tensor, mask: torch.Tensor):
    """Loss of the head output and its gradient: logistic loss of the centre
    heat map over all cells, squared error of (T, dn, dn T) at cells holding
    a centre, squared error of the cell-averaged global channels."""
    # channels by slices only (no index tensors to copy from the host, so
    # the step can be captured as a CUDA graph): T and dn are adjacent, the
    # four global channels too
    o = out.detach().requires_grad_(True)
    heat = torch.nn.functional.binary_cross_entropy_with_logits(o[..., CH_HEAT], tgt[..., CH_HEAT])
    m = mask.float()
    d = o - tgt
    sq = (d[..., CH_T:CH_DN + 1] ** 2).sum(-1) + d[..., CH_OPD] ** 2
    reg = (sq * m).sum() / m.sum().clamp(min=1.0)
    g = o[..., CH_DEFOCUS:CH_MEAN_DN + 1].mean(dim=(1, 2))
    glob = ((g - tgt[:, 0, 0, CH_DEFOCUS:CH_MEAN_DN + 1]) ** 2).sum(-1).mean()
    loss = heat + reg + glob
    loss.backward()
    return loss.detach(), o.grad, torch.stack([heat.detach(), reg.detach(), glob.detach()])


@dataclass
class TrainConfig:
    samples: int = 200_000          # training crops
    canvas: int = 512               # rendered scene size; cut into crops
    crop: int = 256
    scenes_per_batch: int = 16      # 64 crops per step at 512 / 256
    lr: float = 2e-3
    lr_final: float = 1e-4          # cosine decay to this
    seed: int = 0
    log_every: int = 0
    # replay the network's step (forward, loss, backward, Adam) as one CUDA
    # graph after a few eager steps; the render of each batch stays eager
    graph: bool = True
    warmup_steps: int = 3


@dataclass
class TrainResult:
    steps: int
    samples: int
    seconds: float
    losses: np.ndarray              # (steps, 4): total, heat, regression, global


class _GraphedStep:
    """The network's training step on static input buffers with every
    per-step scalar on the device (step count, cosine learning rate, Adam
    bias corrections), so that it can be captured once as a CUDA graph and
    replayed: forward, loss and its gradient, backward, Adam (per tensor,
    with device scalars) and the bf16 weight copies."""

    def __init__(self, net, opt, cfg, steps, x, tgt, mask):
        self.net, self.opt, self.cfg, self.steps = net, opt, cfg, float(steps)
        self.x, self.tgt, self.mask = x.clone(), tgt.clone(), mask.clone()
        self.t = torch.zeros((), dtype=torch.float32, device=net.device)
        self.out = torch.zeros(4, dtype=torch.float32, device=net.device)

    def load(self, x, tgt, mask) -> None:
        self.x.copy_(x)
        self.tgt.copy_(tgt)
        self.mask.copy_(mask)

    def __call__(self) -> None:
        net, opt, cfg = self.net, self.opt, self.cfg
        b1, b2 = opt.betas
        lr = cfg.lr_final + 0.5 * (cfg.lr - cfg.lr_final) * (
            1.0 + torch.cos(math.pi * self.t / self.steps))
        t1 = self.t + 1.0
        c1, c2 = 1.0 - torch.pow(b1, t1), 1.0 - torch.pow(b2, t1)
        out, acts = net.forward(self.x)
        loss, dout, parts = loss_and_grad(out, self.tgt, self.mask)
        grads = net.backward(dout, acts)
        with torch.no_grad():
            for p, g, m, v in zip(opt.p, [g[0] for g in grads] + [g[1] for g in grads],
                                  opt.m, opt.v):
                m.mul_(b1).add_(g, alpha=1 - b1)
                v.mul_(b2).addcmul_(g, g, value=1 - b2)
                p.sub_(lr * (m / c1) / (torch.sqrt(v / c2) + opt.eps))
            net.refresh()
            self.out[0] = loss
            self.out[1:] = parts
            self.t.copy_(t1)


def train(net: WarmStartNet, cfg: TrainConfig | None = None, renderer=None) -> TrainResult:
    """Adam on crops rendered on the fly, one batched render per step.  With
    cfg.graph the network's step runs eagerly for cfg.warmup_steps steps
    and is then replayed as one CUDA graph (the render stays eager: its
    particle counts change every batch)."""
    from .render import Renderer
    cfg = cfg or TrainConfig()
    r = renderer or Renderer(cfg.canvas, cfg.canvas, net.device)
    data = RenderStream(r, cfg.scenes_per_batch, cfg.crop, cfg.seed)
    steps = max(1, math.ceil(cfg.samples / data.crops_per_batch))
    opt = Adam(net.parameters(), cfg.lr)
    hist = torch.zeros((steps, 4), device=net.device)
    if cfg.graph:
        return _train_graphed(net, cfg, data, steps, opt, hist)
    torch.cuda.synchronize(net.device)
    t0 = time.perf_counter()
    for it in range(steps):
        lr = cfg.lr_final + 0.5 * (cfg.lr - cfg.lr_final) * (1 + math.cos(math.pi * it / steps))
        x, tgt, mask = data.next()
        out, acts = net.forward(x)
        loss, dout, parts = loss_and_grad(out, tgt, mask)
        grads = net.backward(dout, acts)
        opt.step([g[0] for g in grads] + [g[1] for g in grads], lr)
        net.refresh()
        hist[it, 0] = loss
        hist[it, 1:] = parts
        if cfg.log_every and it % cfg.log_every == 0:
            print(f"step {it:5d} lr {lr:.2e} loss {float(loss):.4f} parts {parts.tolist()}")
    torch.cuda.synchronize(net.device)
    return TrainResult(steps, steps * data.crops_per_batch, time.perf_counter() - t0,
                       hist.cpu().numpy())


def _train_graphed(net, cfg, data, steps, opt, hist) -> TrainResult:
    dev = net.device
    stream = torch.cuda.Stream(dev)
    stream.wait_stream(torch.cuda.current_stream(dev))
    step, graph = None, None
    with torch.cuda.stream(stream):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for it in range(steps):
            x, tgt, mask = data.next()
            if step is None:
                step = _GraphedStep(net, opt, cfg, steps, x, tgt, mask)
            else:
                step.load(x, tgt, mask)
            if it < max(cfg.warmup_steps, 1):  # eager before the capture
                step()
            else:
                if graph is None:
                    graph = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(graph, stream=stream):
                        step()
                graph.replay()
            hist[it] = step.out
            if cfg.log_every and it % cfg.log_every == 0:
                print(f"step {it:5d} loss {float(step.out[0]):.4f}")
        torch.cuda.synchronize(dev)
        seconds = time.perf_counter() - t0
    torch.cuda.current_stream(dev).wait_stream(stream)
    return TrainResult(steps, steps * data.crops_per_batch, seconds, hist.cpu().numpy())


@torch.no_grad()
def predict(net: WarmStartNet, images: torch.Tensor) -> dict:
    """Denormalised predictions for (S, 2, H, W) images: per-cell heat
    probability, T, dn and dn T ([S][H/8][W/8]) and the image-wide defocus,
    NA, shear length and mean dn ([S])."""
    out, _ = net.forward(pack_input(images))
    glob = out[..., [CH_DEFOCUS, CH_NA, CH_SHEAR, CH_MEAN_DN]].mean(dim=(1, 2))
    return {"heat": torch.sigmoid(out[..., CH_HEAT]), "T": _denorm("T", out[..., CH_T]),
            "dn": _denorm("dn", out[..., CH_DN]), "opd": _denorm("opd", out[..., CH_OPD]),
            "defocus": _denorm("defocus", glob[:, 0]), "NA": _denorm("NA", glob[:, 1]),
            "shear_px": _denorm("shear", glob[:, 2]), "mean_dn": _denorm("dn", glob[:, 3])}


@torch.no_grad()
def evaluate(net: WarmStartNet, renderer, batches: int = 4, seed: int = 12345,
             scenes_per_batch: int = 16, crop: int = 256) -> dict:
    """Errors of the network on held-out rendered crops next to those of the
    prior (predicting each quantity's training-distribution mean): RMS
    errors of T, dn and dn T at centre cells, of defocus, NA and shear per
    crop, and the centre-cell detection rate at heat > 0.5."""
    data = RenderStream(renderer, scenes_per_batch, crop, seed)
    acc = {}

    def add(key, err):
        acc.setdefault(key, []).append(err.reshape(-1).double().cpu())

    for _ in range(batches):
        x, tgt, mask = data.next()
        out, _ = net.forward(x)
        m = mask
        for ch, key in ((CH_T, "T"), (CH_DN, "dn"), (CH_OPD, "opd")):
            scale = NORM[key][1]
            add(key, (out[..., ch][m] - tgt[..., ch][m]) * scale)
            add(key + "_prior", tgt[..., ch][m] * scale)
        g = out[..., [CH_DEFOCUS, CH_NA, CH_SHEAR]].mean(dim=(1, 2))
        for i, (ch, key) in enumerate(((CH_DEFOCUS, "defocus"), (CH_NA, "NA"), (CH_SHEAR, "shear"))):
            scale = NORM[key][1]
            add(key, (g[:, i] - tgt[:, 0, 0, ch]) * scale)
            add(key + "_prior", tgt[:, 0, 0, ch] * scale)
        hit = (torch.sigmoid(out[..., CH_HEAT]) > 0.5)
        add("recall", hit[m].float())
        add("false_pos", hit[~m].float())
    res = {}
    for k, v in acc.items():
        v = torch.cat(v)
        res[k] = float(v.mean()) if k in ("recall", "false_pos") else float(torch.sqrt((v * v).mean()))
    return res


def calibrate(net: WarmStartNet, renderer, batches: int = 4) -> dict:
    """Store the network's held-out RMS errors (evaluate()) in net.sigma;
    warm_start weighs its estimates by them."""
    ev = evaluate(net, renderer, batches)
    net.sigma = {k: ev[k] for k in ("T", "dn", "opd", "defocus", "NA", "shear")}
    return ev


def _fuse(a, sa, b, sb):
    """Inverse-variance weighted mean of two independent estimates."""
    wa, wb = 1.0 / (sa * sa), 1.0 / (sb * sb)
    return (wa * a + wb * b) / (wa + wb)


GUESS_REL_SIGMA = 0.2 / math.sqrt(3.0)  # a factor U(0.8, 1.2)


def warm_start(net: WarmStartNet, image: torch.Tensor, soa_guess: np.ndarray, optics_guess: dict,
               guess_rel_sigma: float = GUESS_REL_SIGMA):
    """Initial values for the inverse solve from the (K=2, H, W) image.

    Each particle's T and optical path dn T are read at the cell holding its
    guessed centre and the defocus and shear length from the image-wide
    channels; every one is combined with the guess by inverse-variance
    weighting, the network's variances being its held-out errors
    (calibrate()) and the guess's a relative spread guess_rel_sigma (dn T:
    sqrt(2) times that; defocus: relative to max(|dz|, 1 um)).  dn is the
    combined dn T over the combined T.  Centres, angles and the fixed
    particle properties keep the guess."""
    if getattr(net, "sigma", None) is None:
        raise RuntimeError("calibrate() the network before warm_start()")
    sg = net.sigma
    p = predict(net, image[None])
    g = p["T"].shape[1:]
    cx = np.clip((soa_guess[0] // CELL).astype(np.int64), 0, g[1] - 1)
    cy = np.clip((soa_guess[1] // CELL).astype(np.int64), 0, g[0] - 1)
    idx = torch.from_numpy(cy * g[1] + cx).to(image.device)
    T_n = p["T"][0].reshape(-1)[idx].double().cpu().numpy()
    opd_n = p["opd"][0].reshape(-1)[idx].double().cpu().numpy()
    T_g = soa_guess[5].astype(np.float64)
    opd_g = T_g * soa_guess[6]
    T = np.clip(_fuse(T_g, guess_rel_sigma * T_g, T_n, sg["T"]), 0.05, None)
    opd = np.clip(_fuse(opd_g, math.sqrt(2.0) * guess_rel_sigma * opd_g, opd_n, sg["opd"]),
                  1e-5, None)
    soa = soa_guess.copy()
    soa[5] = T.astype(np.float32)
    soa[6] = (opd / T).astype(np.float32)
    o = dict(optics_guess)
    dz = float(optics_guess["defocus"])
    o["defocus"] = float(_fuse(dz, guess_rel_sigma * max(abs(dz), 1.0), float(p["defocus"][0]),
                               sg["defocus"]))
    sh = float(optics_guess["shear_px"])
    o["shear_px"] = float(_fuse(sh, guess_rel_sigma * sh, float(p["shear_px"][0]), sg["shear"]))
    return soa, o
