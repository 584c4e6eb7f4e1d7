"""Differentiable inverse rendering (the paper's DiffOSOG, Sec. IV.B), driven
by the hand-written adjoint.

Given target images of a scene, recover each particle's dn, thickness T,
centre and orientation plus the global defocus and DIC shear by gradient
descent on the image misfit, starting from perturbed guesses.  As in the
paper's curriculum (coarse structure first, then detail), the misfit is
taken through a low-pass filter whose cut-off rises from a small numerical
aperture to the objective's over the first part of the run; both the model
and the target images pass through the same filter.

The render, its gradient and the image losses with their gradients run in
libosog's kernels; Adam and the curriculum schedule are plain torch on the
device.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from .autograd import OPTICS_PARAMS, render
from .render import Renderer

# particle-tensor rows the solver updates: cx, cy, theta, T, dn
FREE_ROWS = (0, 1, 2, 5, 6)


@dataclass
class SolveConfig:
    steps: int = 500
    na_start: float = 0.1            # curriculum: low-pass cut-off at step 0 (NA units)
    curriculum_frac: float = 0.6     # fraction of steps over which the cut-off rises
    lr_pos: float = 0.05             # px
    lr_theta: float = 0.01           # rad
    lr_T: float = 0.01               # um
    lr_dn: float = 4e-4
    lr_defocus: float = 0.02         # um
    lr_shear: float = 0.01           # px
    betas: tuple = (0.9, 0.99)
    log_every: int = 0
    spectral_weight: float = 0.0     # weight of the log-amplitude spectral loss (Eq. 8)
    record_every: int = 0            # with a ground truth: error history every n steps
    # "graph": every step on the device, replayed as one CUDA graph after a
    # few eager warm-up steps; "device": the same step launched eagerly;
    # "autograd": torch autograd through autograd.render with the optics
    # scalars on the host (one device-to-host read per step)
    mode: str = "graph"
    warmup_steps: int = 3            # eager steps before the graph is captured
    # device modes: every checkpoint_every steps the solve state is handed to
    # on_checkpoint(state) (see SolveState; 0 = never)
    checkpoint_every: int = 0


@dataclass
class SolveState:
    """Everything the device-resident solve carries from one step to the
    next, as host tensors: the particle tensor, the four optics scalars,
    Adam's moments of both, the step counter (which also sets the
    curriculum's cut-off) and the losses so far.  solve(..., resume=state)
    continues from it bit for bit (same configuration, target and renderer
    size)."""
    step: int
    tensors: dict

    def save(self, path: str) -> None:
        torch.save({"step": self.step, "tensors": self.tensors}, path)

    @staticmethod
    def load(path: str) -> "SolveState":
        d = torch.load(path, map_location="cpu")
        return SolveState(step=int(d["step"]), tensors=d["tensors"])


@dataclass
class SolveResult:
    soa: np.ndarray                  # recovered particle tensor (9, n)
    optics_params: np.ndarray        # recovered (defocus, shear_px, shear_angle, bias)
    losses: list = field(default_factory=list)
    seconds: float = 0.0
    steps: int = 0
    # (step, seconds since start, median rel. dn error, median rel. T error,
    #  fraction of particles with dn and T within 1%)
    history: list = field(default_factory=list)


class ImageLoss:
    """The solve's loss of images against the target, on the GPU
    (osog_image_loss): the squared misfit of the images low-passed at the
    curriculum's cut-off, summed over pixels and divided by the target's
    pixel count, plus spectral_weight times the log-amplitude spectral loss
    of Eq. 8.  The target's spectra are computed once; the cut-off
    (cycles/um) is a device scalar that the step updates in place, so the
    step stays capturable as a CUDA graph.  __call__ returns the device
    loss (2,) = [misfit, spectral] and dL/dimage, both in buffers of this
    object (overwritten by the next call)."""

    def __init__(self, renderer: Renderer, target: torch.Tensor, dx: float,
                 spectral_weight: float = 0.0, eps_rel: float = 1e-4):
        self.r = renderer
        self.target = target.contiguous()
        self.dx = float(dx)
        self.spectral_weight = float(spectral_weight)
        self.eps_rel = float(eps_rel)
        self.scale = 1.0 / float(target.numel())
        self.table = renderer.loss_target(self.target)
        dev = renderer.device
        self.cutoff = torch.zeros(1, dtype=torch.float32, device=dev)
        self.loss = torch.empty(2, dtype=torch.float32, device=dev)
        self.grad = torch.empty_like(self.target)

    def __call__(self, img: torch.Tensor):
        return self.r.image_loss(img.contiguous(), self.table, self.dx, self.cutoff,
                                 misfit_scale=self.scale, spectral_weight=self.spectral_weight,
                                 eps_rel=self.eps_rel, loss=self.loss, grad=self.grad)

    def total(self) -> torch.Tensor:
        """misfit + spectral_weight * spectral of the last call (device scalar)."""
        return self.loss[0] + self.spectral_weight * self.loss[1]


class _ImageLossFunction(torch.autograd.Function):
    """ImageLoss as a differentiable function of the image (autograd mode)."""

    @staticmethod
    def forward(ctx, img, loss_fn: ImageLoss):
        loss, grad = loss_fn(img)
        ctx.save_for_backward(grad.clone())
        return loss_fn.total().clone()

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g, None


def spectral_loss(img: torch.Tensor, target: torch.Tensor, renderer: Renderer,
                  eps_rel: float = 1e-4) -> torch.Tensor:
    """Eq. 8 of (K, H, W) images against a target on the GPU: the mean over
    frequencies of (log(|F(img)| + e) - log(|F(target)| + e))^2 with e =
    eps_rel times the target's largest amplitude per image (device scalar)."""
    fn = ImageLoss(renderer, target, 1.0, spectral_weight=1.0, eps_rel=eps_rel)
    loss, _ = renderer.image_loss(img.contiguous(), fn.table, 1.0, None, spectral_weight=1.0,
                                  eps_rel=eps_rel, want_grad=False)
    return loss[1]


def perturb(soa: np.ndarray, optics: dict, rng: np.random.Generator, frac: float = 0.2):
    """Initial guess: dn, T multiplied by U(1 - frac, 1 + frac); centres moved
    by up to frac times the mean semi-axis; angles by up to frac rad; the
    defocus and shear length multiplied likewise."""
    s = soa.copy()
    n = s.shape[1]
    for row in (5, 6):
        s[row] *= rng.uniform(1 - frac, 1 + frac, n).astype(np.float32)
    r = 0.5 * (s[3] + s[4])
    for row in (0, 1):
        s[row] += (rng.uniform(-frac, frac, n) * r).astype(np.float32)
    s[2] += rng.uniform(-frac, frac, n).astype(np.float32)
    o = dict(optics)
    o["defocus"] = optics["defocus"] * rng.uniform(1 - frac, 1 + frac) if optics["defocus"] else \
        rng.uniform(-frac, frac)
    o["shear_px"] = optics["shear_px"] * rng.uniform(1 - frac, 1 + frac)
    return s, o


def _device_errors(x: torch.Tensor, truth: torch.Tensor) -> torch.Tensor:
    rel_dn = (x[6] - truth[6]).abs() / truth[6].abs()
    rel_T = (x[5] - truth[5]).abs() / truth[5].abs()
    within = ((rel_dn <= 0.01) & (rel_T <= 0.01)).float().mean()
    return torch.stack([rel_dn.median(), rel_T.median(), within])


class _DeviceStep:
    """One solve step with all of its state on the device: the render with
    the forward intermediates kept (osog_render_keep), the curriculum misfit
    and its gradient with respect to the image (torch autograd on the
    misfit alone), the adjoint (osog_render_backward_kept), and Adam on the
    free particle rows and on defocus and shear.  The four optics scalars
    are a device tensor bound to the plan, so the step reads no value back
    to the host and can be captured as a CUDA graph.  The step counter, the
    curriculum cut-off and the Adam bias corrections are device scalars
    too."""

    def __init__(self, target, soa0, optics0, renderer, cfg, fixed_optics):
        dev = renderer.device
        self.r, self.cfg, self.target = renderer, cfg, target
        self.o = dict(optics0)
        self.x = torch.from_numpy(np.ascontiguousarray(soa0, dtype=np.float32)).to(dev)
        self.free = torch.zeros_like(self.x, dtype=torch.bool)
        self.free[list(FREE_ROWS)] = True
        self.lr = torch.zeros_like(self.x)
        self.lr[0] = self.lr[1] = cfg.lr_pos
        self.lr[2] = cfg.lr_theta
        self.lr[5] = cfg.lr_T
        self.lr[6] = cfg.lr_dn
        self.params = torch.tensor([float(optics0[k]) for k in OPTICS_PARAMS],
                                   dtype=torch.float32, device=dev)
        self.plr = torch.tensor([0.0 if fixed_optics else cfg.lr_defocus,
                                 0.0 if fixed_optics else cfg.lr_shear, 0.0, 0.0],
                                dtype=torch.float32, device=dev)
        self.m1, self.m2 = torch.zeros_like(self.x), torch.zeros_like(self.x)
        self.p1, self.p2 = torch.zeros_like(self.params), torch.zeros_like(self.params)
        self.t = torch.zeros((), dtype=torch.float32, device=dev)
        self.losses = torch.zeros(max(cfg.steps, 1), dtype=torch.float32, device=dev)
        K, H, W = target.shape
        self.loss_fn = ImageLoss(renderer, target, optics0["dx"], cfg.spectral_weight)
        self.ramp = float(max(1, int(cfg.steps * cfg.curriculum_frac)))
        self.img = torch.empty((K, H, W), dtype=torch.float32, device=dev)
        self.ws = torch.empty(renderer.backward_workspace_size(self.x.shape[1], K),
                              dtype=torch.uint8, device=dev)

    _STATE = ("x", "params", "m1", "m2", "p1", "p2", "t", "losses")

    def state(self) -> SolveState:
        """A copy of the step's state on the host (synchronises)."""
        return SolveState(step=int(self.t.item()),
                          tensors={k: getattr(self, k).detach().cpu().clone() for k in self._STATE})

    def load_state(self, st: SolveState) -> None:
        """Restore a state in place (the buffers a captured graph refers to)."""
        for k in self._STATE:
            dst, src = getattr(self, k), st.tensors[k]
            if dst.shape != src.shape or dst.dtype != src.dtype:
                raise ValueError(f"solve state field {k} does not match this solve")
            dst.copy_(src.to(dst.device))

    def __call__(self) -> None:
        cfg, o = self.cfg, self.o
        b1, b2 = cfg.betas
        na = cfg.na_start + (o["NA"] - cfg.na_start) * torch.clamp(self.t / self.ramp, max=1.0)
        self.loss_fn.cutoff.copy_((2.0 / o["lambda_um"]) * na)
        self.r.render_keep(self.x, None, o, out=self.img, ws=self.ws)
        _, g_img = self.loss_fn(self.img)
        loss = self.loss_fn.total()
        gx, gp = self.r.backward_kept(self.x, None, o, g_img, self.ws)
        t1 = self.t + 1.0
        c1, c2 = 1.0 - torch.pow(b1, t1), 1.0 - torch.pow(b2, t1)
        self.m1.mul_(b1).add_(gx, alpha=1 - b1)
        self.m2.mul_(b2).addcmul_(gx, gx, value=1 - b2)
        step = self.lr * (self.m1 / c1) / (torch.sqrt(self.m2 / c2) + 1e-30)
        self.x.sub_(torch.where(self.free, step, torch.zeros_like(step)))
        self.x[5].clamp_(min=1e-3)
        self.p1.mul_(b1).add_(gp, alpha=1 - b1)
        self.p2.mul_(b2).addcmul_(gp, gp, value=1 - b2)
        self.params.sub_(self.plr * (self.p1 / c1) / (torch.sqrt(self.p2 / c2) + 1e-30))
        self.losses.index_copy_(0, self.t.long().view(1), loss.detach().view(1))
        self.t.copy_(t1)


def _solve_device(target, soa0, optics0, renderer, cfg, fixed_optics, truth, resume,
                  on_checkpoint) -> SolveResult:
    dev = renderer.device
    st = _DeviceStep(target, soa0, optics0, renderer, cfg, fixed_optics)
    first = 0
    if resume is not None:
        st.load_state(resume)
        first = resume.step
        if not 0 <= first <= cfg.steps:
            raise ValueError("the resumed state's step lies outside this configuration's steps")
    res = SolveResult(soa=None, optics_params=None)
    truth_d = None
    if truth is not None and cfg.record_every:
        truth_d = torch.from_numpy(np.ascontiguousarray(truth, dtype=np.float32)).to(dev)
    stream = torch.cuda.Stream(dev)
    stream.wait_stream(torch.cuda.current_stream(dev))
    renderer.bind_optics_params(st.params)
    try:
        with torch.cuda.stream(stream):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            if truth_d is not None:
                res.history.append((0, 0.0, *_device_errors(st.x, truth_d).tolist()))
            # at least one eager step before the capture (plans and kernels
            # must exist before a graph can record them)
            eager = cfg.steps if cfg.mode == "device" else min(max(cfg.warmup_steps, 1), cfg.steps)
            graph = None
            for it in range(first, cfg.steps):
                if it < first + eager:
                    st()
                else:
                    if graph is None:
                        graph = torch.cuda.CUDAGraph()
                        with torch.cuda.graph(graph, stream=stream):
                            st()
                    graph.replay()
                if truth_d is not None and (it + 1) % cfg.record_every == 0:
                    e = _device_errors(st.x, truth_d).tolist()
                    res.history.append((it + 1, time.perf_counter() - t0, *e))
                if on_checkpoint is not None and cfg.checkpoint_every and \
                        (it + 1) % cfg.checkpoint_every == 0:
                    on_checkpoint(st.state())
            torch.cuda.synchronize(dev)
            res.seconds = time.perf_counter() - t0
    finally:
        renderer.bind_optics_params(None)
    torch.cuda.current_stream(dev).wait_stream(stream)
    res.steps = cfg.steps
    res.losses = st.losses[:cfg.steps].cpu().tolist()
    res.soa = st.x.cpu().numpy()
    res.optics_params = st.params.cpu().double().numpy()
    return res


def solve(target: torch.Tensor, soa0: np.ndarray, optics0: dict, renderer: Renderer,
          cfg: SolveConfig | None = None, fixed_optics: bool = False,
          truth: np.ndarray | None = None, resume: SolveState | None = None,
          on_checkpoint=None) -> SolveResult:
    """Adam on the curriculum-filtered squared image misfit.  target is the
    (K, H, W) measured image; soa0 / optics0 the initial guess.  With the
    true particle tensor and cfg.record_every > 0 the error history is
    recorded (the clock keeps running across the records).  cfg.mode picks
    the device-resident step (CUDA graph or eager) or the autograd loop.
    In the device modes, on_checkpoint(state) receives a SolveState every
    cfg.checkpoint_every steps, and resume=state continues a solve from one
    (the same cfg, target, guess and renderer size)."""
    cfg = cfg or SolveConfig()
    if cfg.mode in ("graph", "device"):
        return _solve_device(target, soa0, optics0, renderer, cfg, fixed_optics, truth, resume,
                             on_checkpoint)
    if resume is not None or on_checkpoint is not None:
        raise ValueError("checkpoints are taken in the device modes ('graph', 'device')")
    if cfg.mode != "autograd":
        raise ValueError("SolveConfig.mode must be 'graph', 'device' or 'autograd'")
    dev = renderer.device
    soa = torch.from_numpy(np.ascontiguousarray(soa0, dtype=np.float32)).to(dev)
    free = torch.zeros_like(soa, dtype=torch.bool)
    free[list(FREE_ROWS)] = True
    x = soa.clone().requires_grad_(True)
    params = torch.tensor([float(optics0[k]) for k in OPTICS_PARAMS], dtype=torch.float64,
                          requires_grad=not fixed_optics)
    lr = torch.zeros_like(soa)
    lr[0] = lr[1] = cfg.lr_pos
    lr[2] = cfg.lr_theta
    lr[5] = cfg.lr_T
    lr[6] = cfg.lr_dn
    plr = torch.tensor([cfg.lr_defocus, cfg.lr_shear, 0.0, 0.0], dtype=torch.float64)
    m1, m2 = torch.zeros_like(soa), torch.zeros_like(soa)
    p1, p2 = torch.zeros_like(params), torch.zeros_like(params)
    b1, b2 = cfg.betas
    res = SolveResult(soa=None, optics_params=None)
    truth_d = None
    if truth is not None and cfg.record_every:
        truth_d = torch.from_numpy(np.ascontiguousarray(truth, dtype=np.float32)).to(dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    if truth_d is not None:
        res.history.append((0, 0.0, *_device_errors(x.detach(), truth_d).tolist()))
    ramp = max(1, int(cfg.steps * cfg.curriculum_frac))
    loss_fn = ImageLoss(renderer, target, optics0["dx"], cfg.spectral_weight)
    for it in range(cfg.steps):
        na = cfg.na_start + (optics0["NA"] - cfg.na_start) * min(1.0, it / ramp)
        img = render(x, optics0, renderer, params)
        loss_fn.cutoff.fill_(2.0 * na / optics0["lambda_um"])
        loss = _ImageLossFunction.apply(img, loss_fn)
        gx, gp = torch.autograd.grad(loss, (x, params), allow_unused=True)
        with torch.no_grad():
            t = it + 1
            m1.mul_(b1).add_(gx, alpha=1 - b1)
            m2.mul_(b2).addcmul_(gx, gx, value=1 - b2)
            step = lr * (m1 / (1 - b1 ** t)) / (torch.sqrt(m2 / (1 - b2 ** t)) + 1e-30)
            x.sub_(torch.where(free, step, torch.zeros_like(step)))
            x[5].clamp_(min=1e-3)
            if gp is not None and not fixed_optics:
                gp = gp.cpu()
                p1.mul_(b1).add_(gp, alpha=1 - b1)
                p2.mul_(b2).addcmul_(gp, gp, value=1 - b2)
                params.sub_(plr * (p1 / (1 - b1 ** t)) / (torch.sqrt(p2 / (1 - b2 ** t)) + 1e-30))
        res.losses.append(loss.detach())
        if truth_d is not None and (it + 1) % cfg.record_every == 0:
            e = _device_errors(x.detach(), truth_d).tolist()
            res.history.append((it + 1, time.perf_counter() - t0, *e))
        if cfg.log_every and it % cfg.log_every == 0:
            print(f"step {it:4d} NA {na:.3f} loss {float(loss):.3e}")
    torch.cuda.synchronize(dev)
    res.seconds = time.perf_counter() - t0
    res.steps = cfg.steps
    res.losses = [float(v) for v in torch.stack(res.losses).cpu()] if res.losses else []
    res.soa = x.detach().cpu().numpy()
    res.optics_params = params.detach().numpy()
    return res


def time_to_error(history: list, tol: float = 0.01):
    """(step, seconds) of the first record at which the median relative dn
    and T errors are both <= tol; None if never."""
    for step, sec, dn, T, _ in history:
        if dn <= tol and T <= tol:
            return step, sec
    return None


def errors(est: np.ndarray, truth: np.ndarray, est_params=None, truth_optics=None) -> dict:
    """Recovery errors: median relative error of dn, T and dn T; median
    centre error (px); median angle error (rad, modulo pi); the fraction of
    particles with both dn and T within 1%; defocus (um) and relative shear
    errors when the optics are given."""
    d = {}
    d["dn_rel_median"] = float(np.median(np.abs(est[6] - truth[6]) / np.abs(truth[6])))
    d["T_rel_median"] = float(np.median(np.abs(est[5] - truth[5]) / np.abs(truth[5])))
    d["dnT_rel_median"] = float(np.median(np.abs(est[6] * est[5] - truth[6] * truth[5])
                                          / np.abs(truth[6] * truth[5])))
    d["centre_px_median"] = float(np.median(np.hypot(est[0] - truth[0], est[1] - truth[1])))
    dth = np.abs((est[2] - truth[2] + math.pi / 2) % math.pi - math.pi / 2)
    d["theta_rad_median"] = float(np.median(dth))
    d["frac_dn_T_within_1pct"] = float(np.mean((np.abs(est[6] - truth[6]) <= 0.01 * np.abs(truth[6]))
                                               & (np.abs(est[5] - truth[5]) <= 0.01 * np.abs(truth[5]))))
    if est_params is not None and truth_optics is not None:
        d["defocus_abs"] = float(abs(est_params[0] - truth_optics["defocus"]))
        d["shear_rel"] = float(abs(est_params[1] - truth_optics["shear_px"]) / truth_optics["shear_px"])
    return d
