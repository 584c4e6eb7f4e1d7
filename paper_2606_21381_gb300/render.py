"""Torch-facing wrapper of libosog: plans, workspaces, device tensors.

PyTorch provides device memory and the current CUDA stream; every step of
the render runs in libosog's kernels, reached through the C ABI in
``_lib``.  There is no CPU path: constructing a :class:`Renderer` without a
CUDA device raises.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import LossParams, OsogError, Optics, Tuning, check, optics_struct


def n_modes(optics: dict) -> int:
    return bin(int(optics["modes"]) & 7).count("1")


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Renderer:
    """A plan for H x W canvases plus a growable device workspace."""

    def __init__(self, H: int, W: int, device: torch.device | str | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("libosog renders on a CUDA device; none is available")
        self.device = torch.device(device or "cuda")
        self.H, self.W = int(H), int(W)
        self._L = _lib.lib()
        self.plan = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self._L.osog_plan_create(ctypes.byref(self.plan), self.H, self.W),
                  "osog_plan_create")
        self._ws = None

    def close(self) -> None:
        if self.plan:
            torch.cuda.synchronize(self.device)
            self._L.osog_plan_destroy(self.plan)
            self.plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ workspace
    def workspace_size(self, n: int, K: int, batch: int = 1) -> int:
        b = self._L.osog_workspace_size(self.plan, int(n), int(K), int(batch))
        if b == 0:
            raise OsogError(1, "osog_workspace_size")
        return int(b)

    def workspace(self, nbytes: int) -> torch.Tensor:
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def _check_soa(self, soa: torch.Tensor) -> None:
        if soa.device.type != "cuda" or soa.dtype != torch.float32 or soa.dim() != 2 \
                or soa.shape[0] != 9 or not soa.is_contiguous():
            raise ValueError("soa must be a contiguous cuda float32 tensor of shape (9, ld)")

    # ------------------------------------------------------------ entry points
    def render(self, soa: torch.Tensor, n: int | None, optics: dict, out=None, stream=None):
        """osog_render: (K, H, W) float32 image of one scene."""
        self._check_soa(soa)
        n = soa.shape[1] if n is None else int(n)
        K = n_modes(optics)
        if out is None:
            out = torch.empty((K, self.H, self.W), dtype=torch.float32, device=self.device)
        ws = self.workspace(self.workspace_size(n, K, 1))
        o = optics_struct(optics)
        check(self._L.osog_render(self.plan, _ptr(soa), soa.shape[1], n, ctypes.byref(o),
                                  _ptr(out), _ptr(ws), ws.numel(), _stream(stream)),
              "osog_render")
        return out

    def render_dic_incoherent(self, soa: torch.Tensor, n: int | None, optics: dict, out=None,
                              stream=None):
        """osog_render_dic_incoherent: (H, W) DIC image in the literal
        reading of Eq. 5 (sheared exit wave, intensity blurred by |h|^2)."""
        self._check_soa(soa)
        n = soa.shape[1] if n is None else int(n)
        if out is None:
            out = torch.empty((self.H, self.W), dtype=torch.float32, device=self.device)
        ws = self.workspace(self._L.osog_dic_incoherent_workspace_size(self.plan, n))
        o = optics_struct(optics)
        check(self._L.osog_render_dic_incoherent(self.plan, _ptr(soa), soa.shape[1], n,
                                                 ctypes.byref(o), _ptr(out), _ptr(ws),
                                                 ws.numel(), _stream(stream)),
              "osog_render_dic_incoherent")
        return out

    def render_polyhedra(self, soa: torch.Tensor, n: int | None, planes: torch.Tensor,
                         plane_offsets: torch.Tensor, optics: dict, out=None, stream=None):
        """osog_render_polyhedra: one scene with general polyhedra (kind 2)
        whose half-spaces are the rows (a_x, a_y, a_z, b) of planes
        (float32 (P, 4)), particle p owning rows plane_offsets[p] ..
        plane_offsets[p+1]-1 (int32 (n + 1,))."""
        self._check_soa(soa)
        n = soa.shape[1] if n is None else int(n)
        if planes.device.type != "cuda" or planes.dtype != torch.float32 or planes.dim() != 2 \
                or planes.shape[1] != 4 or not planes.is_contiguous():
            raise ValueError("planes must be a contiguous CUDA float32 (P, 4) tensor")
        if plane_offsets.device.type != "cuda" or plane_offsets.dtype != torch.int32 \
                or plane_offsets.shape != (n + 1,):
            raise ValueError("plane_offsets must be a CUDA int32 (n + 1,) tensor")
        K = n_modes(optics)
        if out is None:
            out = torch.empty((K, self.H, self.W), dtype=torch.float32, device=self.device)
        P = planes.shape[0]
        ws = self.workspace(self._L.osog_polyhedra_workspace_size(self.plan, n, K, P))
        o = optics_struct(optics)
        check(self._L.osog_render_polyhedra(self.plan, _ptr(soa), soa.shape[1], n, _ptr(planes),
                                            _ptr(plane_offsets), P, ctypes.byref(o), _ptr(out),
                                            _ptr(ws), ws.numel(), _stream(stream)),
              "osog_render_polyhedra")
        return out

    def backward(self, soa: torch.Tensor, n: int | None, optics: dict, grad_image: torch.Tensor,
                 stream=None):
        """osog_render_backward: (dL/dsoa (9, ld), dL/d(defocus, shear_px,
        shear_angle, bias_phase) (4,)) for grad_image = dL/dI of shape (K, H, W)."""
        self._check_soa(soa)
        n = soa.shape[1] if n is None else int(n)
        K = n_modes(optics)
        if grad_image.shape != (K, self.H, self.W) or grad_image.dtype != torch.float32 \
                or not grad_image.is_contiguous() or grad_image.device.type != "cuda":
            raise ValueError("grad_image must be a contiguous cuda float32 (K, H, W) tensor")
        gsoa, gopt = self._grad_buffers(soa, n)
        ws = self.workspace(self.backward_workspace_size(n, K))
        o = optics_struct(optics)
        check(self._L.osog_render_backward(self.plan, _ptr(soa), soa.shape[1], n, ctypes.byref(o),
                                           _ptr(grad_image), _ptr(gsoa), _ptr(gopt), _ptr(ws),
                                           ws.numel(), _stream(stream)),
              "osog_render_backward")
        return gsoa, gopt

    def backward_workspace_size(self, n: int, K: int) -> int:
        nbytes = int(self._L.osog_backward_workspace_size(self.plan, int(n), int(K)))
        if nbytes == 0:
            raise OsogError(1, "osog_backward_workspace_size")
        return nbytes

    def _grad_buffers(self, soa: torch.Tensor, n: int):
        # the adjoint writes every row of particles 0..n-1 and all four optics
        # entries; only the columns n..ld-1 need zeros
        gsoa = torch.empty_like(soa) if n == soa.shape[1] else torch.zeros_like(soa)
        gopt = torch.empty(4, dtype=torch.float32, device=self.device)
        return gsoa, gopt

    def render_keep(self, soa: torch.Tensor, n: int | None, optics: dict, out=None, ws=None,
                    stream=None):
        """osog_render_keep: the (K, H, W) image of render(), with the
        forward intermediates kept in `ws` (a uint8 device tensor, allocated
        when None) for one backward_kept().  Returns (image, ws)."""
        self._check_soa(soa)
        n = soa.shape[1] if n is None else int(n)
        K = n_modes(optics)
        if out is None:
            out = torch.empty((K, self.H, self.W), dtype=torch.float32, device=self.device)
        nbytes = self.backward_workspace_size(n, K)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        o = optics_struct(optics)
        check(self._L.osog_render_keep(self.plan, _ptr(soa), soa.shape[1], n, ctypes.byref(o),
                                       _ptr(out), _ptr(ws), ws.numel(), _stream(stream)),
              "osog_render_keep")
        return out, ws

    def backward_kept(self, soa: torch.Tensor, n: int | None, optics: dict,
                      grad_image: torch.Tensor, ws: torch.Tensor, stream=None):
        """osog_render_backward_kept: backward() from the state that
        render_keep() left in `ws` (same soa, n and optics); consumes it."""
        self._check_soa(soa)
        n = soa.shape[1] if n is None else int(n)
        K = n_modes(optics)
        if grad_image.shape != (K, self.H, self.W) or grad_image.dtype != torch.float32 \
                or not grad_image.is_contiguous() or grad_image.device.type != "cuda":
            raise ValueError("grad_image must be a contiguous cuda float32 (K, H, W) tensor")
        gsoa, gopt = self._grad_buffers(soa, n)
        o = optics_struct(optics)
        check(self._L.osog_render_backward_kept(self.plan, _ptr(soa), soa.shape[1], n,
                                                ctypes.byref(o), _ptr(grad_image), _ptr(gsoa),
                                                _ptr(gopt), _ptr(ws), ws.numel(),
                                                _stream(stream)),
              "osog_render_backward_kept")
        return gsoa, gopt

    def render_opd(self, soa: torch.Tensor, n: int | None, optics: dict, out=None, stream=None):
        """osog_render_opd: (H, W, 2) float32 OPD / ATT map."""
        self._check_soa(soa)
        n = soa.shape[1] if n is None else int(n)
        if out is None:
            out = torch.empty((self.H, self.W, 2), dtype=torch.float32, device=self.device)
        ws = self.workspace(self.workspace_size(n, 1, 1))
        o = optics_struct(optics)
        check(self._L.osog_render_opd(self.plan, _ptr(soa), soa.shape[1], n, ctypes.byref(o),
                                      _ptr(out), _ptr(ws), ws.numel(), _stream(stream)),
              "osog_render_opd")
        return out

    def optics_from_opd(self, opd_att: torch.Tensor, optics: dict, out=None, stream=None):
        """osog_optics_from_opd: (K, H, W) images from an (H, W, 2) OPD/ATT map."""
        if opd_att.shape != (self.H, self.W, 2) or opd_att.dtype != torch.float32 \
                or not opd_att.is_contiguous() or opd_att.device.type != "cuda":
            raise ValueError("opd_att must be a contiguous cuda float32 (H, W, 2) tensor")
        K = n_modes(optics)
        if out is None:
            out = torch.empty((K, self.H, self.W), dtype=torch.float32, device=self.device)
        ws = self.workspace(self.workspace_size(0, K, 1))
        o = optics_struct(optics)
        check(self._L.osog_optics_from_opd(self.plan, _ptr(opd_att), ctypes.byref(o), _ptr(out),
                                           _ptr(ws), ws.numel(), _stream(stream)),
              "osog_optics_from_opd")
        return out

    def batch(self, soa_all: torch.Tensor, offsets, optics_list: list[dict], out=None,
              tuning: dict | None = None, stream=None):
        """osog_batch_submit: (S, K, H, W) images of S scenes."""
        self._check_soa(soa_all)
        offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
        S = len(optics_list)
        if offs.shape != (S + 1,):
            raise ValueError("offsets must have S + 1 entries")
        K = n_modes(optics_list[0])
        if out is None:
            out = torch.empty((S, K, self.H, self.W), dtype=torch.float32, device=self.device)
        n_total = int(offs[-1] - offs[0])
        t = Tuning()
        t.use_graph = 1
        if tuning:
            t.pairs_per_particle = int(tuning.get("pairs_per_particle", 0))
            t.use_graph = int(tuning.get("use_graph", 1))
            t.persistent = int(tuning.get("persistent", 0))
            t.band_rows = int(tuning.get("band_rows", 0))
            t.wait_polls = int(tuning.get("wait_polls", 0))
            t.test_wait_extra = int(tuning.get("test_wait_extra", 0))
            t.raster = int(tuning.get("raster", 0))
        need = self.workspace_size(n_total, K, S)
        if t.pairs_per_particle > 8:
            need = int(need * t.pairs_per_particle / 8) + (1 << 20)
        ws = self.workspace(need)
        arr = (Optics * S)(*[optics_struct(o) for o in optics_list])
        check(self._L.osog_batch_submit(
            self.plan, _ptr(soa_all), soa_all.shape[1],
            offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), S, arr, _ptr(out),
            ctypes.byref(t), _ptr(ws), ws.numel(), _stream(stream)), "osog_batch_submit")
        return out

    def autotune(self, soa_all: torch.Tensor, offsets, optics_list: list[dict], out=None,
                 stream=None) -> dict:
        """osog_autotune: time the batched path's candidate band heights and
        launch modes for this batch shape, keep the fastest in the plan and
        return it as a tuning dict."""
        self._check_soa(soa_all)
        offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
        S = len(optics_list)
        K = n_modes(optics_list[0])
        if out is None:
            out = torch.empty((S, K, self.H, self.W), dtype=torch.float32, device=self.device)
        ws = self.workspace(self.workspace_size(int(offs[-1] - offs[0]), K, S))
        arr = (Optics * S)(*[optics_struct(o) for o in optics_list])
        t = Tuning()
        check(self._L.osog_autotune(
            self.plan, _ptr(soa_all), soa_all.shape[1],
            offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), S, arr, _ptr(out),
            _ptr(ws), ws.numel(), _stream(stream), ctypes.byref(t)), "osog_autotune")
        return {"pairs_per_particle": t.pairs_per_particle, "use_graph": t.use_graph,
                "persistent": t.persistent, "band_rows": t.band_rows, "raster": t.raster}

    def render_host(self, soa_host: torch.Tensor, n: int, optics: dict,
                    image_host: torch.Tensor, stream=None):
        """End-to-end call from host buffers: copy the particle tensor in,
        render, copy the image out (pinned host tensors, stream ordered)."""
        dev = soa_host.to(self.device, non_blocking=True)
        img = self.render(dev, n, optics, stream=stream)
        image_host.copy_(img, non_blocking=True)
        return image_host

    def bind_optics_params(self, params: torch.Tensor | None) -> None:
        """osog_plan_bind_optics_params: every later call of this plan reads
        (defocus, shear_px, shear_angle, bias_phase) from `params` (a float32
        device tensor of 4) when its kernels run, instead of from the optics
        dict; None unbinds.  The renderer keeps a reference while bound."""
        if params is not None and (params.device.type != "cuda" or params.dtype != torch.float32
                                   or params.shape != (4,) or not params.is_contiguous()):
            raise ValueError("params must be a contiguous float32 CUDA tensor of shape (4,)")
        check(self._L.osog_plan_bind_optics_params(self.plan, _ptr(params)),
              "osog_plan_bind_optics_params")
        self._bound_params = params

    # ------------------------------------------------------------ bin reservation
    def set_pairs_per_particle(self, k: int) -> None:
        """osog_plan_set_pairs_per_particle: particle-band pairs reserved per
        particle by this renderer's calls (default 8)."""
        check(self._L.osog_plan_set_pairs_per_particle(self.plan, int(k)),
              "osog_plan_set_pairs_per_particle")

    def fit_pairs(self, soa: torch.Tensor, n: int | None = None) -> int:
        """Size the reservation for a particle tensor from its largest
        half-extent a + b (one device-to-host read); returns it."""
        self._check_soa(soa)
        n = soa.shape[1] if n is None else int(n)
        hh = float((soa[3, :n] + soa[4, :n]).max()) if n > 0 else 0.0
        k = max(1, int(self._L.osog_pairs_for_extent(self.plan, hh)))
        self.set_pairs_per_particle(k)
        return k

    # ------------------------------------------------------------ image losses
    def loss_target(self, target: torch.Tensor, stream=None) -> torch.Tensor:
        """osog_loss_target: the device table of the (K, H, W) target images'
        spectra and largest amplitudes that image_loss() compares with."""
        K = self._check_images(target, "target")
        table = torch.empty(self._L.osog_loss_table_size(self.plan, K), dtype=torch.uint8,
                            device=self.device)
        ws = self._loss_ws(K)
        check(self._L.osog_loss_target(self.plan, _ptr(target), K, _ptr(table), table.numel(),
                                       _ptr(ws), ws.numel(), _stream(stream)), "osog_loss_target")
        return table

    def image_loss(self, image: torch.Tensor, table: torch.Tensor, dx_um: float,
                   cutoff: torch.Tensor | None = None, misfit_scale: float = 0.0,
                   spectral_weight: float = 0.0, eps_rel: float = 1e-4, loss=None, grad=None,
                   want_grad: bool = True, stream=None):
        """osog_image_loss: (loss (2,) = [misfit, spectral], dL/dimage or
        None) for (K, H, W) images against the table of loss_target().
        `cutoff` is a float32 device scalar (cycles/um) read when the
        kernels run; the gradient is that of misfit + spectral_weight *
        spectral."""
        K = self._check_images(image, "image")
        if cutoff is not None and (cutoff.device.type != "cuda" or cutoff.dtype != torch.float32
                                   or cutoff.numel() != 1):
            raise ValueError("cutoff must be a float32 CUDA scalar tensor")
        if loss is None:
            loss = torch.empty(2, dtype=torch.float32, device=self.device)
        if want_grad and grad is None:
            grad = torch.empty_like(image)
        p = LossParams()
        p.dx_um, p.misfit_scale = float(dx_um), float(misfit_scale)
        p.spectral_weight, p.eps_rel = float(spectral_weight), float(eps_rel)
        p.cutoff = None if cutoff is None else cutoff.data_ptr()
        ws = self._loss_ws(K)
        check(self._L.osog_image_loss(self.plan, _ptr(image), K, _ptr(table), table.numel(),
                                      ctypes.byref(p), _ptr(loss),
                                      _ptr(grad) if want_grad else None, _ptr(ws), ws.numel(),
                                      _stream(stream)), "osog_image_loss")
        return loss, (grad if want_grad else None)

    def _check_images(self, t: torch.Tensor, what: str) -> int:
        if t.device.type != "cuda" or t.dtype != torch.float32 or t.dim() != 3 \
                or tuple(t.shape[1:]) != (self.H, self.W) or not t.is_contiguous():
            raise ValueError(f"{what} must be a contiguous cuda float32 (K, H, W) tensor")
        return int(t.shape[0])

    def _loss_ws(self, K: int) -> torch.Tensor:
        # a workspace of its own: the loss may run between a render_keep and
        # its backward_kept, whose state lives in the shared one
        need = int(self._L.osog_loss_workspace_size(self.plan, K))
        if getattr(self, "_lws", None) is None or self._lws.numel() < need:
            self._lws = torch.empty(need, dtype=torch.uint8, device=self.device)
        return self._lws

    # ------------------------------------------------------------ status / timing
    def sync_status(self, stream=None) -> int:
        return int(self._L.osog_sync_status(self.plan, _stream(stream)))

    def launch_count(self) -> int:
        return int(self._L.osog_plan_launch_count(self.plan))

    def profile_begin(self) -> None:
        check(self._L.osog_profile_begin(self.plan), "osog_profile_begin")

    def profile_end(self, stream=None) -> dict:
        nk = len(_lib.KERNEL_CLASSES)
        ms = (ctypes.c_float * nk)()
        cnt = (ctypes.c_int32 * nk)()
        check(self._L.osog_profile_end(self.plan, _stream(stream), ms, cnt), "osog_profile_end")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(_lib.KERNEL_CLASSES)}


class HostBatchPipeline:
    """Batches given in pinned host memory rendered into pinned host images,
    with each batch's copies overlapping the renders of its neighbours: two
    device slots, one stream for the renders, one for host-to-device copies
    and `out_streams` streams that copy parts of each image batch back in
    parallel (several copy engines), ordered by events.  submit() returns
    the events that mark the batch's images as copied to the host."""

    def __init__(self, renderer: Renderer, n_max: int, S: int, K: int, slots: int = 2,
                 out_streams: int = 4):
        dev = renderer.device
        self.r = renderer
        self.slots = slots
        self.render_stream = torch.cuda.Stream(dev)
        self.in_stream = torch.cuda.Stream(dev)
        self.out_streams = [torch.cuda.Stream(dev) for _ in range(max(1, min(out_streams, S)))]
        self.soa = [torch.empty((9, n_max), dtype=torch.float32, device=dev) for _ in range(slots)]
        self.out = [torch.empty((S, K, renderer.H, renderer.W), dtype=torch.float32, device=dev)
                    for _ in range(slots)]
        self.rendered = [None] * slots
        self.copied = [None] * slots
        self.count = 0

    def submit(self, soa_host: torch.Tensor, offsets, optics_list: list[dict],
               image_host: torch.Tensor, tuning: dict | None = None):
        k = self.count % self.slots
        self.count += 1
        n = soa_host.shape[1]
        if n > self.soa[k].shape[1]:
            raise ValueError("more particles than the pipeline was built for")
        if self.rendered[k] is not None:  # the slot's previous render has read soa[k]
            self.in_stream.wait_event(self.rendered[k])
        with torch.cuda.stream(self.in_stream):
            self.soa[k][:, :n].copy_(soa_host, non_blocking=True)
        loaded = torch.cuda.Event()
        loaded.record(self.in_stream)
        self.render_stream.wait_event(loaded)
        for ev in self.copied[k] or ():  # out[k] has reached the host
            self.render_stream.wait_event(ev)
        self.r.batch(self.soa[k], offsets, optics_list, out=self.out[k], tuning=tuning,
                     stream=self.render_stream)
        done = torch.cuda.Event()
        done.record(self.render_stream)
        self.rendered[k] = done
        S = self.out[k].shape[0]
        c = len(self.out_streams)
        copied = []
        for j, st in enumerate(self.out_streams):
            a, b = j * S // c, (j + 1) * S // c
            st.wait_event(done)
            with torch.cuda.stream(st):
                image_host[a:b].copy_(self.out[k][a:b], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
            copied.append(ev)
        self.copied[k] = copied
        return copied

    def synchronize(self) -> None:
        for s in (self.in_stream, self.render_stream, *self.out_streams):
            s.synchronize()
