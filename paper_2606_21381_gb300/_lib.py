"""ctypes binding of libosog (argument marshalling only).

Every function here maps one-to-one onto an ``extern "C"`` entry point of
``include/osog.h``; all computation happens in the CUDA library.  If the
library is missing or cannot be loaded, :func:`lib` raises: there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

MODE_BF, MODE_OBLIQUE, MODE_DIC = 1, 2, 4
KERNEL_CLASSES = ("bin_count", "bin_scan", "bin_fill", "strip_forward", "column",
                  "strip_inverse", "bwd_rows", "bwd_column", "bwd_strip", "bwd_reduce",
                  "persistent", "raster")
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED_SIZE", 3: "WORKSPACE",
          4: "BIN_OVERFLOW", 5: "NONFINITE_INPUT", 6: "TIMEOUT", 7: "CUDA",
          8: "INVALID_PARTICLE"}

EXPORTS = ("osog_plan_create", "osog_plan_destroy", "osog_workspace_size", "osog_render",
           "osog_render_opd", "osog_optics_from_opd", "osog_batch_submit",
           "osog_sync_status", "osog_last_error", "osog_plan_launch_count",
           "osog_profile_begin", "osog_profile_end", "osog_render_noalloc",
           "osog_noalloc_sync_status",
           "osog_backward_workspace_size", "osog_render_backward", "osog_render_keep",
           "osog_render_backward_kept", "osog_autotune",
           "osog_polyhedra_workspace_size", "osog_render_polyhedra",
           "osog_dic_incoherent_workspace_size", "osog_render_dic_incoherent",
           "osog_sensor_noise", "osog_plan_bind_optics_params",
           "osog_loss_table_size", "osog_loss_workspace_size", "osog_loss_target",
           "osog_image_loss", "osog_plan_set_pairs_per_particle", "osog_pairs_for_extent")


class OsogError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} {detail}".strip())


class Optics(ctypes.Structure):
    """Mirror of osog_optics_t."""
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("dx_um", ctypes.c_double), ("lambda_um", ctypes.c_double),
                ("NA", ctypes.c_double), ("n_medium", ctypes.c_double),
                ("defocus_um", ctypes.c_double), ("modes", ctypes.c_uint32),
                ("oblique_frac", ctypes.c_double), ("oblique_angle", ctypes.c_double),
                ("shear_px", ctypes.c_double), ("shear_angle", ctypes.c_double),
                ("bias_phase", ctypes.c_double), ("bevel_slope", ctypes.c_double)]


class ConvShape(ctypes.Structure):
    """Mirror of osog_conv_shape_t."""
    _fields_ = [(k, ctypes.c_int32) for k in ("N", "H", "W", "C", "K", "R", "S", "stride", "pad")]


CNN_EXPORTS = ("osog_conv_out_h", "osog_conv_out_w", "osog_conv2d_forward",
               "osog_conv2d_backward_data", "osog_conv2d_backward_filter_workspace",
               "osog_conv2d_backward_filter", "osog_relu_backward", "osog_conv_use_tcgen05",
               "osog_conv_sync_status", "osog_conv_test_wait_limit")


class LossParams(ctypes.Structure):
    """Mirror of osog_loss_t."""
    _fields_ = [("dx_um", ctypes.c_double), ("cutoff", ctypes.c_void_p),
                ("misfit_scale", ctypes.c_double), ("spectral_weight", ctypes.c_double),
                ("eps_rel", ctypes.c_double)]


class Tuning(ctypes.Structure):
    """Mirror of osog_tuning_t."""
    _fields_ = [("pairs_per_particle", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("band_rows", ctypes.c_int32),
                ("wait_polls", ctypes.c_int32), ("test_wait_extra", ctypes.c_int32),
                ("raster", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def optics_struct(o: dict) -> Optics:
    """osog_optics_t from an optics dict (keys as in scenes.optics)."""
    s = Optics()
    s.H, s.W = int(o["H"]), int(o["W"])
    s.dx_um, s.lambda_um, s.NA = o["dx"], o["lambda_um"], o["NA"]
    s.n_medium, s.defocus_um, s.modes = o["n_medium"], o["defocus"], int(o["modes"])
    s.oblique_frac, s.oblique_angle = o["oblique_frac"], o["oblique_angle"]
    s.shear_px, s.shear_angle = o["shear_px"], o["shear_angle"]
    s.bias_phase, s.bevel_slope = o["bias_phase"], o["bevel_slope"]
    return s


_lib = None


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libosog.so (building it first if needed) and declare signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise OSError(f"libosog.so not found at {_build.LIB}; run paper_2606_21381_gb300.build")
    L = ctypes.CDLL(_build.LIB)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    P = ctypes.POINTER
    L.osog_plan_create.argtypes = [P(vp), i32, i32]
    L.osog_plan_create.restype = ctypes.c_int
    L.osog_plan_destroy.argtypes = [vp]
    L.osog_plan_destroy.restype = None
    L.osog_workspace_size.argtypes = [vp, i32, i32, i32]
    L.osog_workspace_size.restype = sz
    L.osog_render.argtypes = [vp, vp, i64, i32, P(Optics), vp, vp, sz, vp]
    L.osog_render.restype = ctypes.c_int
    L.osog_render_opd.argtypes = [vp, vp, i64, i32, P(Optics), vp, vp, sz, vp]
    L.osog_render_opd.restype = ctypes.c_int
    L.osog_optics_from_opd.argtypes = [vp, vp, P(Optics), vp, vp, sz, vp]
    L.osog_optics_from_opd.restype = ctypes.c_int
    L.osog_batch_submit.argtypes = [vp, vp, i64, P(i32), i32, P(Optics), vp, P(Tuning), vp,
                                    sz, vp]
    L.osog_batch_submit.restype = ctypes.c_int
    L.osog_sync_status.argtypes = [vp, vp]
    L.osog_sync_status.restype = ctypes.c_int
    L.osog_last_error.argtypes = []
    L.osog_last_error.restype = ctypes.c_char_p
    L.osog_plan_launch_count.argtypes = [vp]
    L.osog_plan_launch_count.restype = i64
    L.osog_profile_begin.argtypes = [vp]
    L.osog_profile_begin.restype = ctypes.c_int
    L.osog_profile_end.argtypes = [vp, vp, P(ctypes.c_float), P(i32)]
    L.osog_profile_end.restype = ctypes.c_int
    L.osog_backward_workspace_size.argtypes = [vp, i32, i32]
    L.osog_backward_workspace_size.restype = sz
    L.osog_render_backward.argtypes = [vp, vp, i64, i32, P(Optics), vp, vp, vp, vp, sz, vp]
    L.osog_render_backward.restype = ctypes.c_int
    L.osog_plan_bind_optics_params.argtypes = [vp, vp]
    L.osog_plan_bind_optics_params.restype = ctypes.c_int
    L.osog_render_keep.argtypes = [vp, vp, i64, i32, P(Optics), vp, vp, sz, vp]
    L.osog_render_keep.restype = ctypes.c_int
    L.osog_render_backward_kept.argtypes = [vp, vp, i64, i32, P(Optics), vp, vp, vp, vp, sz, vp]
    L.osog_render_backward_kept.restype = ctypes.c_int
    L.osog_autotune.argtypes = [vp, vp, i64, P(i32), i32, P(Optics), vp, vp, sz, vp, P(Tuning)]
    L.osog_autotune.restype = ctypes.c_int
    L.osog_render_noalloc.argtypes = [vp, i64, i32, P(Optics), vp, vp]
    L.osog_noalloc_sync_status.argtypes = [vp]
    L.osog_polyhedra_workspace_size.argtypes = [vp, i32, i32, i32]
    L.osog_polyhedra_workspace_size.restype = sz
    L.osog_render_polyhedra.argtypes = [vp, vp, i64, i32, vp, vp, i32, P(Optics), vp, vp, sz, vp]
    L.osog_render_polyhedra.restype = ctypes.c_int
    L.osog_dic_incoherent_workspace_size.argtypes = [vp, i32]
    L.osog_dic_incoherent_workspace_size.restype = sz
    L.osog_render_dic_incoherent.argtypes = [vp, vp, i64, i32, P(Optics), vp, vp, sz, vp]
    L.osog_render_dic_incoherent.restype = ctypes.c_int
    L.osog_sensor_noise.argtypes = [vp, i64, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                    vp, vp]
    L.osog_sensor_noise.restype = ctypes.c_int
    L.osog_conv_out_h.argtypes = [P(ConvShape)]
    L.osog_conv_out_h.restype = i32
    L.osog_conv_out_w.argtypes = [P(ConvShape)]
    L.osog_conv_out_w.restype = i32
    L.osog_conv2d_forward.argtypes = [P(ConvShape), vp, vp, vp, i32, vp, vp, vp]
    L.osog_conv2d_forward.restype = ctypes.c_int
    L.osog_conv2d_backward_data.argtypes = [P(ConvShape), vp, vp, vp, vp, vp, vp]
    L.osog_conv2d_backward_data.restype = ctypes.c_int
    L.osog_conv2d_backward_filter_workspace.argtypes = [P(ConvShape)]
    L.osog_conv2d_backward_filter_workspace.restype = sz
    L.osog_conv2d_backward_filter.argtypes = [P(ConvShape), vp, vp, vp, vp, vp, sz, vp]
    L.osog_conv2d_backward_filter.restype = ctypes.c_int
    L.osog_conv_use_tcgen05.argtypes = [i32]
    L.osog_conv_use_tcgen05.restype = None
    L.osog_conv_sync_status.argtypes = [vp]
    L.osog_conv_sync_status.restype = ctypes.c_int
    L.osog_conv_test_wait_limit.argtypes = [i32]
    L.osog_conv_test_wait_limit.restype = ctypes.c_int
    L.osog_relu_backward.argtypes = [vp, vp, vp, i64, vp]
    L.osog_relu_backward.restype = ctypes.c_int
    L.osog_render_noalloc.restype = ctypes.c_int
    L.osog_noalloc_sync_status.restype = ctypes.c_int
    L.osog_loss_table_size.argtypes = [vp, i32]
    L.osog_loss_table_size.restype = sz
    L.osog_loss_workspace_size.argtypes = [vp, i32]
    L.osog_loss_workspace_size.restype = sz
    L.osog_loss_target.argtypes = [vp, vp, i32, vp, sz, vp, sz, vp]
    L.osog_loss_target.restype = ctypes.c_int
    L.osog_image_loss.argtypes = [vp, vp, i32, vp, sz, P(LossParams), vp, vp, vp, sz, vp]
    L.osog_image_loss.restype = ctypes.c_int
    L.osog_plan_set_pairs_per_particle.argtypes = [vp, i32]
    L.osog_plan_set_pairs_per_particle.restype = ctypes.c_int
    L.osog_pairs_for_extent.argtypes = [vp, ctypes.c_double]
    L.osog_pairs_for_extent.restype = i32
    _lib = L
    return L


def check(code: int, where: str) -> None:
    if code != 0:
        detail = lib().osog_last_error().decode(errors="replace")
        raise OsogError(code, where, detail)
