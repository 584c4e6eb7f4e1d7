"""Sensor noise on rendered images (Sec. III.C): Poisson photon shot noise
plus Gaussian read noise, computed by libosog's osog_sensor_noise."""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import check


def sensor_noise(image: torch.Tensor, photons_per_unit: float, read_sigma: float, seed: int,
                 out: torch.Tensor | None = None) -> torch.Tensor:
    """(Poisson(g max(I, 0)) + read_sigma N(0, 1)) / g elementwise, with a
    counter-based generator keyed by seed (reproducible per element)."""
    if image.device.type != "cuda" or image.dtype != torch.float32 or not image.is_contiguous():
        raise ValueError("image must be a contiguous CUDA float32 tensor")
    if out is None:
        out = torch.empty_like(image)
    stream = torch.cuda.current_stream(image.device).cuda_stream
    check(_lib.lib().osog_sensor_noise(ctypes.c_void_p(image.data_ptr()), image.numel(),
                                       float(photons_per_unit), float(read_sigma),
                                       int(seed) & 0xFFFFFFFFFFFFFFFF,
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream)),
          "osog_sensor_noise")
    return out
