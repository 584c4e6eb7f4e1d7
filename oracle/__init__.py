"""FP64 CPU oracle for the OSOG forward model (arxiv 2606.21381).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product package
never imports this module, and this module imports nothing from the product.

The arithmetic lives in ``osog_oracle.c`` (plain C, double precision, one
definition per step, see that file's header for the equations it follows).
This module compiles it with gcc, loads it with ctypes and exposes numpy-level
wrappers.  Optics are passed as plain dicts with the keys of ``OPTICS_KEYS``.

Parity pins (closed forms, brute force, library special cases) live in
``tests/test_oracle_pins.py``.  Every oracle function is pinned there except
the bevel constant of the prism chamfers, whose value the paper does not give
(parity unpinned: the chamfer slope is a definition of this project, shared
by both sides only as a written formula).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "osog_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_BF, MODE_OBLIQUE, MODE_DIC = 1, 2, 4

OPTICS_KEYS = ("H", "W", "dx", "lambda_um", "NA", "n_medium", "defocus",
               "modes", "oblique_frac", "oblique_angle", "shear_px",
               "shear_angle", "bias_phase", "bevel_slope")

DEFAULT_OPTICS = dict(dx=0.5, lambda_um=0.55, NA=0.4, n_medium=1.0, defocus=0.0,
                      modes=MODE_BF, oblique_frac=0.3, oblique_angle=0.0,
                      shear_px=1.0, shear_angle=np.pi / 4, bias_phase=np.pi / 4,
                      bevel_slope=1.0)


class _Optics(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("dx", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("NA", ctypes.c_double), ("n_medium", ctypes.c_double),
                ("defocus", ctypes.c_double), ("modes", ctypes.c_uint32),
                ("oblique_frac", ctypes.c_double), ("oblique_angle", ctypes.c_double),
                ("shear_px", ctypes.c_double), ("shear_angle", ctypes.c_double),
                ("bias_phase", ctypes.c_double), ("bevel_slope", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, -O2, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        d, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.orc_halfspace_chord.restype = ctypes.c_double
        lib.orc_halfspace_chord.argtypes = [d, d, i32, ctypes.c_double, ctypes.c_double]
        lib.orc_prism_halfspaces.argtypes = [ctypes.c_double] * 4 + [d, d]
        lib.orc_opd_att.argtypes = [d, i64, i32, i32, i32, ctypes.c_double,
                                    ctypes.c_double, i32, d, d]
        lib.orc_opd_at.argtypes = [d, i64, i32, ctypes.c_double, ctypes.c_double,
                                   d, i64, i32, d, d]
        lib.orc_field.argtypes = [d, d, i64, ctypes.c_double, d, d]
        lib.orc_fft2.argtypes = [d, d, i32, i32, i32]
        lib.orc_dft2_brute.argtypes = [d, d, i32, i32, i32, d, d]
        lib.orc_transfer.argtypes = [ctypes.POINTER(_Optics), i32, d, d]
        lib.orc_images.argtypes = [ctypes.POINTER(_Optics), d, d, d]
        lib.orc_render.argtypes = [d, i64, i32, ctypes.POINTER(_Optics), d, d, d, d, d]
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.orc_philox4x32.argtypes = [u32p, u32p, u32p]
        lib.orc_poisson.argtypes = [ctypes.c_double, ctypes.c_uint64, i64]
        lib.orc_poisson.restype = i64
        lib.orc_normal.argtypes = [ctypes.c_uint64, i64]
        lib.orc_normal.restype = ctypes.c_double
        lib.orc_sensor_noise.argtypes = [ctypes.POINTER(ctypes.c_float), i64, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_uint64, d]
        lib.orc_set_threads.argtypes = [i32]
        lib.orc_dic_incoherent.argtypes = [ctypes.POINTER(_Optics), d, d, d]
        lib.orc_opd_att_poly.argtypes = [d, i64, i32, i32, i32, ctypes.c_double,
                                         ctypes.c_double, i32, d, d, d, d]
        lib.orc_render_poly.argtypes = [d, i64, i32, d, d, ctypes.POINTER(_Optics), d, d, d,
                                        d, d]
        lib.orc_render_grad.argtypes = [d, i64, i32, ctypes.POINTER(_Optics), d, d, d]
        lib.orc_spectral_loss.argtypes = [d, d, i32, i32, i32, ctypes.c_double, d]
        lib.orc_spectral_loss.restype = ctypes.c_double
        lib.orc_lowpass_misfit.argtypes = [d, d, i32, i32, i32, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, d]
        lib.orc_lowpass_misfit.restype = ctypes.c_double
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def make_optics(H: int, W: int, **kw) -> dict:
    o = dict(DEFAULT_OPTICS)
    o.update(kw)
    o["H"], o["W"] = int(H), int(W)
    unknown = set(o) - set(OPTICS_KEYS)
    if unknown:
        raise KeyError(f"unknown optics keys {sorted(unknown)}")
    return o


def _optics_struct(o: dict) -> _Optics:
    s = _Optics()
    s.H, s.W = int(o["H"]), int(o["W"])
    s.dx, s.lambda_, s.NA = o["dx"], o["lambda_um"], o["NA"]
    s.n_medium, s.defocus, s.modes = o["n_medium"], o["defocus"], int(o["modes"])
    s.oblique_frac, s.oblique_angle = o["oblique_frac"], o["oblique_angle"]
    s.shear_px, s.shear_angle = o["shear_px"], o["shear_angle"]
    s.bias_phase, s.bevel_slope = o["bias_phase"], o["bevel_slope"]
    return s


def n_modes(o: dict) -> int:
    return bin(int(o["modes"]) & 7).count("1")


def _soa(soa: np.ndarray):
    soa = np.ascontiguousarray(soa, dtype=np.float32)
    if soa.ndim != 2 or soa.shape[0] != 9:
        raise ValueError("soa must be a (9, ld) float32 array")
    return soa, soa.shape[1]


# ---------------------------------------------------------------- geometry
def prism_halfspaces(hx_um: float, hy_um: float, T: float, slope: float):
    """(A, b) of the bevelled prism's 14 half-spaces (Eq. 1)."""
    A = np.zeros((14, 3))
    b = np.zeros(14)
    _load().orc_prism_halfspaces(hx_um, hy_um, T, slope, _p(A), _p(b))
    return A, b


def halfspace_chord(A: np.ndarray, b: np.ndarray, u: float, v: float) -> float:
    """Vertical chord through (u, v) of the polyhedron {x: A x <= b}."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return _load().orc_halfspace_chord(_p(A), _p(b), len(b), float(u), float(v))


def _planes(planes, plane_off, n: int):
    """float64 (P, 4) planes and int32 (n + 1,) offsets of kind-2 particles."""
    pl = np.ascontiguousarray(planes, dtype=np.float64).reshape(-1, 4)
    off = np.ascontiguousarray(plane_off, dtype=np.int32)
    if off.shape != (n + 1,) or off[0] < 0 or np.any(np.diff(off) < 0) or off[-1] > len(pl):
        raise ValueError("plane_off must be non-decreasing offsets [n + 1] into planes")
    return pl, off


def opd_att(soa: np.ndarray, n: int, H: int, W: int, dx: float = 0.5,
            bevel_slope: float = 1.0, full_canvas: bool = False, planes=None,
            plane_off=None):
    """OPD (um) and absorption-thickness maps, each (H, W) float64.  Kind-2
    particles (general polyhedra) take their half-spaces from planes
    (rows (a_x, a_y, a_z, b), local frame in um) and plane_off [n + 1]."""
    soa, ld = _soa(soa)
    opd = np.zeros((H, W))
    att = np.zeros((H, W))
    if planes is None:
        if np.any(soa[8, :n] > 1.5):
            raise ValueError("kind-2 particles need planes")
        _load().orc_opd_att(_p(soa), ld, int(n), H, W, dx, bevel_slope,
                            int(full_canvas), _p(opd), _p(att))
    else:
        pl, off = _planes(planes, plane_off, n)
        _load().orc_opd_att_poly(_p(soa), ld, int(n), H, W, dx, bevel_slope,
                                 int(full_canvas), _p(pl), _p(off), _p(opd), _p(att))
    return opd, att


def opd_at(soa: np.ndarray, n: int, W: int, pixels: np.ndarray, dx: float = 0.5,
           bevel_slope: float = 1.0):
    """OPD and ATT at flat pixel indices, by brute force over all particles."""
    soa, ld = _soa(soa)
    pix = np.ascontiguousarray(pixels, dtype=np.int64)
    opd = np.zeros(len(pix))
    att = np.zeros(len(pix))
    _load().orc_opd_at(_p(soa), ld, int(n), dx, bevel_slope, _p(pix), len(pix),
                       W, _p(opd), _p(att))
    return opd, att


def field(opd: np.ndarray, att: np.ndarray, lambda_um: float) -> np.ndarray:
    """Exit wave exp(-att) exp(i 2 pi opd / lambda) as complex128."""
    opd = np.ascontiguousarray(opd, dtype=np.float64)
    att = np.ascontiguousarray(att, dtype=np.float64)
    re = np.empty_like(opd)
    im = np.empty_like(opd)
    _load().orc_field(_p(opd), _p(att), opd.size, lambda_um, _p(re), _p(im))
    return re + 1j * im


# ---------------------------------------------------------------- Fourier
def fft2(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """The oracle's own radix-2 2-D FFT (unnormalised)."""
    re = np.ascontiguousarray(x.real, dtype=np.float64).copy()
    im = np.ascontiguousarray(x.imag, dtype=np.float64).copy()
    H, W = re.shape
    _load().orc_fft2(_p(re), _p(im), H, W, int(sign))
    return re + 1j * im


def dft2_brute(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """O((HW)^2) DFT straight from the definition."""
    re = np.ascontiguousarray(x.real, dtype=np.float64)
    im = np.ascontiguousarray(x.imag, dtype=np.float64)
    H, W = re.shape
    ore = np.empty_like(re)
    oim = np.empty_like(re)
    _load().orc_dft2_brute(_p(re), _p(im), H, W, int(sign), _p(ore), _p(oim))
    return ore + 1j * oim


# ---------------------------------------------------------------- optics
def transfer(o: dict, mode: int) -> np.ndarray:
    """H_m(k) on the (H, W) DFT grid as complex128."""
    s = _optics_struct(o)
    hr = np.empty((o["H"], o["W"]))
    hi = np.empty_like(hr)
    _load().orc_transfer(ctypes.byref(s), int(mode), _p(hr), _p(hi))
    return hr + 1j * hi


def images_from_field(o: dict, E: np.ndarray) -> np.ndarray:
    """(K, H, W) intensities of every selected modality for exit wave E."""
    s = _optics_struct(o)
    re = np.ascontiguousarray(E.real, dtype=np.float64)
    im = np.ascontiguousarray(E.imag, dtype=np.float64)
    out = np.empty((n_modes(o), o["H"], o["W"]))
    _load().orc_images(ctypes.byref(s), _p(re), _p(im), _p(out))
    return out


def dic_incoherent(o: dict, E: np.ndarray) -> np.ndarray:
    """Eq. 5 read literally: |U(r + ds) e^{i theta} - U(r - ds) e^{-i theta}|^2
    blurred by the unit-sum intensity PSF of the brightfield pupil; (H, W)."""
    s = _optics_struct(o)
    re = np.ascontiguousarray(E.real, dtype=np.float64)
    im = np.ascontiguousarray(E.imag, dtype=np.float64)
    out = np.empty((o["H"], o["W"]))
    _load().orc_dic_incoherent(ctypes.byref(s), _p(re), _p(im), _p(out))
    return out


def render_dic_incoherent(soa: np.ndarray, n: int, o: dict) -> np.ndarray:
    """Incoherent DIC image of a scene (H, W): OPD/ATT maps, exit wave, then
    dic_incoherent."""
    opd, att = opd_att(soa, n, o["H"], o["W"], o["dx"], o["bevel_slope"])
    return dic_incoherent(o, field(opd, att, o["lambda_um"]))


def set_threads(n: int) -> None:
    """Number of OpenMP threads of the oracle's parallel loops."""
    _load().orc_set_threads(int(n))


def philox4x32(ctr, key) -> tuple:
    """Philox4x32-10 of a 4-word counter and 2-word key."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    _load().orc_philox4x32(c, k, o)
    return tuple(o)


def poisson(lam: float, seed: int, index: int) -> int:
    """The Poisson sample of element `index` (see orc_poisson)."""
    return int(_load().orc_poisson(float(lam), int(seed), int(index)))


def normal(seed: int, index: int) -> float:
    return float(_load().orc_normal(int(seed), int(index)))


def sensor_noise(img: np.ndarray, photons: float, read_sigma: float, seed: int) -> np.ndarray:
    """(Poisson(g max(I, 0)) + sigma N(0, 1)) / g per element, float64."""
    x = np.ascontiguousarray(img, dtype=np.float32)
    out = np.empty(x.shape)
    _load().orc_sensor_noise(x.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), x.size,
                             float(photons), float(read_sigma), int(seed), _p(out))
    return out


def render(soa: np.ndarray, n: int, o: dict, planes=None, plane_off=None) -> dict:
    """Whole forward model: returns dict(opd, att, field, images).  planes /
    plane_off as for opd_att (kind-2 particles)."""
    soa, ld = _soa(soa)
    s = _optics_struct(o)
    H, W = o["H"], o["W"]
    opd = np.empty((H, W))
    att = np.empty_like(opd)
    er = np.empty_like(opd)
    ei = np.empty_like(opd)
    img = np.empty((n_modes(o), H, W))
    if planes is None:
        if np.any(soa[8, :n] > 1.5):
            raise ValueError("kind-2 particles need planes")
        _load().orc_render(_p(soa), ld, int(n), ctypes.byref(s), _p(opd), _p(att),
                           _p(er), _p(ei), _p(img))
    else:
        pl, off = _planes(planes, plane_off, n)
        _load().orc_render_poly(_p(soa), ld, int(n), _p(pl), _p(off), ctypes.byref(s),
                                _p(opd), _p(att), _p(er), _p(ei), _p(img))
    return dict(opd=opd, att=att, field=er + 1j * ei, images=img)


def render_grad(soa: np.ndarray, n: int, o: dict, gI: np.ndarray):
    """Gradient of L = sum(gI * images) with respect to the particle fields
    ((9, n) float64, kind row zero) and the optics scalars (defocus,
    shear_px, shear_angle, bias_phase), by the FP64 analytic adjoint."""
    soa, ld = _soa(soa)
    s = _optics_struct(o)
    gI = np.ascontiguousarray(gI, dtype=np.float64)
    if gI.shape != (n_modes(o), o["H"], o["W"]):
        raise ValueError("gI must have shape (K, H, W)")
    gsoa = np.zeros((9, max(int(n), 1)))
    gopt = np.zeros(4)
    _load().orc_render_grad(_p(soa), ld, int(n), ctypes.byref(s), _p(gI), _p(gsoa), _p(gopt))
    return gsoa[:, :int(n)], gopt


# ---------------------------------------------------------------- losses
def _images(img: np.ndarray, tgt: np.ndarray):
    img = np.ascontiguousarray(img, dtype=np.float64)
    tgt = np.ascontiguousarray(tgt, dtype=np.float64)
    if img.shape != tgt.shape or img.ndim != 3:
        raise ValueError("image and target must be (K, H, W) arrays of one shape")
    return img, tgt


def spectral_loss(img: np.ndarray, tgt: np.ndarray, eps_rel: float = 1e-6):
    """Eq. 8: (loss, dloss/dimg) of the log-amplitude spectral loss of
    (K, H, W) images (see orc_spectral_loss)."""
    img, tgt = _images(img, tgt)
    K, H, W = img.shape
    g = np.empty_like(img)
    v = _load().orc_spectral_loss(_p(img), _p(tgt), K, H, W, float(eps_rel), _p(g))
    return float(v), g


def lowpass_misfit(img: np.ndarray, tgt: np.ndarray, dx: float, cutoff: float,
                   scale: float = 1.0):
    """(loss, dloss/dimg) of the curriculum misfit: scale times the sum of
    squared differences of the images low-passed at `cutoff` cycles/um
    (see orc_lowpass_misfit)."""
    img, tgt = _images(img, tgt)
    K, H, W = img.shape
    g = np.empty_like(img)
    v = _load().orc_lowpass_misfit(_p(img), _p(tgt), K, H, W, float(dx), float(cutoff),
                                   float(scale), _p(g))
    return float(v), g
