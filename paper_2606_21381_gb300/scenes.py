"""Seeded synthetic scenes shaped like the paper's workloads.

This module only draws random numbers: it holds none of the rendering
arithmetic, and both the CUDA path and the FP64 oracle read the arrays it
returns.  A scene is a structure-of-arrays particle tensor of shape (9, n),
float32, rows

    cx, cy (px), theta (rad), a | hx (px), b | hy (px), T (um), dn, mu (1/um),
    kind (0 = ellipsoid, 1 = bevelled prism)

plus an optics dict with the keys

    H, W, dx (um), lambda_um, NA, n_medium, defocus (um), modes (bit mask:
    1 brightfield, 2 oblique, 4 DIC), oblique_frac, oblique_angle (rad),
    shear_px, shear_angle (rad), bias_phase (rad), bevel_slope.

The state tensor S in R^{N x D} of Sec. III.A is stored planar ([D][N]) so
that each field is one contiguous row.  Distributions follow the workloads
the paper benchmarks (Sec. IV.C: up to 40,000 particles on a single canvas):
half ellipsoids, half prisms, random orientation, centres uniform over the
canvas.
"""
from __future__ import annotations

import math

import numpy as np

FIELDS = ("cx", "cy", "theta", "a", "b", "T", "dn", "mu", "kind")
MODE_BF, MODE_OBLIQUE, MODE_DIC = 1, 2, 4


def optics(H: int, W: int, **kw) -> dict:
    """Optics dict with the defaults of the plain render (0.5 um pixels,
    550 nm, NA 0.4, in focus, brightfield)."""
    o = dict(H=int(H), W=int(W), dx=0.5, lambda_um=0.55, NA=0.4, n_medium=1.0,
             defocus=0.0, modes=MODE_BF, oblique_frac=0.3, oblique_angle=0.0,
             shear_px=1.0, shear_angle=math.pi / 4, bias_phase=math.pi / 4,
             bevel_slope=1.0)
    o.update(kw)
    return o


def draw_particles(rng: np.random.Generator, n: int, H: int, W: int,
                   dn=(0.01, 0.05), mu=(0.0, 0.0), ell_axes=(2.0, 10.0),
                   prism_half=(2.0, 12.0), thickness=(0.5, 3.0),
                   size_scale: float = 1.0) -> np.ndarray:
    """n particles: kind ~ Bernoulli(0.5); ellipsoid semi-axes and prism
    half-lengths uniform in the given ranges (px, times size_scale);
    theta ~ U(0, pi); centres uniform over [0, W) x [0, H); T, dn, mu
    uniform."""
    soa = np.zeros((9, n), dtype=np.float32)
    kind = (rng.random(n) < 0.5).astype(np.float32)
    ea = rng.uniform(*ell_axes, size=(2, n))
    ph = rng.uniform(*prism_half, size=(2, n))
    soa[0] = rng.uniform(0.0, W, n)
    soa[1] = rng.uniform(0.0, H, n)
    soa[2] = rng.uniform(0.0, math.pi, n)
    soa[3] = np.where(kind > 0.5, ph[0], ea[0]) * size_scale
    soa[4] = np.where(kind > 0.5, ph[1], ea[1]) * size_scale
    soa[5] = rng.uniform(*thickness, size=n)
    soa[6] = rng.uniform(*dn, size=n)
    soa[7] = rng.uniform(*mu, size=n) if mu[1] > mu[0] else mu[0]
    soa[8] = kind
    return soa


# ------------------------------------------------------------------ workloads
def plain_256(seed: int = 0):
    """256 x 256, 64 particles, brightfield + oblique (offset 0.3 NA)."""
    rng = np.random.default_rng(seed)
    soa = draw_particles(rng, 64, 256, 256)
    return soa, optics(256, 256, NA=0.4, modes=MODE_BF | MODE_OBLIQUE)


def dic_1024(index: int, dense: bool = False):
    """One image of the 16 x 1024^2 DIC batch (index 0..15): 4,000
    particles, shear 1 px along 45 deg, bias pi/4, NA 0.5, defocus
    U(-2, 2) um.  dense=True scales sizes by 1.8 (about 2x coverage)."""
    rng = np.random.default_rng(1 + index)
    soa = draw_particles(rng, 4000, 1024, 1024, size_scale=1.8 if dense else 1.0)
    dz = float(rng.uniform(-2.0, 2.0))
    return soa, optics(1024, 1024, NA=0.5, modes=MODE_DIC, defocus=dz,
                       shear_px=1.0, shear_angle=math.pi / 4, bias_phase=math.pi / 4)


def batch_2048_counts(seed: int = 100, scenes: int = 32, lo: int = 1000,
                      hi: int = 40000) -> list[int]:
    """Particle counts of the batched workload: scenes-1 draws
    round(exp(U(ln lo, ln hi))) plus one scene with exactly hi, shuffled."""
    rng = np.random.default_rng(seed)
    c = [int(round(math.exp(x))) for x in rng.uniform(math.log(lo), math.log(hi), scenes - 1)]
    c.append(hi)
    rng.shuffle(c)
    return c


def batch_2048_scene(s: int, count: int, size: int = 2048):
    """Scene s of the batched workload: dn U(0.005, 0.06), mu U(0, 0.02),
    oblique illumination, NA 0.4."""
    rng = np.random.default_rng(100 + s)
    soa = draw_particles(rng, count, size, size, dn=(0.005, 0.06), mu=(0.0, 0.02))
    return soa, optics(size, size, NA=0.4, modes=MODE_OBLIQUE)


def batch_2048(scenes: int = 32, size: int = 2048, seed: int = 100):
    """All scenes of the batched workload: (list of soa, list of optics)."""
    counts = batch_2048_counts(seed, scenes)
    out = [batch_2048_scene(s, c, size) for s, c in enumerate(counts)]
    return [a for a, _ in out], [o for _, o in out]


def inverse_512(seed: int = 3, n: int = 200):
    """512 x 512, 200 particles, brightfield + DIC, NA 0.4; each particle
    has a known absorption mu U(0.005, 0.02) so that the amplitude pins
    the thickness separately from dn."""
    rng = np.random.default_rng(seed)
    soa = draw_particles(rng, n, 512, 512, mu=(0.005, 0.02))
    return soa, optics(512, 512, NA=0.4, modes=MODE_BF | MODE_DIC)


def concat(soas: list[np.ndarray]):
    """Concatenate scenes into one (9, total) array plus offsets [S+1]."""
    counts = [s.shape[1] for s in soas]
    offsets = np.zeros(len(soas) + 1, dtype=np.int32)
    offsets[1:] = np.cumsum(counts)
    return np.concatenate(soas, axis=1), offsets
