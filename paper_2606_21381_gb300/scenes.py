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


def draw_polyhedra(rng: np.random.Generator, n: int, H: int, W: int, dn=(0.01, 0.05),
                   mu=(0.0, 0.0), sides=(5, 8), dist=(3.0, 10.0), thickness=(0.5, 3.0),
                   slope: float = 1.0, dx: float = 0.5):
    """n general polyhedra (kind 2): bevelled convex polygons.  Each has k ~
    U{sides} edges with outward normals at angles 2 pi j / k jittered by up
    to a quarter of the spacing and distances U(dist) px from the centre, a
    top and a bottom face at +-T/2 and, on every edge, a top and a bottom
    chamfer plane of the given slope (2 + 2k half-spaces, no vertical wall).
    Returns (soa (9, n) float32, planes (P, 4) float32 of (a_x, a_y, a_z, b)
    in the local frame (um), offsets (n + 1,) int32); soa row 3 (and 4)
    holds the footprint's circumscribed radius in px."""
    soa = np.zeros((9, n), dtype=np.float32)
    soa[0] = rng.uniform(0.0, W, n)
    soa[1] = rng.uniform(0.0, H, n)
    soa[2] = rng.uniform(0.0, math.pi, n)
    soa[5] = rng.uniform(*thickness, size=n)
    soa[6] = rng.uniform(*dn, size=n)
    soa[7] = rng.uniform(*mu, size=n) if mu[1] > mu[0] else mu[0]
    soa[8] = 2.0
    planes, offsets = [], [0]
    for p in range(n):
        k = int(rng.integers(sides[0], sides[1] + 1))
        ang = 2 * math.pi * np.arange(k) / k + rng.uniform(-0.25, 0.25, k) * (2 * math.pi / k)
        d = rng.uniform(*dist, size=k) * dx
        nx, ny = np.cos(ang), np.sin(ang)
        T = float(soa[5, p])
        rows = [(0.0, 0.0, 1.0, 0.5 * T), (0.0, 0.0, -1.0, 0.5 * T)]
        for j in range(k):
            rows.append((slope * nx[j], slope * ny[j], 1.0, slope * d[j]))
            rows.append((slope * nx[j], slope * ny[j], -1.0, slope * d[j]))
        # circumscribed radius: the farthest vertex of the polygon
        # {n_j . x <= d_j}, among the pairwise line intersections that
        # satisfy every edge
        r2 = 0.0
        for i in range(k):
            for j in range(i + 1, k):
                det = nx[i] * ny[j] - ny[i] * nx[j]
                if abs(det) < 1e-12:
                    continue
                x = (d[i] * ny[j] - ny[i] * d[j]) / det
                y = (nx[i] * d[j] - d[i] * nx[j]) / det
                if np.all(nx * x + ny * y <= d + 1e-9):
                    r2 = max(r2, x * x + y * y)
        soa[3, p] = soa[4, p] = math.sqrt(r2) / dx
        planes.extend(rows)
        offsets.append(len(planes))
    return soa, np.asarray(planes, dtype=np.float32), np.asarray(offsets, dtype=np.int32)


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


def polyhedra_256(seed: int = 5, n: int = 48):
    """256 x 256, n bevelled convex polygons given as planes (kind 2),
    brightfield + oblique, NA 0.4."""
    rng = np.random.default_rng(seed)
    soa, planes, off = draw_polyhedra(rng, n, 256, 256)
    return soa, planes, off, optics(256, 256, NA=0.4, modes=MODE_BF | MODE_OBLIQUE)


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
