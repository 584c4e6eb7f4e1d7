"""Pins of the oracle's general polyhedra (kind 2, Eq. 1 with the caller's
M half-spaces): the prism's 14 planes reproduce the prism, an octahedron
and a bevelled polygon match their closed-form chords, and the footprint
lies inside the stated circumscribed radius."""
import math

import numpy as np

import oracle
from paper_2606_21381_gb300 import scenes

DX = 0.5


def one(cx, cy, th, radius, T, dn=1.0, mu=0.0, kind=2.0):
    s = np.zeros((9, 1), dtype=np.float32)
    s[:, 0] = [cx, cy, th, radius, radius, T, dn, mu, kind]
    return s


def local(H, W, cx, cy, th):
    """Local (u, v) in um of every pixel centre, rounded like the oracle's
    inputs (centre and angle as float32)."""
    cx, cy, th = float(np.float32(cx)), float(np.float32(cy)), float(np.float32(th))
    y, x = np.mgrid[0:H, 0:W] + 0.5
    c, s = math.cos(th), math.sin(th)
    return (c * (x - cx) + s * (y - cy)) * DX, (-s * (x - cx) + c * (y - cy)) * DX


def test_prism_planes_reproduce_the_prism():
    hx, hy, T, slope = (float(np.float32(v)) for v in (7.3, 4.1, 1.7, 1.0))
    A, b = oracle.prism_halfspaces(hx * DX, hy * DX, T, slope)
    planes = np.concatenate([A, b[:, None]], axis=1)
    prism = one(30.2, 27.9, 0.6, hx, T, kind=1.0)
    prism[4, 0] = hy
    poly = one(30.2, 27.9, 0.6, math.hypot(hx, hy), T)
    want, _ = oracle.opd_att(prism, 1, 64, 64, DX, slope)
    got, _ = oracle.opd_att(poly, 1, 64, 64, DX, slope, planes=planes, plane_off=[0, 14])
    assert want.max() > 0.5 * T
    assert np.array_equal(got, want)


def test_octahedron_chord_closed_form():
    # |u|/A + |v|/B + |z|/C <= 1: chord 2 C (1 - |u|/A - |v|/B)+
    A_, B_, C_ = 6.0, 4.0, 1.2
    planes = [(sx / A_, sy / B_, sz / C_, 1.0) for sx in (1, -1) for sy in (1, -1)
              for sz in (1, -1)]
    cx, cy, th = 31.3, 30.6, 0.35
    p = one(cx, cy, th, max(A_, B_) / DX, 2 * C_)
    got, _ = oracle.opd_att(p, 1, 64, 64, DX, planes=planes, plane_off=[0, 8])
    u, v = local(64, 64, cx, cy, th)
    want = np.maximum(2 * C_ * (1 - np.abs(u) / A_ - np.abs(v) / B_), 0.0)
    assert want.max() > 1.5
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_tilted_slab_keeps_its_vertical_thickness():
    # z <= h + 0.3 u and z >= -h + 0.3 u inside |u|, |v| <= 5 um: chord 2 h
    h = 0.8
    planes = [(-0.3, 0, 1, h), (0.3, 0, -1, h), (1, 0, 0, 5.0), (-1, 0, 0, 5.0),
              (0, 1, 0, 5.0), (0, -1, 0, 5.0)]
    cx, cy = 32.25, 32.25  # pixel centres avoid the walls
    p = one(cx, cy, 0.0, 5.0 * math.sqrt(2) / DX, 2 * h)
    got, _ = oracle.opd_att(p, 1, 64, 64, DX, planes=planes, plane_off=[0, 6])
    u, v = local(64, 64, cx, cy, 0.0)
    inside = (np.abs(u) <= 5.0) & (np.abs(v) <= 5.0)
    np.testing.assert_allclose(got, np.where(inside, 2 * h, 0.0), rtol=0, atol=1e-12)


def test_bevelled_polygon_matches_distance_to_nearest_edge():
    rng = np.random.default_rng(11)
    soa, planes, off = scenes.draw_polyhedra(rng, 3, 96, 96)
    soa[0], soa[1] = [24.3, 60.7, 47.9], [30.1, 40.2, 70.6]
    opd, _ = oracle.opd_att(soa, 3, 96, 96, DX, planes=planes, plane_off=off)
    want = np.zeros((96, 96))
    for p in range(3):
        rows = planes[off[p]:off[p + 1]].astype(np.float64)
        T = 2 * rows[0, 3]
        top = rows[2::2]  # (s n_x, s n_y, 1, s d)
        u, v = local(96, 96, soa[0, p], soa[1, p], soa[2, p])
        # chord = clamp(2 (s d_j - s n_j . (u, v))_min, 0, T)
        gap = np.min([r[3] - r[0] * u - r[1] * v for r in top], axis=0)
        want += float(soa[6, p]) * np.clip(2 * gap, 0.0, T)
    np.testing.assert_allclose(opd, want, rtol=0, atol=1e-12)


def test_footprint_lies_inside_the_circumscribed_radius():
    rng = np.random.default_rng(12)
    soa, planes, off = scenes.draw_polyhedra(rng, 6, 80, 80)
    win, _ = oracle.opd_att(soa, 6, 80, 80, DX, planes=planes, plane_off=off)
    full, _ = oracle.opd_att(soa, 6, 80, 80, DX, planes=planes, plane_off=off, full_canvas=True)
    assert np.array_equal(win, full)
    assert full.max() > 0


def test_render_with_planes_is_the_render_of_the_map():
    soa, planes, off, o = scenes.polyhedra_256(n=12)
    o = dict(o, H=64, W=64)
    soa[0] *= 0.25
    soa[1] *= 0.25
    out = oracle.render(soa, 12, o, planes=planes, plane_off=off)
    opd, att = oracle.opd_att(soa, 12, 64, 64, o["dx"], planes=planes, plane_off=off)
    assert np.array_equal(out["opd"], opd)
    np.testing.assert_allclose(out["images"], oracle.images_from_field(o, oracle.field(opd, att, o["lambda_um"])),
                               rtol=0, atol=1e-12)
