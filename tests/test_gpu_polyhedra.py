"""General convex polyhedra (kind 2) through osog_render_polyhedra against
the FP64 oracle, mixed with ellipsoids and prisms; the prism's 14 planes
render like the prism; bad plane ranges are latched and skipped."""
import math

import numpy as np
import pytest

import oracle
from paper_2606_21381_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_I = 2e-4  # of the empty-field background (1 for brightfield and oblique)


@pytest.fixture(scope="module")
def R256():
    from paper_2606_21381_gb300.render import Renderer
    return Renderer(256, 256)


def _dev(soa, planes, off):
    return (torch.from_numpy(np.ascontiguousarray(soa)).cuda(),
            torch.from_numpy(np.ascontiguousarray(planes, dtype=np.float32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(off, dtype=np.int32)).cuda())


def test_polyhedra_match_the_oracle(R256):
    soa, planes, off, o = scenes.polyhedra_256()
    n = soa.shape[1]
    want = oracle.render(soa, n, o, planes=planes, plane_off=off)["images"]
    s, p, f = _dev(soa, planes, off)
    got = R256.render_polyhedra(s, n, p, f, o).cpu().numpy()
    assert R256.sync_status() == 0
    assert np.abs(want - 1).max() > 0.05  # the scene has contrast
    assert np.abs(got - want).max() <= TOL_I


def test_mixed_kinds_match_the_oracle():
    from paper_2606_21381_gb300.render import Renderer
    rng = np.random.default_rng(21)
    H = W = 512
    poly, planes, poff = scenes.draw_polyhedra(rng, 60, H, W, mu=(0.0, 0.02))
    other = scenes.draw_particles(rng, 140, H, W, mu=(0.0, 0.02))
    soa = np.concatenate([other[:, :70], poly, other[:, 70:]], axis=1)
    # offsets over all 200 particles: kinds 0 and 1 own no rows
    counts = np.zeros(200, dtype=np.int32)
    counts[70:130] = np.diff(poff)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    o = scenes.optics(H, W, NA=0.5, modes=scenes.MODE_BF | scenes.MODE_DIC, defocus=0.7)
    want = oracle.render(soa, 200, o, planes=planes, plane_off=off)["images"]
    r = Renderer(H, W)
    s, p, f = _dev(soa, planes, off)
    got = r.render_polyhedra(s, 200, p, f, o).cpu().numpy()
    assert r.sync_status() == 0
    bg = np.array([1.0, 4 * math.sin(o["bias_phase"]) ** 2])[:, None, None]
    assert np.abs(got - want).max() <= TOL_I * bg.max()
    assert np.all(np.abs(got - want).max(axis=(1, 2)) <= TOL_I * bg[:, 0, 0])


def test_prism_planes_render_like_the_prism(R256):
    rng = np.random.default_rng(22)
    soa = scenes.draw_particles(rng, 30, 256, 256)
    soa[8] = 1.0
    rows, off = [], [0]
    poly = soa.copy()
    for p in range(30):
        hx, hy, T = (float(v) for v in soa[[3, 4, 5], p])
        A, b = oracle.prism_halfspaces(hx * 0.5, hy * 0.5, T, 1.0)
        rows.extend(np.concatenate([A, b[:, None]], axis=1).tolist())
        off.append(len(rows))
        poly[3, p] = poly[4, p] = math.hypot(hx, hy)
    poly[8] = 2.0
    o = scenes.optics(256, 256, modes=scenes.MODE_BF | scenes.MODE_OBLIQUE)
    a = R256.render(torch.from_numpy(soa).cuda(), None, o).cpu().numpy()
    s, p, f = _dev(poly, np.asarray(rows), off)
    b = R256.render_polyhedra(s, None, p, f, o).cpu().numpy()
    assert R256.sync_status() == 0
    assert np.abs(a - b).max() <= TOL_I


def test_bad_plane_ranges_are_latched_and_skipped(R256):
    soa, planes, off, o = scenes.polyhedra_256(n=8)

    def render(k, offsets):
        s, p, f = _dev(soa[:, :k], planes, offsets)
        return R256.render_polyhedra(s, k, p, f, o).cpu().numpy()

    ref3, ref4 = render(3, off[:4]), render(4, off[:5])
    assert R256.sync_status() == 0
    # particle 4's range runs past the plane list: 0..3 intact
    img = render(5, [*off[:5], len(planes) + 1])
    assert R256.sync_status() == 8
    assert np.array_equal(img, ref4)
    # particle 3 with 33 planes, particle 4 with none: 0..2 intact
    img = render(5, [*off[:4], off[3] + 33, off[3] + 33])
    assert R256.sync_status() == 8
    assert np.array_equal(img, ref3)


def test_kind_two_needs_the_polyhedra_entry(R256):
    soa, _, _, o = scenes.polyhedra_256(n=4)
    img = R256.render(torch.from_numpy(soa).cuda(), None, o).cpu().numpy()
    assert R256.sync_status() == 8
    assert np.allclose(img, 1.0, atol=1e-5)  # every particle skipped: empty field
