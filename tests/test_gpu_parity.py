"""GPU path (through the C ABI) against the FP64 oracle on seeded scenes.

Tolerances (fixed by the method's specification): max |dOPD| <= 1e-5 max OPD;
max |dI| <= 2e-4 of the mean background intensity (1 for brightfield and
oblique, 4 sin^2(theta_b) for DIC).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_21381_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OPD_TOL = 1e-5
I_TOL = 2e-4

_renderers = {}


def renderer(H, W):
    from paper_2606_21381_gb300.render import Renderer
    if (H, W) not in _renderers:
        _renderers[(H, W)] = Renderer(H, W)
    return _renderers[(H, W)]


def background(optics):
    """Empty-field intensity of each selected modality, in bit order."""
    out = []
    for bit in (1, 2, 4):
        if optics["modes"] & bit:
            out.append(4 * math.sin(optics["bias_phase"]) ** 2 if bit == 4 else 1.0)
    return np.array(out)


def gpu_render(soa, optics, n=None):
    r = renderer(optics["H"], optics["W"])
    img = r.render(torch.from_numpy(np.ascontiguousarray(soa)).cuda(), n, optics)
    assert r.sync_status() == 0
    return img.cpu().numpy().astype(np.float64)


def gpu_opd(soa, optics, n=None):
    r = renderer(optics["H"], optics["W"])
    m = r.render_opd(torch.from_numpy(np.ascontiguousarray(soa)).cuda(), n, optics)
    assert r.sync_status() == 0
    m = m.cpu().numpy().astype(np.float64)
    return m[..., 0], m[..., 1]


def assert_images_close(got, ref, optics):
    bg = background(optics)
    for k in range(len(bg)):
        err = np.abs(got[k] - ref[k]).max()
        assert err <= I_TOL * bg[k], f"modality {k}: max |dI| {err:.3g} > {I_TOL * bg[k]:.3g}"


def assert_opd_close(soa, optics, n=None):
    n = soa.shape[1] if n is None else n
    o_ref, a_ref = oracle.opd_att(soa, n, optics["H"], optics["W"], optics["dx"],
                                  optics["bevel_slope"])
    o, a = gpu_opd(soa, optics, n)
    scale = max(np.abs(o_ref).max(), 1e-30)
    assert np.abs(o - o_ref).max() <= OPD_TOL * scale
    ascale = max(np.abs(a_ref).max(), 1e-30)
    assert np.abs(a - a_ref).max() <= OPD_TOL * ascale + 1e-30


# ---------------------------------------------------------------- plain 256^2
def test_plain_256_opd_and_images():
    soa, o = scenes.plain_256()
    assert_opd_close(soa, o)
    ref = oracle.render(soa, soa.shape[1], oracle.make_optics(**o))["images"]
    assert_images_close(gpu_render(soa, o), ref, o)


def test_optics_stage_from_oracle_opd():
    """Optics-only entry: the same float32 OPD/ATT map through both sides."""
    soa, o = scenes.plain_256(seed=7)
    o = dict(o, modes=7, defocus=0.8)
    opd, att = oracle.opd_att(soa, soa.shape[1], 256, 256)
    m = np.stack([opd, att], -1).astype(np.float32)
    ref = oracle.images_from_field(oracle.make_optics(**o),
                                   oracle.field(m[..., 0].astype(np.float64),
                                                m[..., 1].astype(np.float64), o["lambda_um"]))
    r = renderer(256, 256)
    got = r.optics_from_opd(torch.from_numpy(m).cuda(), o).cpu().numpy().astype(np.float64)
    assert r.sync_status() == 0
    assert_images_close(got, ref, o)


@pytest.mark.parametrize("H,W", [(64, 128), (128, 32), (32, 2048), (2048, 32), (512, 256)])
def test_nonsquare_all_modes(H, W):
    rng = np.random.default_rng(H * 7 + W)
    n = max(8, H * W // 400)
    soa = scenes.draw_particles(rng, n, H, W, mu=(0.0, 0.02))
    soa[0, :3] = [-2.0, W + 1.0, W / 2]   # ragged: particles across the edges
    soa[1, :3] = [H / 2, H / 2, -3.0]
    o = scenes.optics(H, W, modes=7, defocus=-1.1, oblique_angle=0.7, shear_angle=0.3)
    assert_opd_close(soa, o)
    ref = oracle.render(soa, n, oracle.make_optics(**o))["images"]
    assert_images_close(gpu_render(soa, o), ref, o)


@pytest.mark.parametrize("N", [32, 64, 128, 256, 512, 1024, 2048])
def test_empty_scene_background_every_size(N):
    o = scenes.optics(N, N, modes=7, defocus=0.5)
    soa = np.zeros((9, 1), np.float32)
    got = gpu_render(soa, o, n=0)
    bg = background(o)
    for k in range(3):
        assert np.abs(got[k] - bg[k]).max() <= I_TOL * bg[k]


@pytest.mark.parametrize("N", [32, 64, 128, 256, 512, 1024])
def test_random_scene_every_fft_plan(N):
    """Every transform length below 2048 (each has its own radix plan, and
    the strip height and column-block width follow from its set size)."""
    rng = np.random.default_rng(N)
    n = max(4, N * N // 300)
    soa = scenes.draw_particles(rng, n, N, N, mu=(0.0, 0.02))
    o = scenes.optics(N, N, modes=7, defocus=1.5, NA=0.6)
    ref = oracle.render(soa, n, oracle.make_optics(**o))["images"]
    assert_images_close(gpu_render(soa, o), ref, o)


def test_dic_1024_image():
    soa, o = scenes.dic_1024(3)
    assert_opd_close(soa, o)
    ref = oracle.render(soa, soa.shape[1], oracle.make_optics(**o))["images"]
    assert_images_close(gpu_render(soa, o), ref, o)


def test_dense_dic_1024_image():
    soa, o = scenes.dic_1024(5, dense=True)
    ref = oracle.render(soa, soa.shape[1], oracle.make_optics(**o))["images"]
    assert_images_close(gpu_render(soa, o), ref, o)


def test_full_size_2048_40k_scene():
    """The largest scene of the batched workload: 2048^2, 40,000 particles."""
    counts = scenes.batch_2048_counts()
    s = counts.index(40000)
    soa, o = scenes.batch_2048_scene(s, 40000)
    assert_opd_close(soa, o)
    ref = oracle.render(soa, soa.shape[1], oracle.make_optics(**o))["images"]
    assert_images_close(gpu_render(soa, o), ref, o)


# ---------------------------------------------------------------- invariants
def test_bitwise_deterministic():
    soa, o = scenes.dic_1024(1)
    a = gpu_render(soa, o)
    b = gpu_render(soa, o)
    assert np.array_equal(a, b)


def test_batch_equals_per_scene_bitwise():
    rng = np.random.default_rng(11)
    soas = [scenes.draw_particles(rng, c, 512, 512, mu=(0, 0.02)) for c in (0, 700, 37, 2500)]
    optics = [scenes.optics(512, 512, modes=3, defocus=d) for d in (0.0, 1.0, -1.5, 0.3)]
    soa_all, offs = scenes.concat(soas)
    r = renderer(512, 512)
    dev = torch.from_numpy(soa_all).cuda()
    out = r.batch(dev, offs, optics).cpu().numpy()
    out2 = r.batch(dev, offs, optics).cpu().numpy()   # graph replay
    out3 = r.batch(dev, offs, optics, tuning={"use_graph": 0}).cpu().numpy()
    assert r.sync_status() == 0
    for s in range(4):
        single = gpu_render(soas[s], optics[s]).astype(np.float32)
        assert np.array_equal(out[s], single), s
    assert np.array_equal(out, out2) and np.array_equal(out, out3)


def test_batch_more_than_one_launch_group():
    rng = np.random.default_rng(12)
    soas = [scenes.draw_particles(rng, int(c), 64, 64) for c in rng.integers(0, 30, 37)]
    optics = [scenes.optics(64, 64, modes=1, defocus=0.1 * i) for i in range(37)]
    soa_all, offs = scenes.concat(soas)
    r = renderer(64, 64)
    out = r.batch(torch.from_numpy(soa_all).cuda(), offs, optics).cpu().numpy()
    assert r.sync_status() == 0
    for s in (0, 31, 32, 36):
        ref = oracle.render(soas[s], soas[s].shape[1], oracle.make_optics(**optics[s]))["images"]
        assert_images_close(out[s].astype(np.float64), ref, optics[s])


# ---------------------------------------------------------------- edge cases
def test_particles_off_canvas_and_single_pixel():
    soa = np.zeros((9, 4), np.float32)
    soa[:, 0] = [-50, 10, 0, 5, 5, 1, 0.03, 0, 0]       # fully off canvas
    soa[:, 1] = [10, 5000, 0, 5, 5, 1, 0.03, 0, 1]      # fully off canvas
    soa[:, 2] = [20.5, 20.5, 0.3, 0.6, 0.6, 1, 0.03, 0.01, 0]   # about one pixel
    soa[:, 3] = [40.2, 33.1, 1.0, 0.4, 3.0, 2, 0.05, 0.0, 1]    # thin prism
    o = scenes.optics(64, 64, modes=7)
    assert_opd_close(soa, o)
    ref = oracle.render(soa, 4, oracle.make_optics(**o))["images"]
    assert_images_close(gpu_render(soa, o), ref, o)


def test_large_particle_spanning_the_canvas():
    """A particle spanning all 64 bands of a 1024^2 canvas overflows the
    default reservation of 8 pairs per particle (reported, not a fault); a
    larger reservation, set for the batch or sized for the plan from the
    particles' extent, renders it exactly."""
    soa = np.zeros((9, 2), np.float32)
    soa[:, 0] = [512, 512, 0.2, 600, 350, 1.0, 0.02, 0.001, 0]
    soa[:, 1] = [400, 560, 0.7, 60, 20, 2.0, 0.03, 0.0, 1]
    o = scenes.optics(1024, 1024, modes=1)
    r = renderer(1024, 1024)
    r.render(torch.from_numpy(soa).cuda(), None, o)
    assert r.sync_status() == 4
    soa_all, offs = scenes.concat([soa])
    got = r.batch(torch.from_numpy(soa_all).cuda(), offs, [o],
                  tuning={"pairs_per_particle": 64}).cpu().numpy()[0]
    assert r.sync_status() == 0
    ref = oracle.render(soa, 2, oracle.make_optics(**o))["images"]
    assert_images_close(got.astype(np.float64), ref, o)
    # the single-scene call sized from the particles' extent renders it too
    try:
        k = r.fit_pairs(torch.from_numpy(soa).cuda())
        assert 8 < k <= 64
        got = r.render(torch.from_numpy(soa).cuda(), None, o).cpu().numpy()
        assert r.sync_status() == 0
        assert_images_close(got.astype(np.float64), ref, o)
    finally:
        r.set_pairs_per_particle(8)


def test_invalid_particles_are_reported_and_skipped():
    rng = np.random.default_rng(3)
    soa = scenes.draw_particles(rng, 20, 128, 128)
    bad = soa.copy()
    bad[5, 3] = np.nan
    r = renderer(128, 128)
    o = scenes.optics(128, 128)
    got = r.render(torch.from_numpy(bad).cuda(), None, o).cpu().numpy().astype(np.float64)
    assert r.sync_status() == 5
    keep = np.delete(soa, 3, axis=1)
    ref = oracle.render(keep, 19, oracle.make_optics(**o))["images"]
    assert_images_close(got, ref, o)
    bad2 = soa.copy()
    bad2[3, 7] = 0.0
    r.render(torch.from_numpy(bad2).cuda(), None, o)
    assert r.sync_status() == 8
    assert r.sync_status() == 0  # cleared


def test_host_side_errors():
    from paper_2606_21381_gb300._lib import OsogError
    r = renderer(64, 64)
    soa = torch.zeros((9, 4), device="cuda")
    with pytest.raises(OsogError) as e:
        r.render(soa, None, scenes.optics(128, 128))
    assert e.value.code == 1
    with pytest.raises(OsogError) as e:
        r.render(soa, None, scenes.optics(64, 64, NA=1.5))
    assert e.value.code == 1


def test_launch_count_and_profile():
    # more than one binning chunk (256 particles): count, scan, fill, strip,
    # column, inverse
    r = renderer(256, 256)
    rng = np.random.default_rng(31)
    soa = scenes.draw_particles(rng, 300, 256, 256)
    o = scenes.optics(256, 256, modes=3)
    before = r.launch_count()
    r.profile_begin()
    r.render(torch.from_numpy(soa).cuda(), None, o)
    prof = r.profile_end()
    assert r.launch_count() - before == 6
    fwd = ("bin_count", "bin_scan", "bin_fill", "strip_forward", "column", "strip_inverse")
    assert all(prof[k][1] == 1 and prof[k][0] > 0 for k in fwd)
    assert all(v[1] == 0 for k, v in prof.items() if k not in fwd)
    # one chunk (64 particles): the three binning passes in one launch,
    # counted as bin_count
    soa, o = scenes.plain_256()
    before = r.launch_count()
    r.profile_begin()
    r.render(torch.from_numpy(soa).cuda(), None, o)
    prof = r.profile_end()
    assert r.launch_count() - before == 4
    assert prof["bin_count"][1] == 1 and prof["bin_scan"][1] == 0 and prof["bin_fill"][1] == 0
    assert r.sync_status() == 0


def test_single_chunk_binning_equals_the_three_passes():
    # the same 256 particles rendered alone (one chunk, one launch) and as
    # the first scene of a batch whose other scene makes the group span
    # several chunks (count, scan and fill): bitwise the same image
    r = renderer(256, 256)
    rng = np.random.default_rng(32)
    a = scenes.draw_particles(rng, 256, 256, 256, mu=(0.0, 0.02))
    b = scenes.draw_particles(rng, 700, 256, 256, mu=(0.0, 0.02))
    o = scenes.optics(256, 256, modes=7, defocus=0.4)
    alone = r.render(torch.from_numpy(np.ascontiguousarray(a)).cuda(), None, o).clone()
    soa_all, offs = scenes.concat([a, b])
    both = r.batch(torch.from_numpy(soa_all).cuda(), offs, [o, o],
                   tuning={"use_graph": 0}).clone()
    assert r.sync_status() == 0
    assert torch.equal(alone, both[0])
