"""Batched path: the persistent launch, band-height choices and the
autotuner give results bitwise identical to the three-launch path (the
same arithmetic in the same order per pixel), and match the oracle."""
import numpy as np
import pytest

import oracle
from paper_2606_21381_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

_renderers = {}


def renderer(H, W):
    from paper_2606_21381_gb300.render import Renderer
    if (H, W) not in _renderers:
        _renderers[(H, W)] = Renderer(H, W)
    return _renderers[(H, W)]


def batch(seed, S, size, modes, lo=0, hi=600):
    rng = np.random.default_rng(seed)
    soas = [scenes.draw_particles(rng, int(c), size, size, mu=(0, 0.02))
            for c in rng.integers(lo, hi, S)]
    optics = [scenes.optics(size, size, modes=modes, defocus=rng.uniform(-1, 1)) for _ in range(S)]
    soa_all, offs = scenes.concat(soas)
    return soas, optics, torch.from_numpy(soa_all).cuda(), offs


@pytest.mark.parametrize("modes,S", [(2, 5), (3, 4), (1, 37)])
def test_persistent_launch_is_bitwise_identical(modes, S):
    soas, optics, dev, offs = batch(modes * 10 + S, S, 256, modes)
    r = renderer(256, 256)
    base = r.batch(dev, offs, optics, tuning={"use_graph": 0, "persistent": -1}).clone()
    pers = r.batch(dev, offs, optics, tuning={"use_graph": 0, "persistent": 1}).clone()
    graph = r.batch(dev, offs, optics, tuning={"use_graph": 1, "persistent": 1}).clone()
    assert r.sync_status() == 0
    assert torch.equal(base, pers) and torch.equal(base, graph)
    s = S - 1
    ref = oracle.render(soas[s], soas[s].shape[1], oracle.make_optics(**optics[s]))["images"]
    assert np.abs(pers[s].cpu().numpy().astype(np.float64) - ref).max() <= 2e-4


@pytest.mark.parametrize("band_rows", [64, 128, 256])
def test_band_height_does_not_change_results(band_rows):
    soas, optics, dev, offs = batch(3, 4, 512, 1, 100, 2000)
    r = renderer(512, 512)
    base = r.batch(dev, offs, optics, tuning={"use_graph": 0}).clone()
    other = r.batch(dev, offs, optics, tuning={"use_graph": 0, "band_rows": band_rows,
                                              "pairs_per_particle": 8}).clone()
    assert r.sync_status() == 0
    assert torch.equal(base, other)


def test_invalid_band_height_is_rejected_on_the_host():
    from paper_2606_21381_gb300._lib import OsogError
    soas, optics, dev, offs = batch(4, 2, 512, 1)
    r = renderer(512, 512)
    with pytest.raises(OsogError) as e:
        r.batch(dev, offs, optics, tuning={"use_graph": 0, "band_rows": 12})
    assert e.value.code == 1


def test_autotuner_choice_is_used_and_exact():
    soas, optics, dev, offs = batch(5, 8, 1024, 2, 500, 5000)
    r = renderer(1024, 1024)
    base = r.batch(dev, offs, optics, tuning={"use_graph": 0, "persistent": -1}).clone()
    t = r.autotune(dev, offs, optics)
    assert r.sync_status() == 0
    assert t["band_rows"] in (16, 32, 64, 128) and 1 <= t["pairs_per_particle"] <= 8
    assert t["persistent"] in (1, -1)
    tuned = r.batch(dev, offs, optics).clone()   # picks the stored choice
    assert r.sync_status() == 0                  # the exact reservation does not overflow
    assert torch.equal(base, tuned)


def test_host_pipeline_matches_batch():
    # three batches through the two-slot pipeline (slot reuse included)
    # equal the same batches rendered one at a time
    from paper_2606_21381_gb300.render import HostBatchPipeline, Renderer
    r = Renderer(256, 256)
    rng = np.random.default_rng(41)
    batches = []
    for b in range(3):
        soas = [scenes.draw_particles(rng, int(c), 256, 256, mu=(0.0, 0.02)) for c in (50, 120, 7)]
        optics = [scenes.optics(256, 256, modes=scenes.MODE_BF | scenes.MODE_OBLIQUE,
                                defocus=0.3 * b + 0.1 * s) for s in range(3)]
        soa_all, offs = scenes.concat(soas)
        batches.append((soa_all, offs, optics))
    pipe = HostBatchPipeline(r, 200, 3, 2)
    outs = []
    for soa_all, offs, optics in batches:
        h = torch.empty((3, 2, 256, 256)).pin_memory()
        pipe.submit(torch.from_numpy(soa_all).pin_memory(), offs, optics, h)
        outs.append(h)
    pipe.synchronize()
    assert r.sync_status() == 0
    for (soa_all, offs, optics), h in zip(batches, outs):
        want = r.batch(torch.from_numpy(soa_all).cuda(), offs, optics).cpu()
        assert torch.equal(h, want)


def test_bound_optics_scalars_in_the_batched_path():
    """With a bound device array every scene of a batch takes its defocus,
    shear and bias from it, also through the cached CUDA graph (whose key
    includes the binding), and unbinding restores the per-scene values."""
    from paper_2606_21381_gb300.autograd import OPTICS_PARAMS
    soas, optics, dev, offs = batch(77, 4, 256, 7)
    r = renderer(256, 256)
    vals = {"defocus": 0.7, "shear_px": 1.4, "shear_angle": 0.3, "bias_phase": 1.1}
    same = [dict(o, **vals) for o in optics]
    want = r.batch(dev, offs, same, tuning={"use_graph": 1}).clone()
    own = r.batch(dev, offs, optics, tuning={"use_graph": 1}).clone()
    params = torch.tensor([vals[k] for k in OPTICS_PARAMS], dtype=torch.float32, device="cuda")
    r.bind_optics_params(params)
    try:
        got = [r.batch(dev, offs, optics, tuning={"use_graph": g}).clone() for g in (0, 1, 1)]
    finally:
        r.bind_optics_params(None)
    back = r.batch(dev, offs, optics, tuning={"use_graph": 1}).clone()
    assert r.sync_status() == 0
    scale = float(want.abs().max())
    for g in got:
        assert float((g - want).abs().max()) <= 1e-5 * scale
    assert torch.equal(got[1], got[2]) and torch.equal(got[0], got[1])
    assert torch.equal(back, own)
    assert float((own - want).abs().max()) > 1e-3 * scale


def test_tile_raster_and_strip_raster_agree_bitwise():
    # the raster's phase and absorption words are integer sums, so the tile
    # kernel and the strip pass compose bitwise the same exit waves
    for size, modes, S in ((512, 1, 3), (256, 3, 5)):
        soas, optics, dev, offs = batch(40 + size, S, size, modes, 200, 3000)
        r = renderer(size, size)
        fused = r.batch(dev, offs, optics, tuning={"use_graph": 0, "raster": -1}).clone()
        tiles = r.batch(dev, offs, optics, tuning={"use_graph": 0, "raster": 1}).clone()
        graph = r.batch(dev, offs, optics, tuning={"raster": 1}).clone()
        assert r.sync_status() == 0
        assert torch.equal(fused, tiles) and torch.equal(fused, graph)
        s = S - 1
        ref = oracle.render(soas[s], soas[s].shape[1], oracle.make_optics(**optics[s]))["images"]
        assert np.abs(tiles[s].cpu().numpy().astype(np.float64) - ref).max() <= 2e-4
