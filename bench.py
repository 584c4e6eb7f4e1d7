"""Throughput of the OSOG render path on GB300.

One step = one batched render (osog_batch_submit, replayed as a CUDA graph)
of 32 scenes of 2048 x 2048 pixels whose particle counts are log-uniform in
[1,000, 40,000] (one scene holds exactly 40,000), oblique illumination
(NA 0.4, pupil offset 0.3 NA), inputs resident in HBM.  The value is
frames/s over all ranks; particles/s, the per-scene-launch comparison, the
single 40,000-particle scene, per-kernel times and the roofline of the
dominant kernel are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank renders its own batch (different seeds), no data
collective; rank 0 prints one JSON line.  --impl reference times the FP64
CPU oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2606_21381_gb300 import scenes  # noqa: E402

METRIC = ("frames/s & particles/s at 2048²/40k particles; fwd+bwd ms; "
          "% HBM roofline")
SIZE = 2048
SCENES = 32  # overridden by --scenes (small cases for profiling)
PAPER_CONTEXT = ("paper: 40,000 particles at 1024x1024 in < 50 ms (> 20 frames/s) "
                 "on one A100 (Sec. IV.C, Fig. 5)")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------ workload
def workload(seed_offset: int = 0):
    counts = scenes.batch_2048_counts(seed=100 + seed_offset, scenes=SCENES)
    soas, optics = [], []
    for s, c in enumerate(counts):
        soa, o = scenes.batch_2048_scene(s + seed_offset, c, SIZE)
        soas.append(soa)
        optics.append(o)
    return counts, soas, optics


def workload_config(counts):
    return {"workload": f"batched render, {SCENES} scenes of {SIZE}x{SIZE}, particles "
                        f"log-uniform in [1000, 40000] (one scene 40000), oblique NA 0.4",
            "scenes": SCENES, "H": SIZE, "W": SIZE, "modalities": 1,
            "particles_per_batch": int(sum(counts)), "max_particles": int(max(counts)),
            "l2": "flushed between timed steps (256 MB write)"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def __enter__(self):
        def run():
            while not self._stop.is_set():
                try:
                    out = subprocess.run(
                        ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                         "--format=csv,noheader,nounits"], capture_output=True, text=True,
                        timeout=5).stdout.strip()
                    if out:
                        self.rows.append([x.strip() for x in out.split(",")])
                except Exception:
                    pass
                self._stop.wait(0.1)
        self._t = threading.Thread(target=run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        sm, mx, reasons = [], [], set()
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except ValueError:
                continue
            for k, v in zip(names, r[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def measured_peaks(kind: str = "hbm"):
    """(peak, source): HBM copy GB/s, or dense bf16 TFLOP/s as a burst."""
    key, fallback = {"hbm": ("hbm_gbs", 6800.0), "bf16": ("bf16_tflops", 1900.0)}[kind]
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d[key]), "measured"
    except Exception:
        return fallback, "fallback"


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if
    it was taken on the current kernel sources (matching source digest)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    digest = source_digest()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel \
                and parts[1] == digest:
            return float(parts[2])
    return None


RENDER_SOURCES = ("osog_api.cu", "osog_bin.cu", "osog_render.cu", "osog_common.cuh",
                  "osog_fft.cuh", "osog_strip.cuh", "osog_kernels.h")


def ncu_instructions(kernel: str):
    """Warp instructions per launch of `kernel` from the committed ncu
    summary, if taken on the current render sources."""
    path = os.path.join(ROOT, "profiles", "ncu_instructions.txt")
    if not os.path.exists(path):
        return None
    digest = source_digest()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel \
                and parts[1] == digest:
            return float(parts[2])
    return None


def sm_count(device=None) -> int:
    """Streaming multiprocessors of the device (152 on a GB300)."""
    import torch
    return int(torch.cuda.get_device_properties(device or 0).multi_processor_count)


def issue_peak_ginst(sms: int):
    """Warp-instruction issue peak (G/s): one warp instruction per clock
    on each of the 4 sub-partitions of every SM at the measured maximum SM
    clock."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
    except Exception:
        mhz = 2070.0
    return 4 * sms * mhz / 1e3


def source_digest(csrc: str | None = None) -> str:
    """Hash of the code the render kernels and their launches are built
    from (the convolution and noise kernels do not enter): comments and
    blank lines are removed first, so that editing a comment keeps the
    recorded counters valid while any change to the code voids them."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = csrc or os.path.join(ROOT, "paper_2606_21381_gb300", "csrc")
    for f in RENDER_SOURCES:
        text = open(os.path.join(csrc, f), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        lines = [ln.rstrip() for ln in text.splitlines() if ln.strip()]
        h.update("\n".join(lines).encode())
    return h.hexdigest()[:12]


def active_fraction(optics: dict) -> float:
    """Fraction of DFT columns that some selected pupil passes at all: the
    render writes, filters and reads only these columns of the row spectra.
    Computed here from the optics (measurement bookkeeping only)."""
    W, dx, lam, NA = optics["W"], optics["dx"], optics["lambda_um"], optics["NA"]
    r = NA / lam
    f = np.fft.fftfreq(W, dx)
    act = np.zeros(W, bool)
    for bit in (1, 2, 4):
        if optics["modes"] & bit:
            ox = optics["oblique_frac"] * r * np.cos(optics["oblique_angle"]) if bit == 2 else 0.0
            act |= (f + ox) ** 2 <= r * r
    return float(act.mean())


def algorithmic_bytes(kernel: str, counts, H: int, W: int, K: int, pairs: int,
                      active: float = 1.0):
    """Minimum HBM bytes of one launch of each kernel over the batch, per
    pixel of every scene: 8 B for the row spectra G written by the strip
    pass, 8 + 8K B for the column pass's read of G and write of the K
    filtered spectra Q, 8K + 4K B for the inverse pass's read of Q and write
    of the float32 images (16 + 20K B/px in all), plus 36 B of particle
    tensor, 64 + 48 + 8 B of records and rectangle per particle written at
    setup, read again by the raster (48 + 8 B), and 4 B per particle-band
    pair.  With active < 1 the G and Q terms count only the
    columns some pupil passes (the pruned figure: the render never writes
    or reads the others)."""
    px = len(counts) * H * W
    n = int(sum(counts))
    return int({
        "bin_count": n * (36 + 64 + 48 + 8),
        "bin_scan": 0,
        "bin_fill": n * 8 + pairs * 4,
        # the tile raster: records and rectangles in, pair ids; the per-pixel
        # phase words it hands to the strip pass are not algorithmic bytes
        # (a fused pass keeps them on chip), so the strip pass counts G only
        "raster": n * (48 + 8) + pairs * 4,
        "strip_forward": px * 8 * active,
        "column": px * (8 + 8 * K) * active,
        "strip_inverse": px * 8 * K * active + px * 4 * K,
        # the three render stages in one launch: their bytes together
        "persistent": px * 8 * active + n * (48 + 8) + pairs * 4 + px * (8 + 8 * K) * active
        + px * 8 * K * active + px * 4 * K,
    }[kernel])


# ------------------------------------------------------------------ GPU arm
def bind_to_gpu_numa_node(local_rank: int):
    """Restrict this process to the CPUs of the GPU's NUMA node (from sysfs),
    so that pinned host buffers are allocated next to the GPU's link.
    Returns the node, or None where the topology is not exposed."""
    import torch
    try:
        props = torch.cuda.get_device_properties(local_rank)
        bus = f"{props.pci_domain_id:04x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
        node = int(open(f"/sys/bus/pci/devices/{bus}/numa_node").read().strip())
        if node < 0:
            return None
        cpus = set()
        for part in open(f"/sys/devices/system/node/node{node}/cpulist").read().strip().split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        if cpus:
            os.sched_setaffinity(0, cpus)
        return node
    except Exception:
        return None


def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2606_21381_gb300.render import Renderer

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    numa_node = bind_to_gpu_numa_node(local_rank)
    counts, soas, optics = workload(seed_offset=1000 * rank)
    soa_all, offs = scenes.concat(soas)
    K = 1
    r = Renderer(SIZE, SIZE, dev)
    soa_dev = torch.from_numpy(soa_all).to(dev)
    out = torch.empty((SCENES, K, SIZE, SIZE), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    fixed = json.loads(args.tuning) if args.tuning else None

    def step(tuning=None):
        t = dict(fixed or {}, **(tuning or {})) if (fixed or tuning) else None
        r.batch(soa_dev, offs, optics, out=out, tuning=t, stream=stream)

    with torch.cuda.stream(stream):
        # the project's autotuner picks band height, pair reservation and
        # launch mode for this batch shape; later submits use its choice
        # (a fixed --tuning replaces it in profiling runs)
        tuned = dict(fixed) if fixed else r.autotune(soa_dev, offs, optics, out=out, stream=stream)
        for _ in range(max(3, args.warmup)):
            flush.fill_(1)
            step()
        stream.synchronize()
        if r.sync_status(stream) != 0:
            raise RuntimeError("device status set during warm-up")

        # ---- timed region: graph replays, per-step events on the launch stream
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        launches0 = r.launch_count()
        barrier()
        torch.cuda.synchronize(dev)
        with ClockSampler(local_rank) as clocks:
            t0 = time.perf_counter()
            for i in range(args.steps):
                flush.fill_(i & 0xff)
                starts[i].record(stream)
                step()
                ends[i].record(stream)
            torch.cuda.synchronize(dev)
            wall = time.perf_counter() - t0
        barrier()
        launches = r.launch_count() - launches0
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        timed_ms = float(sum(step_ms))

        # ---- per-kernel times: the timed configuration (direct launches,
        #      events per kernel), then the three-launch breakdown
        r.profile_begin()
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            step({"use_graph": 0})
        prof = r.profile_end(stream)
        r.profile_begin()
        for i in range(min(args.steps, 20)):
            flush.fill_(i & 0xff)
            step({"use_graph": 0, "persistent": -1})
        prof3 = r.profile_end(stream)

        # ---- both launch modes of the batched path (graph replays)
        modes_ms = {}
        for name, pers in (("three_launch", -1), ("persistent", 1)):
            t = []
            for i in range(max(3, min(args.steps, 20))):
                flush.fill_(1)
                a, b = torch.cuda.Event(True), torch.cuda.Event(True)
                a.record(stream)
                step({"persistent": pers})
                b.record(stream)
                stream.synchronize()
                t.append(a.elapsed_time(b))
            modes_ms[name] = round(statistics.median(t[1:]), 4)

        # ---- per-scene launches of the same batch (osog_render per scene)
        per_scene_ms, single40k, e2e_ms = [float("nan")], [float("nan")], [float("nan")]
        if args.quick:
            status = r.sync_status(stream)
            if status != 0:
                raise RuntimeError(f"device status {status} after the timed runs")
            return finish(args, rank, world, dev, counts, soa_all, timed_ms, prof, per_scene_ms,
                          single40k, e2e_ms, launches, clocks, wall, K,
                          extra={"autotuned": tuned, "kernels_three_launch": prof3})
        per_scene_ms = []
        singles = [torch.from_numpy(s).to(dev) for s in soas]
        for i in range(max(2, args.steps // 4)):
            flush.fill_(1)
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record(stream)
            for s in range(SCENES):
                r.render(singles[s], None, optics[s], out=out[s], stream=stream)
            b.record(stream)
            stream.synchronize()
            per_scene_ms.append(a.elapsed_time(b))
        big = int(np.argmax(counts))
        single40k = []
        for i in range(max(5, args.steps)):
            flush.fill_(1)
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record(stream)
            r.render(singles[big], None, optics[big], out=out[big], stream=stream)
            b.record(stream)
            stream.synchronize()
            single40k.append(a.elapsed_time(b))

        # ---- the 16 x 1024^2 DIC batch
        dic_batch = dic_1024_batch(dev, stream, args.steps, *measured_peaks())

        # ---- forward + adjoint of the inverse-rendering scene (512^2, 200
        #      particles, brightfield + DIC), one loss gradient per iteration
        fb_soa, fb_o = scenes.inverse_512()
        fb_r = Renderer(512, 512, dev)
        fb_x = torch.from_numpy(fb_soa).to(dev)
        fb_w = torch.randn((2, 512, 512), device=dev)
        # one training step's pair of calls: the forward keeps its
        # intermediates (osog_render_keep), the adjoint reads them
        # (osog_render_backward_kept); and the pair that recomputes them
        fb_ms, fb_re_ms = [], []
        fb_ws = None
        for i in range(max(5, min(args.steps, 50)) + 3):
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record(stream)
            img, fb_ws = fb_r.render_keep(fb_x, None, fb_o, ws=fb_ws, stream=stream)
            fb_r.backward_kept(fb_x, None, fb_o, fb_w, fb_ws, stream=stream)
            b.record(stream)
            stream.synchronize()
            if i >= 3:
                fb_ms.append(a.elapsed_time(b))
        for i in range(max(5, min(args.steps, 50)) + 3):
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record(stream)
            img = fb_r.render(fb_x, None, fb_o, stream=stream)
            fb_r.backward(fb_x, None, fb_o, fb_w, stream=stream)
            b.record(stream)
            stream.synchronize()
            if i >= 3:
                fb_re_ms.append(a.elapsed_time(b))
        if fb_r.sync_status(stream) != 0:
            raise RuntimeError("device status set in the forward + adjoint run")
        del img
        # the same on one DIC 1024^2 image (4,000 particles, K = 1)
        c1_soa, c1_o = scenes.dic_1024(0)
        c1_r = Renderer(1024, 1024, dev)
        c1_x = torch.from_numpy(c1_soa).to(dev)
        c1_w = torch.randn((1, 1024, 1024), device=dev)
        fb1_ms = []
        c1_ws = None
        for i in range(max(5, min(args.steps, 50)) + 3):
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record(stream)
            _, c1_ws = c1_r.render_keep(c1_x, None, c1_o, ws=c1_ws, stream=stream)
            c1_r.backward_kept(c1_x, None, c1_o, c1_w, c1_ws, stream=stream)
            b.record(stream)
            stream.synchronize()
            if i >= 3:
                fb1_ms.append(a.elapsed_time(b))
        if c1_r.sync_status(stream) != 0:
            raise RuntimeError("device status set in the DIC 1024 forward + adjoint run")
        # bitwise determinism of the batched render: two renders, same bytes
        step()
        out2 = out.clone()
        step()
        deterministic = bool(torch.equal(out2, out))
        del out2
    with torch.cuda.stream(stream):
        # ---- end to end from pinned host buffers through the public API:
        #      each step copies its particles in and its images out; the
        #      pipeline overlaps one step's copies with the next step's render
        from paper_2606_21381_gb300.render import HostBatchPipeline
        soa_host = torch.from_numpy(soa_all).pin_memory()
        img_host = [torch.empty((SCENES, K, SIZE, SIZE), dtype=torch.float32).pin_memory()
                    for _ in range(2)]
        e2e_ms = []  # serial: one step at a time on one stream
        for i in range(max(3, min(args.steps // 2, 20))):
            flush.fill_(1)
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record(stream)
            d = soa_host.to(dev, non_blocking=True)
            r.batch(d, offs, optics, out=out, stream=stream)
            img_host[0].copy_(out, non_blocking=True)
            b.record(stream)
            stream.synchronize()
            e2e_ms.append(a.elapsed_time(b))
    pipe = HostBatchPipeline(r, soa_all.shape[1], SCENES, K)
    for i in range(2):
        pipe.submit(soa_host, offs, optics, img_host[i % 2])
    pipe.synchronize()
    n_pipe = max(4, min(args.steps, 40))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i in range(n_pipe):
        pipe.submit(soa_host, offs, optics, img_host[i % 2])
    pipe.synchronize()
    pipe_s = time.perf_counter() - t0
    del pipe
    # the device-to-host rate of the image batch alone (the pipeline's bound
    # once its copies overlap the renders)
    d2h_ms = []
    for i in range(3):
        a, b = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record(stream)
        img_host[0].copy_(out, non_blocking=True)
        b.record(stream)
        stream.synchronize()
        d2h_ms.append(a.elapsed_time(b))
    with torch.cuda.stream(stream):
        status = r.sync_status(stream)
        if status != 0:
            raise RuntimeError(f"device status {status} after the timed runs")
    # the learned warm start last, in a process of its own: its training
    # allocates and pins its own buffers, which should not share allocator
    # state with the measurements above
    warm = None if (args.no_warm_start or rank != 0) else warm_start_in_child(local_rank)
    return finish(args, rank, world, dev, counts, soa_all, timed_ms, prof, per_scene_ms,
                  single40k, e2e_ms, launches, clocks, wall, K, soas=soas, optics=optics,
                  fwd_bwd_ms=fb_ms, extra={"autotuned": tuned, "batched_modes_ms": modes_ms,
                                           "kernels_three_launch": prof3, "warm_start": warm,
                                           "numa_node": numa_node, "fwd_bwd_dic1024_ms": fb1_ms,
                                           "fwd_bwd_recompute_ms": fb_re_ms,
                                           "deterministic": deterministic,
                                           "dic_1024_batch": dic_batch,
                                           "e2e_pipelined": (n_pipe, pipe_s),
                                           "d2h_ms": min(d2h_ms)})


def conv_profile(net, x, reps: int = 10):
    """Per-launch CUDA-event times of every convolution kernel call of one
    training step (forward, data and filter gradients of each layer) on the
    batch x, with the algorithmic FLOPs 2 N P Q K R S C of each."""
    import torch

    from paper_2606_21381_gb300 import cnn
    out, acts = net.forward(x)
    rows = []
    for i, (cin, cout, k, stride, pad) in enumerate(net.specs):
        a = acts[i]
        y = acts[i + 1] if i + 1 < len(acts) else out.to(torch.bfloat16)
        dy = torch.ones_like(y)
        calls = [("fwd", lambda: cnn.conv2d(a, net.wb[i], net.b[i], stride, pad, True)),
                 ("wgrad", lambda: cnn.conv2d_backward_filter(dy, a, tuple(net.w[i].shape),
                                                              stride, pad))]
        if i > 0:
            calls.append(("dgrad", lambda: cnn.conv2d_backward_data(dy, net.wb[i], tuple(a.shape),
                                                                    stride, pad, x_act=a)))
        flops = 2.0 * a.shape[0] * y.shape[1] * y.shape[2] * cout * k * k * cin
        for name, fn in calls:
            fn()
            e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            rows.append({"layer": i, "pass": name, "ms": round(ms, 4),
                         "tflops": round(flops / (ms / 1e3) / 1e12, 2)})
    return rows


def _warm_start_child(local_rank: int, queue) -> None:
    import torch
    torch.cuda.set_device(local_rank)
    try:
        queue.put(("ok", warm_start_bench(torch.device("cuda", local_rank))))
    except Exception as e:  # reported by the parent
        queue.put(("error", repr(e)))


def warm_start_in_child(local_rank: int):
    """warm_start_bench in a spawned process on the same GPU (the parent
    waits idle)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_warm_start_child, args=(local_rank, q))
    p.start()
    status, result = q.get()
    p.join()
    if status != "ok":
        raise RuntimeError(f"warm-start benchmark failed: {result}")
    return result


def convs_only(reps: int = 10) -> None:
    """Per-launch times of the network's convolutions on a 64-crop batch
    with the tcgen05 engine and with the warp-level MMA (random weights;
    the kernels' work does not depend on their values)."""
    import torch

    from paper_2606_21381_gb300 import cnn
    from paper_2606_21381_gb300.render import Renderer
    dev = torch.device("cuda")
    r = Renderer(512, 512, dev)
    net = cnn.WarmStartNet(dev, seed=0)
    x, _, _ = cnn.RenderStream(r, 16, 256, seed=5).next()
    out = {}
    for engine in ("tcgen05", "mma_sync"):
        cnn.use_tcgen05(engine == "tcgen05")
        out[engine] = conv_profile(net, x, reps)
    cnn.use_tcgen05(True)
    if cnn.sync_status() != 0:
        raise RuntimeError("convolution status set")
    print(json.dumps({"workload": "6-layer warm-start CNN, batch of 64 crops of 256x256",
                      "conv_kernels": out}))


def warm_start_bench(dev, samples: int = 200_000, seeds=(7, 9, 10)):
    """Learned warm start on the 512^2 inverse-rendering scene: train the
    network on `samples` rendered crops, then time the plain and the
    warm-started solves to 1% median dn and T error from the same perturbed
    guesses (500 curriculum steps)."""
    import torch

    from paper_2606_21381_gb300 import cnn, inverse
    from paper_2606_21381_gb300.render import Renderer
    r = Renderer(512, 512, dev)
    # warm-up of every code path the timed training takes (kernel modules,
    # the captured step), on a network of its own
    cnn.train(cnn.WarmStartNet(dev, seed=1), cnn.TrainConfig(samples=64 * 8, seed=99), r)
    net = cnn.WarmStartNet(dev, seed=0)
    tr = cnn.train(net, cnn.TrainConfig(samples=samples), r)
    ev = cnn.calibrate(net, r)
    x, _, _ = cnn.RenderStream(r, 16, 256, seed=5).next()
    convs = conv_profile(net, x)
    soa, o = scenes.inverse_512()
    o = dict(o, defocus=0.8, shear_px=1.0)
    target = r.render(torch.from_numpy(soa).to(dev), None, o)
    s0, o0 = inverse.perturb(soa, o, np.random.default_rng(seeds[0]))
    inverse.solve(target, s0, o0, r, inverse.SolveConfig(steps=20, record_every=5),
                  truth=soa)  # warm-up of every code path the timed solves take
    arms = {"plain": [], "warm": []}
    for seed in seeds:
        s0, o0 = inverse.perturb(soa, o, np.random.default_rng(seed))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        sw, ow = cnn.warm_start(net, target, s0, o0)
        torch.cuda.synchronize(dev)
        t_inf = time.perf_counter() - t0
        cfg = inverse.SolveConfig(steps=500, record_every=5)
        for arm, (ss, oo, extra) in (("plain", (s0, o0, 0.0)), ("warm", (sw, ow, t_inf))):
            res = inverse.solve(target, ss, oo, r, cfg, truth=soa)
            hit = inverse.time_to_error(res.history)
            e = inverse.errors(res.soa, soa, res.optics_params, o)
            arms[arm].append({"seed": seed, "steps_to_1pct": hit[0] if hit else None,
                              "seconds_to_1pct": round(hit[1] + extra, 4) if hit else None,
                              "start_s": round(extra, 4),
                              "final_frac_within_1pct": round(e["frac_dn_T_within_1pct"], 3)})
    if r.sync_status() != 0:
        raise RuntimeError("device status set in the warm-start run")
    mean = lambda arm, k: (statistics.mean(a[k] for a in arms[arm])
                           if all(a[k] is not None for a in arms[arm]) else None)
    peak_t = measured_peaks(kind="bf16")
    dom = max(convs, key=lambda c: c["ms"])
    tot = sum(c["ms"] for c in convs)
    flops_tot = sum(c["tflops"] * c["ms"] for c in convs)  # TF/s x ms = GFLOP
    return {
        "workload": "6-layer BF16 CNN (32-64-128-128-64-32, 3x3) on 256x256 brightfield + DIC "
                    "crops of batched 512x512 renders, then the 512x512 / 200-particle inverse "
                    "solve (500 curriculum steps) from perturbed guesses",
        "train": {"samples": tr.samples, "steps": tr.steps, "seconds": round(tr.seconds, 2),
                  "samples_per_s": round(tr.samples / tr.seconds, 1),
                  "final_loss": round(float(tr.losses[-50:, 0].mean()), 4)},
        "held_out_rms": {k: round(v, 5) for k, v in ev.items()},
        "inverse_512": arms,
        "mean_steps_to_1pct": {"plain": mean("plain", "steps_to_1pct"),
                               "warm": mean("warm", "steps_to_1pct")},
        "mean_seconds_to_1pct": {"plain": mean("plain", "seconds_to_1pct"),
                                 "warm": mean("warm", "seconds_to_1pct")},
        "conv_kernels": convs,
        "roofline": {"bound": "tensor", "kernel": f"layer {dom['layer']} {dom['pass']}",
                     "achieved": dom["tflops"], "peak": peak_t[0], "unit": "TFLOP/s",
                     "frac": round(dom["tflops"] / peak_t[0], 4), "peak_source": peak_t[1],
                     "step_convs_tflops": round(flops_tot / tot, 2)},
    }


def issue_roofline(kernels: dict, sms: int):
    """The bound the render kernels actually meet: warp instructions per
    launch (committed ncu counts) over the live launch time, against the
    issue peak."""
    peak = issue_peak_ginst(sms)
    out = {}
    for k in ("strip_forward", "column", "strip_inverse"):
        inst = ncu_instructions(k)
        if inst is None or k not in kernels:
            continue
        rate = inst / (kernels[k]["ms_per_launch"] / 1e3) / 1e9
        out[k] = {"warp_instructions": inst, "achieved_ginst_s": round(rate, 1),
                  "frac": round(rate / peak, 4)}
    return {"bound": "issue", "unit": "G warp-instructions/s", "peak": round(peak, 1),
            "kernels": out} if out else None


def single_scene_entry(ms_list, n: int, K: int, peak: float, peak_src: str) -> dict:
    """The 40,000-particle 2048^2 scene rendered alone (osog_render): frames/s
    and its whole-frame roofline (16 + 20K B/px plus particle and bin bytes
    over the event-timed frame)."""
    ms = statistics.median(ms_list)
    b = sum(algorithmic_bytes(k, [n], SIZE, SIZE, K, 2 * n)
            for k in ("bin_count", "bin_fill", "raster", "strip_forward", "column",
                      "strip_inverse"))
    gbs = b / (ms / 1e3) / 1e9
    return {"ms": round(ms, 4), "frames_per_s": round(1e3 / ms, 2),
            "particles_per_s": round(n / (ms / 1e3), 1),
            "roofline": {"bound": "hbm", "algorithmic_bytes": b, "achieved": round(gbs, 1),
                         "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
                         "peak_source": peak_src},
            "context": PAPER_CONTEXT}


def dic_1024_batch(dev, stream, steps: int, peak: float, peak_src: str) -> dict:
    """16 DIC images of 1024^2 with 4,000 particles each (shear 1 px at 45
    degrees, bias pi/4, NA 0.5, defocus U(-2, 2) um per image), rendered as
    one batch replayed as a CUDA graph: frames/s and the step's roofline."""
    import torch

    from paper_2606_21381_gb300.render import Renderer
    soas, optics = zip(*[scenes.dic_1024(i) for i in range(16)])
    soa_all, offs = scenes.concat(list(soas))
    r = Renderer(1024, 1024, dev)
    x = torch.from_numpy(soa_all).to(dev)
    out = torch.empty((16, 1, 1024, 1024), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        r.autotune(x, offs, list(optics), out=out, stream=stream)
        for _ in range(3):
            r.batch(x, offs, list(optics), out=out, stream=stream)
        t = []
        for i in range(max(5, min(steps, 50))):
            flush.fill_(i & 0xff)
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record(stream)
            r.batch(x, offs, list(optics), out=out, stream=stream)
            b.record(stream)
            stream.synchronize()
            t.append(a.elapsed_time(b))
        if r.sync_status(stream) != 0:
            raise RuntimeError("device status set in the DIC 1024 batch")
    counts = [s.shape[1] for s in soas]
    ms = statistics.median(t)
    b = sum(algorithmic_bytes(k, counts, 1024, 1024, 1, 2 * sum(counts))
            for k in ("bin_count", "bin_fill", "raster", "strip_forward", "column",
                      "strip_inverse"))
    gbs = b / (ms / 1e3) / 1e9
    return {"workload": "16 x 1024^2 DIC, 4,000 particles per image, NA 0.5, shear 1 px at 45 "
                        "deg, bias pi/4, defocus U(-2, 2) um; one batch as a CUDA graph",
            "ms_per_batch": round(ms, 4), "frames_per_s": round(16 / (ms / 1e3), 1),
            "particles_per_s": round(sum(counts) / (ms / 1e3), 1),
            "roofline": {"bound": "hbm", "algorithmic_bytes": b, "achieved": round(gbs, 1),
                         "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
                         "peak_source": peak_src}}


def max_over_ranks(value: float, world: int, device) -> float:
    """The largest value over all ranks (the slowest rank's timed region)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_step_per_rank: float, steps: int, world: int,
                   max_ms: float) -> float:
    """Whole-job units per second: every rank's units over the slowest
    rank's time (weak scaling: each rank renders its own batch)."""
    return units_per_step_per_rank * steps * world / (max_ms / 1e3)


def finish(args, rank, world, dev, counts, soa_all, timed_ms, prof, per_scene_ms, single40k,
           e2e_ms, launches, clocks, wall, K, soas=None, optics=None, fwd_bwd_ms=None,
           extra=None):
    timed_max = max_over_ranks(timed_ms, world, dev)
    value = job_throughput(SCENES, args.steps, world, timed_max)
    if rank != 0:
        return None

    # dominant kernel and its roofline
    kernels = {k: {"ms_total": v[0], "launches": v[1], "ms_per_launch": v[0] / v[1]}
               for k, v in prof.items() if v[1] > 0}
    tot = sum(v["ms_total"] for v in kernels.values()) or 1.0
    for v in kernels.values():
        v["share"] = v["ms_total"] / tot
    dom = max(kernels, key=lambda k: kernels[k]["ms_total"])
    pairs_est = int(sum(counts) * 2)
    peak, peak_src = measured_peaks()
    act = active_fraction(scenes.batch_2048_scene(0, 1, SIZE)[1])
    bytes_dom = algorithmic_bytes(dom, counts, SIZE, SIZE, K, pairs_est)
    bytes_dom_pruned = algorithmic_bytes(dom, counts, SIZE, SIZE, K, pairs_est, act)
    dur_s = kernels[dom]["ms_per_launch"] / 1e3
    achieved = bytes_dom / dur_s / 1e9
    traffic = ncu_traffic(dom)
    step_bytes = sum(algorithmic_bytes(k, counts, SIZE, SIZE, K, pairs_est) for k in kernels)
    step_bytes_pruned = sum(algorithmic_bytes(k, counts, SIZE, SIZE, K, pairs_est, act)
                            for k in kernels)
    ms_step = timed_max / args.steps
    return {
        "metric": METRIC, "value": round(value, 2), "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded scenes shaped like the paper's workloads)",
        "config": dict(workload_config(counts), parallelism=f"replicas x{world}",
                       tuning=(extra or {}).get("autotuned")),
        "particles_per_s": round(sum(counts) * args.steps * world / (timed_max / 1e3), 1),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic, "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": bytes_dom,
                     "pruned": {"what": "G and Q counted only on the pupil-passed columns "
                                        "(the bytes the kernel does move)",
                                "pupil_active_columns": round(act, 4),
                                "algorithmic_bytes_per_launch": bytes_dom_pruned,
                                "achieved": round(bytes_dom_pruned / dur_s / 1e9, 1),
                                "frac": round(bytes_dom_pruned / dur_s / 1e9 / peak, 4)}},
        "issue_roofline": issue_roofline(kernels, sm_count(dev)),
        "step_roofline": {"algorithmic_bytes": step_bytes,
                          "achieved_gbs": round(step_bytes / (ms_step / 1e3) / 1e9, 1),
                          "frac": round(step_bytes / (ms_step / 1e3) / 1e9 / peak, 4),
                          "pruned_frac": round(step_bytes_pruned / (ms_step / 1e3) / 1e9 / peak, 4)},
        "kernels": kernels,
        "kernels_three_launch": {k: {"ms_per_launch": v[0] / v[1], "share": v[0] / max(
            sum(x[0] for x in (extra or {}).get("kernels_three_launch", {}).values()), 1e-30)}
            for k, v in (extra or {}).get("kernels_three_launch", {}).items() if v[1] > 0},
        "batched_modes_ms": (extra or {}).get("batched_modes_ms"),
        "per_scene_launches": None if args.quick else {
                               "ms_per_batch": round(statistics.median(per_scene_ms), 4),
                               "frames_per_s": round(SCENES / (statistics.median(per_scene_ms) / 1e3), 2),
                               "batched_speedup": round(statistics.median(per_scene_ms) / ms_step, 3)},
        "single_scene_40k": None if args.quick else single_scene_entry(
            single40k, max(counts), K, peak, peak_src),
        "dic_1024_batch": (extra or {}).get("dic_1024_batch"),
        "e2e": None if args.quick else {
                "value": round(SCENES * extra["e2e_pipelined"][0] / extra["e2e_pipelined"][1], 2),
                "unit": "frames/s",
                "h2d_bytes_per_step": int(soa_all.nbytes),
                "d2h_bytes_per_step": int(SCENES * K * SIZE * SIZE * 4),
                "how": "HostBatchPipeline: pinned host particles in, pinned host images out, "
                       "every step; copies of one step overlap the render of the next; "
                       "host wall clock over %d steps" % extra["e2e_pipelined"][0],
                "serial_value": round(SCENES / (statistics.median(e2e_ms) / 1e3), 2),
                "host_numa_node": extra.get("numa_node"),
                "d2h_gbs": round(SCENES * K * SIZE * SIZE * 4 / extra["d2h_ms"] / 1e6, 1),
                "copy_bound_value": round(SCENES / (max(extra["d2h_ms"], ms_step) / 1e3), 2),
                "bound": "the image batch's device-to-host copy (d2h_gbs) or the render, "
                         "whichever is longer, with copies and renders fully overlapped"},
        "fwd_bwd": None if not fwd_bwd_ms else {
            "ms": round(statistics.median(fwd_bwd_ms), 4),
            "workload": "512x512, 200 particles, brightfield + DIC: osog_render_keep + "
                        "osog_render_backward_kept (forward intermediates kept, adjoint)",
            "ms_recomputed": round(statistics.median(extra["fwd_bwd_recompute_ms"]), 4),
            "recomputed": "osog_render + osog_render_backward (the adjoint recomputes the forward)",
            "dic_1024_ms": round(statistics.median(extra["fwd_bwd_dic1024_ms"]), 4),
            "dic_1024_workload": "1024x1024, 4,000 particles, DIC (K = 1), defocus"},
        "bitwise_deterministic": (extra or {}).get("deterministic"),
        "warm_start": (extra or {}).get("warm_start"),
        "gpu_launches": int(launches),
        "clocks": clocks.summary(),
        "wall_s_timed": round(wall, 4),
        "cpu_baseline": cpu_baseline(soas, optics, counts)
        if (world == 1 and soas is not None) else None,
    }


# ------------------------------------------------------------------ CPU oracle
def oracle_frames(soas, optics, budget_s: float, max_scenes: int, start: int = 0):
    import oracle
    done, t0, parts = 0, time.perf_counter(), 0
    i = start
    while done < max_scenes:
        soa = soas[i % len(soas)]
        oracle.render(soa, soa.shape[1], oracle.make_optics(**optics[i % len(soas)]))
        done += 1
        parts += soa.shape[1]
        i += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    return done, parts, time.perf_counter() - t0


def oracle_config_times(counts, soas, optics) -> dict:
    """Seconds per frame of the oracle on the plain 256^2 scene, one DIC
    1024^2 image and the 40,000-particle 2048^2 scene, on all host cores
    and on one."""
    import oracle
    cases = {"plain_256": scenes.plain_256(),
             "dic_1024_image": scenes.dic_1024(0),
             "scene_2048_40k": (soas[int(np.argmax(counts))], optics[int(np.argmax(counts))])}
    out = {}
    for threads in (os.cpu_count(), 1):
        oracle.set_threads(threads)
        for name, (soa, o) in cases.items():
            t0 = time.perf_counter()
            oracle.render(soa, soa.shape[1], oracle.make_optics(**o))
            out.setdefault(name, {})[f"s_{threads}_cores"] = round(time.perf_counter() - t0, 4)
    oracle.set_threads(os.cpu_count())
    return out


def cpu_baseline(soas, optics, counts):
    import oracle
    oracle.build()
    n, parts, dt = oracle_frames(soas, optics, budget_s=15.0, max_scenes=SCENES)
    return {"value": round(n / dt, 4), "unit": "frames/s", "cores": os.cpu_count(),
            "kind": "oracle", "particles_per_s": round(parts / dt, 1),
            "sample": f"{n} of the {SCENES} scenes ({parts} particles), FP64 C oracle, "
                      f"OpenMP over FFT lines, {dt:.1f} s",
            "per_config": oracle_config_times(counts, soas, optics)}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle
    oracle.build()
    counts, soas, optics = workload()
    for i in range(args.warmup):
        oracle_frames(soas, optics, 0.0, 1, start=i)
    t0 = time.perf_counter()
    parts = 0
    for i in range(args.steps):
        _, p, _ = oracle_frames(soas, optics, 0.0, 1, start=args.warmup + i)
        parts += p
    dt = time.perf_counter() - t0
    value = args.steps / dt
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "frames/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded scenes shaped like the paper's workloads)",
            "config": workload_config(counts),
            "cpu_baseline": {"value": round(value, 4), "unit": "frames/s",
                             "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"one {SIZE}x{SIZE} scene of the batch per step "
                                       f"({parts} particles over {args.steps} steps)"},
            "e2e": {"value": round(value, 4), "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def fwd_bwd_only(reps: int = 5) -> None:
    """The inverse-rendering scene's training step alone (512^2, 200
    particles, brightfield + DIC): `reps` pairs of osog_render_keep and
    osog_render_backward_kept, timed with CUDA events (profiling runs)."""
    import torch

    from paper_2606_21381_gb300 import scenes
    from paper_2606_21381_gb300.render import Renderer
    dev = torch.device("cuda")
    soa, o = scenes.inverse_512()
    r = Renderer(512, 512, dev)
    x = torch.from_numpy(soa).to(dev)
    w = torch.randn((2, 512, 512), device=dev)
    ws, ms = None, []
    for _ in range(reps):
        a, b = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        _, ws = r.render_keep(x, None, o, ws=ws)
        r.backward_kept(x, None, o, w, ws)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    if r.sync_status() != 0:
        raise RuntimeError("device status set in the forward + adjoint run")
    print(json.dumps({"workload": "512x512, 200 particles, brightfield + DIC: "
                                  "osog_render_keep + osog_render_backward_kept",
                      "ms": [round(v, 4) for v in ms]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="osog", choices=["osog", "reference"])
    ap.add_argument("--scenes", type=int, default=32,
                    help="scenes per batch (32 is the benchmarked workload)")
    ap.add_argument("--convs-only", action="store_true",
                    help="time the warm-start network's convolution kernels on one 64-crop "
                         "batch (both tensor-core engines) and exit")
    ap.add_argument("--fwd-bwd-only", action="store_true",
                    help="run five forward + adjoint pairs of the 512x512 inverse-rendering "
                         "scene and exit (profiling runs)")
    ap.add_argument("--no-warm-start", action="store_true",
                    help="skip the learned warm-start benchmark (training + inverse solves)")
    ap.add_argument("--quick", action="store_true",
                    help="timed region and per-kernel pass only (profiling runs)")
    ap.add_argument("--tuning", default=None,
                    help="JSON tuning of the batched path used instead of the autotuner's "
                         "choice, e.g. '{\"band_rows\": 64, \"pairs_per_particle\": 2}' "
                         "(profiling runs: the kernel launches are then the same every run)")
    args = ap.parse_args()
    global SCENES
    SCENES = args.scenes
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.convs_only:
        convs_only()
        return
    if args.fwd_bwd_only:
        fwd_bwd_only()
        return
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        if args.warmup < 3:
            args.warmup = 3
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl")
        res = run_gpu(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
