#!/usr/bin/env python
"""Benchmark of the halfway-domain scene-flow solve (arXiv 1610.07159).

Workload: a seeded synthetic 640x480 stereo video (30 frames of 3-6
value-noise textured planes and spheres, disparities 5-40 px, motion up to
12 px per frame), warp-grid stride 8, 4 pyramid levels, 3 Gauss-Newton x 20
PCG iterations per level, Figure-2 weights of Table 1. One step = one pass of
the whole hot path (pyramid, coarse-to-fine Gauss-Newton/PCG with the delta
hierarchy and temporal transfer) over the 30-frame video through
sf_solve_video, from a zero initialisation; the levels of consecutive frames
run concurrently (the fields equal those of frame-by-frame sf_solve, which
is timed beside it as a variant).

Metric: stereo frames/s (higher is better). Each rank solves its own
sequence (weak scaling, no collective on the data path); value = frames of
all ranks / max-over-ranks time.

Timing: W warm-up steps, then K steps, each between CUDA events on the
launching stream with an L2 flush (a 256 MB write) between steps outside
the events; inputs of all 30 frames are resident in HBM before timing.
`e2e` repeats the run through sf_solve_video_host from pinned host memory
(the copies in and out inside the timed region). `roofline` is for the kernel
class with the larger device time, measured live with CUDA events recorded
around its launches inside the pipeline, over a second timed pass of the same
K steps (the headline steps run without those events). `cpu_baseline` and
`--impl reference` time the FP64 CPU oracle on a bounded sample of the same
workload.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WIDTH, HEIGHT, STRIDE, LEVELS, GN, PCG, NFRAMES = 640, 480, 8, 4, 3, 20, 30
METRIC = "stereo frames/sec at 640x480 vs plain FP32 at equal energy; % of HBM roofline"
UNIT = "frames/s"
WORKLOAD = (f"{WIDTH}x{HEIGHT} synthetic stereo video, {NFRAMES} frames, grid stride {STRIDE}, {LEVELS} levels, "
            f"{GN} GN x {PCG} PCG per level, Figure-2 weights, FP32")
FP32_LANES_PER_SM = 128

# Algorithmic work per unit (derivations in the design notes):
#   PCG, the byte model of the hot-path scope table: per node and iteration
#   168 floats of stencil blocks (672 B) + about 8 vectors x 24 B = 860 B
#   PCG, as the one-reduction kernel (k_pcg1) moves it: per node 96 B (init)
#   + 588 B per iteration (420 B of its five 6x6 blocks, 24 B of M, 72 B of
#   published r, w, s read, 72 B written) + 24 B (solution)
#   PCG, as the staged kernels (k_pcg1h, k_pcg1p) move it, per node of a
#   level with rows of nx nodes: once per launch its five blocks staged with
#   those of the nx + 1 nodes before each 64-node segment,
#   420 B x (64 + nx + 1) / 64, plus b and M (48 B) and the solution (24 B);
#   per iteration its published vectors written as tagged 8-byte words (r, w
#   and s: 144 B for k_pcg1h, w: 48 B for k_pcg1p) and the same words of the
#   halo, 2 (nx + 1) nodes per 64 owned, with their M (24 B)
#   assembly: 2250 FP32 flops per pixel
PCG_MODEL_ITER_B = 860
PCG_INIT_B, PCG_ITER_B, PCG_OUT_B = 96, 588, 24
ASM_FLOPS_PER_PX = 2250
# kernel of each PCG schedule kind (sf_pcg_schedule)
PCG_KERNEL = {0: "k_pcg", 1: "k_pcg", 2: "k_pcg_dsm", 3: "k_pcg1", 4: "k_pcg1", 5: "k_pcg1h", 6: "k_pcg1p"}


def level_sizes():
    w, h, out = WIDTH, HEIGHT, []
    for _ in range(LEVELS):
        out.append((w, h, (w + STRIDE - 1) // STRIDE, (h + STRIDE - 1) // STRIDE))
        w, h = (w + 1) // 2, (h + 1) // 2
    return out


def pcg_bytes_per_frame(model="per_node_860"):
    """Algorithmic PCG bytes of one frame: the 860 B/node/iteration model
    ("per_node_860"), or the own count of the one-reduction kernel ("one_reduction"),
    of the staged one ("staged") or of the pipelined one ("pipelined")."""
    if model == "per_node_860":
        return sum(GN * nx * ny * PCG * PCG_MODEL_ITER_B for _, _, nx, ny in level_sizes())
    if model in ("staged", "pipelined"):
        words = 144 if model == "staged" else 48
        return sum(GN * nx * ny * (420.0 * (64 + nx + 1) / 64 + 48 + 24 +
                                   PCG * (words + (words + 24) * 2.0 * (nx + 1) / 64))
                   for _, _, nx, ny in level_sizes())
    return sum(GN * nx * ny * (PCG_INIT_B + PCG * PCG_ITER_B + PCG_OUT_B) for _, _, nx, ny in level_sizes())


def asm_flops_per_frame():
    return sum(GN * w * h * ASM_FLOPS_PER_PX for w, h, _, _ in level_sizes())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def source_hash(rel):
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def recorded_traffic(kernel):
    """Per-launch DRAM bytes from the committed ncu summary, if taken on the current source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)[kernel]
    except (OSError, ValueError, KeyError):
        return None
    if d.get("source_sha256_16") != source_hash(d["source"]):
        return None
    return d.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid, self.proc, self.lines = uuid, None, []

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(backend):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None, rank, world, local


def max_over_ranks(dist, value, device):
    """Largest value over the ranks (each rank's own timed region)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, steps, t_max_ms):
    """Frames of all ranks per second of the slowest rank (weak scaling)."""
    return world * steps / (t_max_ms / 1e3)


def cpu_baseline(video, max_seconds=20.0, max_frames=4):
    import numpy as np
    import oracle as O
    p = O.Params.preset("fig2", gn_iters=(GN,) * 8, pcg_iters=(PCG,) * 8)
    prev, n, t0 = None, 0, time.perf_counter()
    while n < max_frames and time.perf_counter() - t0 < max_seconds:
        prev = O.solve_frame(video[n].astype(np.float64), STRIDE, LEVELS, p, prev=prev)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n} frames of the same {WIDTH}x{HEIGHT} video (temporal chain), single-threaded "
                      f"FP64 C oracle, {dt:.1f} s"}


def _oracle_worker(seed, n_frames):
    """One process: renders its own seeded 640x480 video and solves its first
    n_frames with the FP64 oracle (temporal chain); returns (frames, seconds)."""
    import numpy as np
    import oracle as O
    from paper_1610_07159_gb300 import scenes
    video = scenes.SceneVideo(WIDTH, HEIGHT, n_frames, seed=seed).frames(n_frames)
    p = O.Params.preset("fig2", gn_iters=(GN,) * 8, pcg_iters=(PCG,) * 8)
    prev, t0 = None, time.perf_counter()
    for f in range(n_frames):
        prev = O.solve_frame(video[f].astype(np.float64), STRIDE, LEVELS, p, prev=prev)
    return n_frames, time.perf_counter() - t0


def cpu_baseline_all_cores(n_frames=2):
    """The same oracle on every host core at once, one independent sequence per
    process (spawned, so no CUDA state is inherited); frames of all processes /
    wall time of the solves."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        res = pool.starmap(_oracle_worker, [(7000 + i, n_frames) for i in range(cores)])
    frames = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return {"value": frames / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes, each the first {n_frames} frames of its own {WIDTH}x{HEIGHT} video "
                      f"(temporal chain), single-threaded FP64 C oracle per process; slowest process {wall:.1f} s"}


def variant_batched(dev, steps=3):
    """64 independent sequences of uneven sizes solved together: one launch per
    frame step (one thread-block cluster per sequence) under a captured graph,
    with the autotuned schedule."""
    import torch

    from paper_1610_07159_gb300 import scenes, scenes_device, sf

    sizes = scenes.batch_sizes(64, seed=4000)
    levels = [4 if w * h <= 640 * 480 else 5 for w, h in sizes]
    b = sf.Batch(sizes, levels, STRIDE, sf.preset(sf.PRESET_FIG2, gn_iters=[GN], pcg_iters=[PCG]))
    vids = [scenes_device.frames(scenes.SceneVideo(w, h, steps + 1, seed=5000 + i), steps + 1, dev,
                                 dtype=torch.float32) for i, (w, h) in enumerate(sizes)]
    packed = [b.pack([v[f] for v in vids]) for f in range(steps + 1)]
    del vids
    out = torch.empty(b.out_total, device=dev, dtype=torch.float32)
    t0 = time.time()
    b.tune(packed[0], out, steps=2)
    tune_s = time.time() - t0
    b.solve(packed[0], out)  # warm-up frame
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for f in range(1, steps + 1):
        b.solve(packed[f], out)
    e.record()
    e.synchronize()
    ms = s.elapsed_time(e) / steps
    px = sum(w * h for w, h in sizes)
    flops = sum(GN * ASM_FLOPS_PER_PX * w * h * sum(4.0 ** -l for l in range(L)) for (w, h), L in zip(sizes, levels))
    nodes = 0
    for (w, h), L in zip(sizes, levels):
        for l in range(L):
            wl, hl = -(-w // 2 ** l), -(-h // 2 ** l)
            nodes += (-(-wl // STRIDE)) * (-(-hl // STRIDE))
    pcg_bytes = GN * nodes * (PCG_INIT_B + PCG * PCG_ITER_B + PCG_OUT_B)
    energies = [b.sequence(i).stats().energy for i in range(len(sizes))]
    res = {"sequences": len(sizes), "sizes": "seeded uniform draw from {320x240, 640x480, 960x540, 1280x720}",
           "levels": "4 up to 640x480, 5 above", "ms_per_frame_step": ms, "frames_per_s": len(sizes) * 1e3 / ms,
           "Mpx_per_s": px / ms / 1e3, "schedule": {"cluster_ctas": b.schedule()[0], "cpb_div": b.schedule()[1]},
           "tune_s": tune_s, "launches_per_frame_step": 1,
           "assembly_TFLOPs": flops / (ms / 1e3) / 1e12, "pcg_GBps": pcg_bytes / (ms / 1e3) / 1e9,
           "note": "rates over the whole launch (all stages share it)",
           "all_finite": bool(all(e == e for e in energies))}
    b.close()
    return res


def variant_batched_640(dev, frames_d, n_seq=32, steps=3):
    """n_seq independent 640x480 sequences in one launch per frame step, against
    the plain FP32 solve at equal final energy (sequence 0 is the headline
    video itself; its energies are compared frame by frame with the plain
    frame-by-frame solve)."""
    import torch

    from paper_1610_07159_gb300 import scenes, scenes_device, sf

    b = sf.Batch([(WIDTH, HEIGHT)] * n_seq, [LEVELS] * n_seq, STRIDE,
                 sf.preset(sf.PRESET_FIG2, gn_iters=[GN], pcg_iters=[PCG]))
    others = [scenes_device.frames(scenes.SceneVideo(WIDTH, HEIGHT, steps + 1, seed=6000 + i), steps + 1, dev,
                                   dtype=torch.float32) for i in range(1, n_seq)]
    packed = [b.pack([frames_d[f]] + [v[f] for v in others]) for f in range(steps + 1)]
    b_in_off = list(b.in_offsets)
    del others
    out = torch.empty(b.out_total, device=dev, dtype=torch.float32)
    b.tune(packed[0], out, steps=2)
    plain = sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS, sf.preset(sf.PRESET_FIG2, gn_iters=[GN], pcg_iters=[PCG]))
    plain.tune_pcg(frames_d[0])
    out1 = torch.empty((6, HEIGHT // STRIDE, WIDTH // STRIDE), device=dev, dtype=torch.float32)
    rel = []
    ms = 0.0
    for f in range(steps + 1):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        b.solve(packed[f], out)
        e.record()
        e.synchronize()
        if f > 0:
            ms += s.elapsed_time(e)
        plain.solve(frames_d[f], out1)
        eb, ep = b.sequence(0).stats().energy, plain.stats().energy
        rel.append(abs(eb - ep) / abs(ep))
    res = {"sequences": n_seq, "frames_per_s": n_seq * steps * 1e3 / ms, "ms_per_frame_step": ms / steps,
           "schedule": {"cluster_ctas": b.schedule()[0], "cpb_div": b.schedule()[1]},
           "energy_rel_vs_plain_max": max(rel), "frames_compared": len(rel)}
    batched_energies = [b.sequence(i).stats().energy for i in range(n_seq)]
    b.close()
    plain.close()
    # the throughput baseline: the same n_seq sequences through n_seq plain FP32 contexts, each replaying its
    # frame graph on its own stream, all streams running at once
    ctxs = [sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS, sf.preset(sf.PRESET_FIG2, gn_iters=[GN], pcg_iters=[PCG]))
            for _ in range(n_seq)]
    for c in ctxs:
        c.tune_pcg(frames_d[0])  # the cached per-level schedules
    streams = [torch.cuda.Stream() for _ in range(n_seq)]
    outs = [torch.empty((6, HEIGHT // STRIDE, WIDTH // STRIDE), device=dev, dtype=torch.float32) for _ in range(n_seq)]
    seq_frames = [[frames_d[f] for f in range(steps + 1)]] + \
        [[packed[f][b_in_off[i]:b_in_off[i] + 4 * WIDTH * HEIGHT].view(4, HEIGHT, WIDTH) for f in range(steps + 1)]
         for i in range(1, n_seq)]
    main = torch.cuda.current_stream()
    ms_ms = 0.0
    for f in range(steps + 1):
        s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(main)
        for i, c in enumerate(ctxs):
            streams[i].wait_event(s0)
            with torch.cuda.stream(streams[i]):
                c.solve(seq_frames[i][f], outs[i])
        for st in streams:
            main.wait_stream(st)
        e0.record(main)
        e0.synchronize()
        if f > 0:
            ms_ms += s0.elapsed_time(e0)
    ms_energies = [c.stats().energy for c in ctxs]
    for c in ctxs:
        c.close()
    ms_fps = n_seq * steps * 1e3 / ms_ms
    res["plain_fp32_multistream"] = {
        "contexts": n_seq, "frames_per_s": ms_fps, "ms_per_frame_step": ms_ms / steps,
        "note": "one plain context per sequence, each replaying its frame graph on its own stream",
        "energy_rel_vs_batched_max": max(abs(a - bb) / abs(bb) for a, bb in zip(ms_energies, batched_energies))}
    res["vs_plain_fp32_multistream"] = res["frames_per_s"] / ms_fps
    return res


SCHWARZ_SCHEDULES = (
    # (tile, overlap, sweeps, patch iterations): the paper's shape (16 px subdomains with 2 px of boundary at its
    # stride 2 are 8x8 nodes with 1 node of overlap; 5 PCG x 5 patch iterations), and the cheapest schedule
    # measured to stay within 1e-4 of the global PCG's energy on every frame of this video
    (8, 1, 5, 5),
    (7, 1, 6, 6),
)


def variant_schwarz(dev, frames_d, pcg_energies, pcg_fps, reps=3):
    """The domain decomposition of Section 5.2 (restricted additive Schwarz over
    square subdomains, local PCG in shared memory) on the headline video: the
    level pipeline's frames/s, and every frame's final energy against the
    global PCG's (frame by frame, the same frames)."""
    import torch

    from paper_1610_07159_gb300 import sf

    _, _, nx, ny = level_sizes()[0]
    outs = torch.empty((NFRAMES, 6, ny, nx), device=dev, dtype=torch.float32)
    out1 = torch.empty((6, ny, nx), device=dev, dtype=torch.float32)
    res = []
    for tile, ov, sweeps, patch in SCHWARZ_SCHEDULES:
        kw = dict(gn_iters=[GN], pcg_iters=[sweeps], patch_iters=[patch], solver=sf.SOLVER_SCHWARZ,
                  schwarz_tile=tile, schwarz_overlap=ov)
        v = sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS, sf.preset(sf.PRESET_FIG2, video=1, **kw))
        v.solve_video(frames_d, outs)
        best = None
        for _ in range(reps):
            v.reset()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            v.solve_video(frames_d, outs)
            b.record()
            b.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        v.close()
        fr = sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS, sf.preset(sf.PRESET_FIG2, **kw))
        rel = []
        for f in range(NFRAMES):
            fr.solve(frames_d[f], out1)
            e_sw = fr.stats().energy
            rel.append((e_sw - pcg_energies[f]) / pcg_energies[f])
        fr.close()
        fps = NFRAMES * 1e3 / best
        res.append({"tile_nodes": tile, "overlap_nodes": ov, "sweeps": sweeps, "patch_iters": patch,
                    "video_fps": fps, "vs_global_pcg_fps": fps / pcg_fps,
                    "energy_rel_vs_global_pcg_max": max(rel), "energy_rel_vs_global_pcg_mean": sum(rel) / len(rel),
                    "equal_energy_1e-4": bool(max(rel) <= 1e-4)})
    return {"global_pcg_video_fps": pcg_fps, "schedules": res,
            "note": "best of a few passes of the level pipeline each; energies frame by frame from the same frames"}


def variant_pipelined_pcg(dev, frames_d, pcg_energies, pcg_fps, reps=3):
    """The pipelined PCG (SF_PCG_PIPELINED: the grid reduction behind the
    matrix-vector product, tuned per level among the schedules that include
    it) on the headline video: the level pipeline's frames/s, and every
    frame's final energy against the default's (frame by frame, the same
    frames)."""
    import torch

    from paper_1610_07159_gb300 import sf

    _, _, nx, ny = level_sizes()[0]
    outs = torch.empty((NFRAMES, 6, ny, nx), device=dev, dtype=torch.float32)
    out1 = torch.empty((6, ny, nx), device=dev, dtype=torch.float32)
    kw = dict(gn_iters=[GN], pcg_iters=[PCG], pcg_mode=sf.PCG_PIPELINED)
    v = sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS, sf.preset(sf.PRESET_FIG2, video=1, **kw))
    sched = v.tune_pcg(frames_d[0])
    v.solve_video(frames_d, outs)
    best = None
    for _ in range(reps):
        v.reset()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        v.solve_video(frames_d, outs)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    v.close()
    fr = sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS, sf.preset(sf.PRESET_FIG2, **kw))
    fr.tune_pcg(frames_d[0])
    fr.reset()
    rel = []
    for f in range(NFRAMES):
        fr.solve(frames_d[f], out1)
        rel.append((fr.stats().energy - pcg_energies[f]) / pcg_energies[f])
    fr.close()
    fps = NFRAMES * 1e3 / best
    return {"video_fps": fps, "vs_default_fps": fps / pcg_fps,
            "pcg_schedules": [{"level": l, "kind": k, "ctas": b_, "nodes_per_group": t}
                              for l, (k, b_, t) in enumerate(sched)],
            "energy_rel_vs_default_max": max(abs(r) for r in rel), "energy_rel_vs_default_mean": sum(rel) / len(rel),
            "equal_energy_1e-4": bool(max(abs(r) for r in rel) <= 1e-4),
            "note": "best of a few passes of the level pipeline; energies frame by frame from the same frames"}


STEREO_W, STEREO_H, STEREO_LEVELS = 4288, 2848, 7


def variant_stereo_12mp(dev, reps=3):
    """The paper's 12 MP stereo-only workload (Section 6): one seeded synthetic
    4288x2848 stereo pair (disparities 30-200 px) used at both times, stride 8,
    7 levels, 3 Gauss-Newton steps per level, the Figures 7/9 column of Table
    1. The level-0 grid (536 x 356 nodes) is solved by the Schwarz
    decomposition of Section 5.2 (tile 7 nodes, overlap 1, 6 sweeps x 6 patch
    iterations); the global PCG does not hold a grid that large in one launch.
    The paper reports 700 ms per pair on its 2016 GPU (context only)."""
    import numpy as np
    import torch

    from paper_1610_07159_gb300 import scenes, scenes_device, sf

    video = scenes.SceneVideo(STEREO_W, STEREO_H, 1, seed=700, disparity=(30.0, 200.0), max_motion=0.0)
    q = scenes_device.stereo_pair_quadruple(video, dev)
    p = sf.preset(sf.PRESET_FIG79, gn_iters=[GN], pcg_iters=[6], patch_iters=[6], solver=sf.SOLVER_SCHWARZ,
                  schwarz_tile=7, schwarz_overlap=1)
    s = sf.Solver(STEREO_W, STEREO_H, STRIDE, STEREO_LEVELS, p)
    out = s.solve(q)  # warm-up (captures the frame graph)
    times = []
    for _ in range(reps):
        s.reset()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        s.solve(q, out)
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    st = s.stats()
    f = out.cpu().numpy()
    s.close()
    ms = min(times)
    return {"workload": f"{STEREO_W}x{STEREO_H} stereo pair at both times, stride {STRIDE}, {STEREO_LEVELS} levels, "
                        f"{GN} GN per level, Schwarz 6 sweeps x 6 patch iterations (tile 7, overlap 1), Figures 7/9 "
                        "weights, FP32",
            "ms_per_pair": ms, "pairs_per_s": 1e3 / ms, "launches": st.launches,
            "max_abs_motion_and_difference_px": float(np.max(np.abs(f[2:]))),
            "energy": st.energy, "paper_context_ms_per_pair": 700.0}


def variant_maps(dev, frames_d, plain_fps, reps=3):
    """The headline video with the occlusion and illumination correction maps
    of Algorithm 1 computed after every level and used by the next: frames/s
    through the level pipeline, and the share of the map kernels in a frame
    (serialised, CUDA events around their launches inside the frame graph)."""
    import torch

    from paper_1610_07159_gb300 import sf

    kw = dict(gn_iters=[GN], pcg_iters=[PCG], occlusion=1, illumination=1)
    v = sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS, sf.preset(sf.PRESET_FIG2, video=1, **kw))
    v.tune_pcg(frames_d[0])
    _, _, nx, ny = level_sizes()[0]
    outs = torch.empty((NFRAMES, 6, ny, nx), device=dev, dtype=torch.float32)
    v.solve_video(frames_d, outs)
    best = None
    for _ in range(reps):
        v.reset()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        v.solve_video(frames_d, outs)
        b.record()
        b.synchronize()
        best = a.elapsed_time(b) if best is None else min(best, a.elapsed_time(b))
    st = v.stats()
    v.close()
    fps = NFRAMES * 1e3 / best
    return {"video_fps": fps, "vs_plain_video_fps": fps / plain_fps, "launches_per_frame": st.launches,
            "energy_last_frame": st.energy,
            "note": "occlusion maps (z-buffered warp grid, visibility, prolongation) and illumination maps (stereo "
                    "residual, Gaussian sigma 3.2 px, box prolongation) after levels 3, 2, 1"}


HR_W, HR_H, HR_STRIDE, HR_LEVELS, HR_FRAMES = 1920, 1080, 16, 6, 20
PREC_NAMES = (("fp32", 0), ("fp16", 2), ("bf16", 1))  # sf.FP32, sf.MIXED_FP16, sf.MIXED_BF16


def variant_high_resolution(dev, reps=2):
    """The 1920x1080 video (20 frames, disparities up to 96 px, motion up to
    40 px; stride 16, 6 levels, 3 GN x 20 PCG, the Figures 5/6/8 weights) in
    FP32, FP16 and BF16 texels through the level pipeline: frames/s and the
    last frame's energy. Also keeps, per precision, frame 0's fields and the
    integer decisions of its solve (W masks; the cell decisions in FP32), for
    the per-field comparison with the FP64 oracle in the CPU leg."""
    import torch

    from paper_1610_07159_gb300 import scenes, scenes_device, sf

    video = scenes.SceneVideo(HR_W, HR_H, HR_FRAMES, seed=300, disparity=(15.0, 96.0), max_motion=40.0)
    frames = scenes_device.frames(video, HR_FRAMES, dev, dtype=torch.float32)
    nx, ny = -(-HR_W // HR_STRIDE), -(-HR_H // HR_STRIDE)
    outs = torch.empty((HR_FRAMES, 6, ny, nx), device=dev, dtype=torch.float32)
    res, keep = {}, {}
    for name, prec in PREC_NAMES:
        kw = dict(gn_iters=[GN], pcg_iters=[PCG], precision=prec)
        v = sf.Solver(HR_W, HR_H, HR_STRIDE, HR_LEVELS, sf.preset(sf.PRESET_FIG568, video=1, **kw))
        v.tune_pcg(frames[0])
        v.solve_video(frames, outs)
        best = None
        for _ in range(reps):
            v.reset()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            v.solve_video(frames, outs)
            b.record()
            b.synchronize()
            best = a.elapsed_time(b) if best is None else min(best, a.elapsed_time(b))
        res[name] = {"fps": HR_FRAMES * 1e3 / best, "energy_last_frame": v.stats().energy}
        v.close()
        one = sf.Solver(HR_W, HR_H, HR_STRIDE, HR_LEVELS,
                        sf.preset(sf.PRESET_FIG568, record_cells=1 if prec == 0 else 0, **kw))
        f0 = one.solve(frames[0]).cpu().numpy()
        keep[name] = {"fields": f0, "energy": one.stats().energy, "W": one.wmasks(),
                      "cells": one.cell_records() if prec == 0 else None}
        one.close()
    for name in ("fp16", "bf16"):
        res[name]["energy_rel_vs_fp32"] = (res[name]["energy_last_frame"] - res["fp32"]["energy_last_frame"]) / \
            res["fp32"]["energy_last_frame"]
        res[name]["vs_fp32_fps"] = res[name]["fps"] / res["fp32"]["fps"]
    res["workload"] = (f"{HR_W}x{HR_H} synthetic stereo video, {HR_FRAMES} frames, disparities up to 96 px, motion up "
                       f"to 40 px, stride {HR_STRIDE}, {HR_LEVELS} levels, {GN} GN x {PCG} PCG, Figures 5/6/8 weights")
    return res, {"frame0": frames[0].cpu().numpy(), "runs": keep}


def webcam_frame0_runs(frames_d):
    """Frame 0 of the headline video in the three texel precisions: fields and
    the integer decisions of the solve, for the per-field oracle comparison."""
    from paper_1610_07159_gb300 import sf

    keep = {}
    for name, prec in PREC_NAMES:
        one = sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS,
                        sf.preset(sf.PRESET_FIG2, gn_iters=[GN], pcg_iters=[PCG], precision=prec,
                                  record_cells=1 if prec == 0 else 0))
        f0 = one.solve(frames_d[0]).cpu().numpy()
        keep[name] = {"fields": f0, "energy": one.stats().energy, "W": one.wmasks(),
                      "cells": one.cell_records() if prec == 0 else None}
        one.close()
    return {"frame0": frames_d[0].cpu().numpy(), "runs": keep}


def per_field_errors(saved, w, h, stride, levels, preset):
    """CPU leg: every output field of the GPU's frame 0 against the FP64
    oracle solving the same quadruple with the GPU's W masks replayed (and its
    cell decisions at cell edges in FP32): max-abs px per field, energy."""
    import numpy as np

    import oracle as O

    names = ("s_x", "s_y", "m_x", "m_y", "d_x", "d_y")
    p = O.Params.preset(preset, gn_iters=(GN,) * 8, pcg_iters=(PCG,) * 8)
    q = saved["frame0"].astype(np.float64)
    out = {}
    for name, run in saved["runs"].items():
        ref = O.solve_frame(q, stride, levels, p, W_given=run["W"], cells_given=run["cells"])
        err = np.max(np.abs(run["fields"] - ref.fields(0)), axis=(1, 2))
        out[name] = {**{n: float(e) for n, e in zip(names, err)},
                     "energy_rel": abs(run["energy"] - ref.energy) / abs(ref.energy),
                     "replayed": "W and cell decisions" if run["cells"] is not None else "W"}
    return out


def variant_mixed(dev, frames_d):
    """The headline video in the 16-bit texel modes, with the final energy of
    the last frame against FP32."""
    import torch

    from paper_1610_07159_gb300 import sf

    out = {}
    for name, prec in (("fp32", sf.FP32), ("fp16", sf.MIXED_FP16), ("bf16", sf.MIXED_BF16)):
        s = sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS,
                      sf.preset(sf.PRESET_FIG2, gn_iters=[GN], pcg_iters=[PCG], video=1, precision=prec))
        outs = torch.empty((NFRAMES, 6, HEIGHT // STRIDE, WIDTH // STRIDE), device=dev, dtype=torch.float32)
        s.solve_video(frames_d, outs)
        s.reset()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        s.solve_video(frames_d, outs)
        b.record()
        b.synchronize()
        out[name] = {"fps": NFRAMES * 1e3 / a.elapsed_time(b), "energy_last_frame": s.stats().energy}
        s.close()
    for name in ("fp16", "bf16"):
        out[name]["energy_rel_vs_fp32"] = (out[name]["energy_last_frame"] - out["fp32"]["energy_last_frame"]) / \
            out["fp32"]["energy_last_frame"]
    return out


def variant_warm_start(dev, n_videos=8):
    """First frames at 640x480: the zero start with the full schedule against
    the learned warm start with the cheapest schedule whose mean final energy
    is within 1% of it (the 1e-4 acceptance is reported per schedule)."""
    import numpy as np
    import torch

    from paper_1610_07159_gb300 import scenes, scenes_device, sf, warmstart as ws

    d = np.load(os.path.join(ROOT, "paper_1610_07159_gb300", "data", "warmstart_640x480.npz"))
    net = sf.Net(1)
    net.set_params(torch.from_numpy(d["params"]).to(dev))
    ev = ws.evaluate(net, n_videos, seed0=980000, schedules=ws.SCHEDULES)
    ok = [r for r in ev["schedules"] if r["warm_mean_rel"] <= 0.01]
    pick = min(ok, key=lambda r: r["cost"]) if ok else None
    quads = [scenes_device.frames(scenes.SceneVideo(WIDTH, HEIGHT, 1, seed=980000 + v), 1, dev)[0]
             for v in range(n_videos)]

    def fps(gn, warm):
        """First-frame rate: every frame from a reset state, each timed alone
        (the warm start's pyramid and network pass inside the timed region)."""
        s = sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS, ws.solver_params(gn))
        tot = 0.0
        for rep in range(2):
            for q in quads:
                s.reset()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                if warm:
                    net.warm_start(s, q)
                s.solve(q)
                b.record()
                b.synchronize()
                if rep:
                    tot += a.elapsed_time(b)
        s.close()
        return len(quads) * 1e3 / tot

    tte = ws.evaluate_time_to_energy(net, 32, seed0=970000)
    res = {"frames": n_videos, "cold_schedule": list(ws.FULL), "cold_first_frame_fps": fps(ws.FULL, False),
           "time_to_cold_energy_1e-4": {k: tte[k] for k in ("frames", "bar", "cold_full_cost", "warm_accepted")},
           "accepted_at_1e-4": ev["cheapest_warm"],
           "per_schedule": [{k: r[k] for k in ("gn", "cost", "warm_mean_rel", "warm_max_rel", "cold_mean_rel",
                                                "cold_max_rel", "warm_accepted")} for r in ev["schedules"]]}
    for start, r in tte["starts"].items():
        res["time_to_cold_energy_1e-4"][start] = {k: r[k] for k in ("reached", "mean_cost", "frames_per_s_to_reach")}
    if pick:
        res.update({"warm_schedule": pick["gn"], "warm_first_frame_fps": fps(pick["gn"], True),
                    "warm_mean_rel_energy": pick["warm_mean_rel"], "warm_max_rel_energy": pick["warm_max_rel"]})
    return res


def run_ours(args):
    import numpy as np
    import torch

    from paper_1610_07159_gb300 import scenes, sf

    dist, rank, world, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.arm == "batch8":
        # profiling aid: 8 sequences of 640x480 in one launch per frame step, two frame steps
        from paper_1610_07159_gb300 import scenes_device
        b = sf.Batch([(WIDTH, HEIGHT)] * 8, [LEVELS] * 8, STRIDE,
                     sf.preset(sf.PRESET_FIG2, gn_iters=[GN], pcg_iters=[PCG]))
        b.set_schedule(8, 1)
        v = [scenes_device.frames(scenes.SceneVideo(WIDTH, HEIGHT, 2, seed=5000 + i), 2, dev, dtype=torch.float32)
             for i in range(8)]
        o = torch.empty(b.out_total, device=dev, dtype=torch.float32)
        for f in range(2):
            b.solve(b.pack([x[f] for x in v]), o)
        torch.cuda.synchronize()
        print(json.dumps({"arm": "batch8", "energy": b.sequence(0).stats().energy}), flush=True)
        return
    if args.arm == "train":
        # profiling aid: two training steps of the warm-start network, batch 256
        from paper_1610_07159_gb300 import warmstart as ws
        net = sf.Net(256)
        net.set_params(ws.init_params(1))
        g = torch.Generator(device=dev)
        g.manual_seed(7)
        x = torch.rand(256, 4, 60, 80, device=dev, generator=g)
        y = 0.2 * torch.randn(256, 6, 8, 10, device=dev, generator=g)
        for _ in range(2):
            net.train_step(x, y, 1e-3)
        net.status()
        print(json.dumps({"arm": "train"}), flush=True)
        return
    video = scenes.SceneVideo(WIDTH, HEIGHT, NFRAMES, seed=100 + rank).frames()
    frames_d = torch.from_numpy(video).to(dev)  # all frames resident in HBM (147 MB)
    flush = torch.empty(64 * 1024 * 1024, device=dev, dtype=torch.float32)  # 256 MB > L2
    stream = torch.cuda.current_stream(dev)
    prof = (1 << sf.K_PCG) | (1 << sf.K_ASSEMBLE)

    if args.arm in ("frames", "frames_maps", "frames_schwarz"):
        # profiling aid: the frame-by-frame graph path only, W + K frames in level order (with both maps, or with
        # the Schwarz solver of the equal-energy schedule)
        extra = {}
        if args.arm == "frames_maps":
            extra = dict(occlusion=1, illumination=1)
        elif args.arm == "frames_schwarz":
            extra = dict(solver=sf.SOLVER_SCHWARZ, pcg_iters=[6], patch_iters=[6], schwarz_tile=7, schwarz_overlap=1)
        plain = sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS,
                          sf.preset(sf.PRESET_FIG2, **{**dict(gn_iters=[GN], pcg_iters=[PCG]), **extra}))
        out1 = torch.empty((6, 60, 80), device=dev, dtype=torch.float32)
        if args.tune_pcg:
            plain.tune_pcg(frames_d[0])  # the headline's per-level PCG schedules
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("frames")  # ncu --nvtx --nvtx-include "frames/" skips the set-up launches
        for k in range(args.warmup + args.steps):
            plain.solve(frames_d[k % NFRAMES], out1)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"arm": args.arm, "frames": args.warmup + args.steps, "tuned_pcg": args.tune_pcg}), flush=True)
        return

    # headline: the level-pipelined video solve, one step = one pass over the 30 frames. A second
    # context runs the same steps with per-kernel CUDA events recorded inside the pipeline, for the
    # kernel times and the roofline, so that the headline steps carry no instrumentation.
    solver = sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS,
                       sf.preset(sf.PRESET_FIG2, gn_iters=[GN], pcg_iters=[PCG], video=1))
    profiled = sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS,
                         sf.preset(sf.PRESET_FIG2, gn_iters=[GN], pcg_iters=[PCG], profile_mask=prof, video=1))
    # set-up, outside the timed region: the PCG schedule of every level, picked by timing
    pcg_schedules = solver.tune_pcg(frames_d[0])
    profiled.tune_pcg(frames_d[0])  # the same schedules, from the per-process cache
    _, _, nx, ny = solver.dims(0)
    outs = torch.empty((NFRAMES, 6, ny, nx), device=dev, dtype=torch.float32)
    acc = {"ms": 0.0, "prof_ms": 0.0, sf.K_PCG: [0.0, 0], sf.K_ASSEMBLE: [0.0, 0]}

    def vstep(ctx, timed):
        ctx.reset()
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        ctx.solve_video(frames_d, outs)
        e.record(stream)
        e.synchronize()
        if timed and ctx is solver:
            acc["ms"] += s.elapsed_time(e)
        elif timed:
            acc["prof_ms"] += s.elapsed_time(e)
            for kc in (sf.K_PCG, sf.K_ASSEMBLE):
                ms, n = ctx.kernel_times(kc)
                acc[kc][0] += ms
                acc[kc][1] += n

    for _ in range(args.warmup):
        vstep(solver, False)
        vstep(profiled, False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        vstep(solver, True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    st = solver.stats()
    frames_timed = args.steps * NFRAMES
    t_max = max_over_ranks(dist, acc["ms"], dev)
    value = aggregate_rate(world, frames_timed, t_max)
    video_out = outs.clone()
    # the profiled pass: the same K steps, per-kernel events inside the pipeline
    for _ in range(args.steps):
        vstep(profiled, True)
    torch.cuda.synchronize()
    clk = clocks.stop()
    profiled_fps = frames_timed / (acc["prof_ms"] / 1e3)

    if args.arm == "video":
        if rank == 0:
            print(json.dumps({"arm": "video", "value": value, "unit": UNIT}), flush=True)
        return

    # plain FP32 frame by frame (one captured graph per frame), for comparison
    plain = sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS, sf.preset(sf.PRESET_FIG2, gn_iters=[GN], pcg_iters=[PCG]))
    plain.tune_pcg(frames_d[0])  # the tuned schedules, from the per-process cache
    out1 = torch.empty((6, ny, nx), device=dev, dtype=torch.float32)
    passes = max(1, args.steps // 4)
    plain_ms, same = 0.0, True
    plain_energies = []
    for p_ in range(1 + passes):
        plain.reset()
        for f in range(NFRAMES):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            plain.solve(frames_d[f], out1)
            e.record(stream)
            e.synchronize()
            if p_ > 0:
                plain_ms += s.elapsed_time(e)
            else:
                same = same and torch.equal(out1, video_out[f])
                plain_energies.append(plain.stats().energy)
    plain_fps = passes * NFRAMES / (plain_ms / 1e3)

    # end to end through the host entry point: pinned video in, fields out, inside the timed region
    host_frames = torch.from_numpy(video).pin_memory()
    host_outs = torch.empty((NFRAMES, 6, ny, nx), dtype=torch.float32).pin_memory()
    solver_e2e = sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS,
                           sf.preset(sf.PRESET_FIG2, gn_iters=[GN], pcg_iters=[PCG], video=1))
    solver_e2e.tune_pcg(frames_d[0])
    for _ in range(args.warmup):
        solver_e2e.reset()
        solver_e2e.solve_video_host(host_frames, host_outs)
    e2e_ms = 0.0
    for _ in range(args.steps):
        solver_e2e.reset()
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        solver_e2e.solve_video_host(host_frames, host_outs)
        e.record(stream)
        e.synchronize()
        e2e_ms += s.elapsed_time(e)
    e2e_max = max_over_ranks(dist, e2e_ms, dev)
    e2e_value = aggregate_rate(world, frames_timed, e2e_max)

    # serialised pass for the roofline: the same frames, frame by frame on one stream (one captured graph
    # per frame), with CUDA events recorded around every launch of the PCG and assembly classes inside the
    # graph, so that no other kernel runs beside a timed one; L2 flushed before every frame
    ser_classes = (sf.K_PCG, sf.K_ASSEMBLE, sf.K_GATHER, sf.K_ENERGY)
    serial = sf.Solver(WIDTH, HEIGHT, STRIDE, LEVELS,
                       sf.preset(sf.PRESET_FIG2, gn_iters=[GN], pcg_iters=[PCG],
                                 profile_mask=sum(1 << k for k in ser_classes)))
    serial.tune_pcg(frames_d[0])
    ser = {k: [0.0, 0] for k in ser_classes}
    ser_frame_ms, ser_worst_frac = 0.0, 0.0
    for p_ in range(2):  # a warm pass, then the measured one
        serial.reset()
        for f in range(NFRAMES):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            serial.solve(frames_d[f], out1)
            e.record(stream)
            e.synchronize()
            if p_:
                fms = s.elapsed_time(e)
                ser_frame_ms += fms
                cls = 0.0
                for kc in ser_classes:
                    ms, n = serial.kernel_times(kc)
                    ser[kc][0] += ms
                    ser[kc][1] += n
                    cls += ms
                ser_worst_frac = max(ser_worst_frac, cls / fms)

    # roofline of the dominant kernel class, from the serialised pass
    peaks, peak_src = measured_peaks()
    fma_flops = sf.fma_rate()
    alu_peak_tflops = fma_flops / 1e12
    pcg_ms, pcg_n = ser[sf.K_PCG]
    asm_ms, asm_n = ser[sf.K_ASSEMBLE]
    pcg_s, asm_s = pcg_ms / 1e3, asm_ms / 1e3
    pcg_model_bytes = pcg_bytes_per_frame("per_node_860") * NFRAMES
    pcg_kern = PCG_KERNEL.get(pcg_schedules[0][0], "k_pcg1")
    own_model = {"k_pcg1p": "pipelined", "k_pcg1h": "staged"}.get(pcg_kern, "one_reduction")
    pcg_kernel_bytes = pcg_bytes_per_frame(own_model) * NFRAMES
    asm_flops = asm_flops_per_frame() * NFRAMES
    hbm_peak = float(peaks["hbm_gbs"])
    kernels = {
        "pcg": {"launches": pcg_n, "ms_total": pcg_ms, "us_per_launch": 1e3 * pcg_ms / max(pcg_n, 1),
                "bytes_per_launch_model_860B": pcg_model_bytes / max(pcg_n, 1),
                "bytes_per_launch_kernel_count": pcg_kernel_bytes / max(pcg_n, 1),
                "kernel_count_model": own_model,
                "GBps_model_860B": pcg_model_bytes / pcg_s / 1e9 if pcg_ms else None,
                "GBps_kernel_count": pcg_kernel_bytes / pcg_s / 1e9 if pcg_ms else None},
        "assemble": {"launches": asm_n, "ms_total": asm_ms, "us_per_launch": 1e3 * asm_ms / max(asm_n, 1),
                     "flops_per_launch": asm_flops / max(asm_n, 1),
                     "TFLOPs": asm_flops / asm_s / 1e12 if asm_ms else None,
                     "frac_of_measured_fp32_fma": asm_flops / asm_s / fma_flops if asm_ms else None},
        "gather": {"launches": ser[sf.K_GATHER][1], "ms_total": ser[sf.K_GATHER][0],
                   "us_per_launch": 1e3 * ser[sf.K_GATHER][0] / max(ser[sf.K_GATHER][1], 1),
                   "note": "k_gather (node blocks, right-hand side, preconditioner and energy in one launch)"},
        "trials": {"launches": ser[sf.K_ENERGY][1], "ms_total": ser[sf.K_ENERGY][0],
                   "us_per_launch": 1e3 * ser[sf.K_ENERGY][0] / max(ser[sf.K_ENERGY][1], 1)},
        "pipelined_pass": {"note": "the same classes inside the level pipeline, where launches of different "
                                   "levels overlap, so these event times include shared time",
                           "pcg_ms_per_step": acc[sf.K_PCG][0] / args.steps,
                           "assemble_ms_per_step": acc[sf.K_ASSEMBLE][0] / args.steps},
    }
    all_cls_ms = sum(v[0] for v in ser.values())
    self_check = {"frames": NFRAMES, "frame_ms_total": ser_frame_ms, "class_ms_total": all_cls_ms,
                  "classes": "PCG, assembly, gather, trials",
                  "largest_frame_share_of_the_classes": ser_worst_frac,
                  "ok": bool(all_cls_ms <= ser_frame_ms and ser_worst_frac <= 1.0)}
    if pcg_ms >= asm_ms:
        ach = kernels["pcg"]["GBps_model_860B"]
        roof = {"kernel": pcg_kern, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak if ach else None, "traffic": recorded_traffic(pcg_kern),
                "bytes_model": "860 B per node and PCG iteration (168 floats of stencil blocks + 8 vectors)",
                "kernel_count": {"model": own_model,
                                 "achieved": kernels["pcg"]["GBps_kernel_count"],
                                 "frac": kernels["pcg"]["GBps_kernel_count"] / hbm_peak if pcg_ms else None},
                "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json)"}
    else:
        ach = kernels["assemble"]["TFLOPs"]
        roof = {"kernel": "k_assemble", "bound": "alu", "achieved": ach, "peak": alu_peak_tflops, "unit": "TFLOP/s",
                "frac": ach / alu_peak_tflops if ach else None, "traffic": recorded_traffic("k_assemble"),
                "peak_source": "FP32 FMA rate measured in this run (sf_probe_fma_rate)"}
    roof["timing"] = ("CUDA events around every launch of the class inside the frame graph, over one serialised "
                      f"pass of the {NFRAMES} frames on one stream (no other kernel runs beside a timed one; "
                      "L2 flushed before every frame)")
    roof["self_check"] = self_check
    roof["fp32_fma_peak_tflops_measured"] = alu_peak_tflops

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ray-cast stereo video; the paper's webcam and Volker data are not available)",
        "config": {"workload": WORKLOAD, "step": f"one pass over the {NFRAMES}-frame video (sf_solve_video)",
                   "global_batch": world, "seq_len": NFRAMES,
                   "parallelism": f"replicas x{world} (independent sequences); levels of consecutive frames pipelined",
                   "l2": "flushed between steps (256 MB write outside the timed events)"},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": NFRAMES * 4 * WIDTH * HEIGHT * 4,
                "d2h_bytes_per_step": NFRAMES * 6 * nx * ny * 4},
        "gpu_launches": st.launches * frames_timed,
        "clocks": clk,
        "variants": {"frame_by_frame_graph_fps": plain_fps, "video_pipeline_fps": value,
                     "video_pipeline_profiled_fps": profiled_fps,
                     "pcg_schedules": [{"level": l, "kind": k, "ctas": b, "nodes_per_group": t}
                                       for l, (k, b, t) in enumerate(pcg_schedules)],
                     "fields_identical": bool(same),
                     "note": "same FP32 kernels; the pipeline overlaps the levels of consecutive frames"},
        "energy_last_frame": st.energy,
        "kernels": kernels,
    }
    if rank == 0 and not args.no_variants:
        line["variants"]["schwarz_640x480"] = variant_schwarz(dev, frames_d, plain_energies, value)
        line["variants"]["pipelined_pcg_640x480"] = variant_pipelined_pcg(dev, frames_d, plain_energies, value)
        line["variants"]["stereo_only_4288x2848"] = variant_stereo_12mp(dev)
        line["variants"]["occlusion_and_illumination_maps"] = variant_maps(dev, frames_d, value)
        line["variants"]["batched_640x480"] = variant_batched_640(dev, frames_d)
        line["variants"]["batched_640x480"]["vs_plain_fp32_video"] = \
            line["variants"]["batched_640x480"]["frames_per_s"] / value
        line["variants"]["batched_64_uneven"] = variant_batched(dev)
        line["variants"]["mixed_precision"] = variant_mixed(dev, frames_d)
        hr, hr_saved = variant_high_resolution(dev)
        line["variants"]["mixed_precision_1920x1080"] = hr
        webcam_saved = webcam_frame0_runs(frames_d)
        line["variants"]["learned_warm_start"] = variant_warm_start(dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(video)
        if not args.no_variants:
            line["variants"]["cpu_oracle_all_cores"] = cpu_baseline_all_cores()
            # every output field against the FP64 oracle (the oracle runs in this CPU leg only)
            line["variants"]["per_field_error_vs_fp64_oracle"] = {
                "note": "frame 0; max-abs px per field on the finest level; the oracle replays the GPU's W masks (and "
                        "its cell decisions at cell edges in FP32), integer decisions taken in floating point",
                f"{WIDTH}x{HEIGHT}": per_field_errors(webcam_saved, WIDTH, HEIGHT, STRIDE, LEVELS, "fig2"),
                f"{HR_W}x{HR_H}": per_field_errors(hr_saved, HR_W, HR_H, HR_STRIDE, HR_LEVELS, "fig568")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args):
    """The FP64 CPU oracle as the reference arm, on the headline workload itself:
    each step solves the next whole 640x480 frame of the same video from the
    previous frame's state (the temporal chain), single-threaded."""
    import numpy as np

    import oracle as O
    from paper_1610_07159_gb300 import scenes

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.warmup + args.steps
    video = scenes.SceneVideo(WIDTH, HEIGHT, NFRAMES, seed=100).frames(min(n, NFRAMES))
    p = O.Params.preset("fig2", gn_iters=(GN,) * 8, pcg_iters=(PCG,) * 8)
    prev = None
    for k in range(args.warmup):
        prev = O.solve_frame(video[k % NFRAMES].astype(np.float64), STRIDE, LEVELS, p, prev=prev)
    t0 = time.perf_counter()
    for k in range(args.warmup, n):
        prev = O.solve_frame(video[k % NFRAMES].astype(np.float64), STRIDE, LEVELS, p, prev=prev)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    sample = (f"frames {args.warmup + 1}-{n} of the same {WIDTH}x{HEIGHT} video (frames 1-{args.warmup} as warm-up), "
              "each from the previous frame's state, with the single-threaded FP64 C oracle on one host core; "
              "frames/s = timed frames / time")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded ray-cast stereo video)",
        "config": {"workload": WORKLOAD, "step": "one frame of the video (temporal chain)", "global_batch": 1,
                   "seq_len": NFRAMES, "parallelism": "single host core"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the batched, mixed and warm-start variants")
    ap.add_argument("--tune-pcg", action="store_true",
                    help="frames arms: pick the per-level PCG schedules by timing first, as the headline does")
    ap.add_argument("--arm", choices=("all", "video", "frames", "frames_maps", "frames_schwarz", "batch8", "train"),
                    default="all",
                    help="for profiling runs: only the pipelined video arm, only the frame-by-frame arm (plain, with "
                         "both maps, or with the Schwarz solver), one 8-sequence batched launch pair, or two training "
                         "steps of the warm-start network")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
