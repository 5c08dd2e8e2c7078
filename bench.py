"""Benchmark of the GB300 tile rasterizer (forward render, Speedy-Splat localization).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the 3M-Gaussian outdoor-like scene at 1280x840 (blob mixture plus
background shell, seed 0), tile 16.  One step is one full forward frame:
preprocess -> intersect (scan + emit) -> radix sort -> tile ranges -> blend.
``value`` is AccuTile frames/s with the scene resident in HBM (CUDA events on
the rendering stream, W warm-up frames, then exactly K timed frames bracketed
by barrier + synchronize, max over ranks).  The scene (708 MB) is larger than
L2 (129 MB), so no L2 flush is inserted between frames.  The 3-sigma and
SnugBox modes of the same library are timed the same way for the comparison.

Multi-GPU (torchrun, N ranks): every rank renders its own frames of a full
replica of the scene (the path does not shard a frame); value = frames of all
ranks / max elapsed.

``--impl reference`` times the CPU oracle (FP32, the documented operation
order, built with OpenMP over its independent loops, all host cores) on the
same workload; each step renders the frame, or one horizontal band of it when
a frame is slow, through the whole oracle pipeline, so the run stays within
minutes; value = 1 / (bands x mean band time).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ms/frame & FPS, AccuTile vs 3-sigma box on 1 GB300; served p50/p99 ms"
WORKLOAD = "outdoor-3M-1280x840"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=3_000_000)
    p.add_argument("--width", type=int, default=1280)
    p.add_argument("--height", type=int, default=840)
    p.add_argument("--tile", type=int, default=16)
    p.add_argument("--modes", default="accutile,snugbox,3sigma,tbc,pixel",
                   help="modes to time; the first is the headline (profiling runs pass one mode)")
    p.add_argument("--stage-steps", type=int, default=10, help="frames per mode for the per-stage breakdown (0: skip)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-multiview", action="store_true")
    p.add_argument("--mv-cams", type=int, default=64)
    p.add_argument("--mv-n", type=int, default=1_500_000)
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-backward", action="store_true")
    p.add_argument("--no-configs", action="store_true", help="skip the 16k-box and 300k-prune mode tables")
    p.add_argument("--no-pruning", action="store_true", help="skip the Soft/Hard pruning and PUP-score experiments")
    p.add_argument("--prune-scale", type=float, default=0.1, help="pruning schedule length relative to 30k iterations")
    p.add_argument("--serve-duration", type=float, default=10.0, help="seconds of arrivals per rate")
    p.add_argument("--serve-rates", default="200,500,1000,2000")
    a = p.parse_args()
    a.steps = max(a.steps, 1)
    a.warmup = max(a.warmup, 0)
    return a


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """Samples SM clock / power / throttle reasons with nvidia-smi every 50 ms."""

    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile

            fd, self.path = tempfile.mkstemp(prefix="gs_clocks_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            if self.path:
                try:
                    self.fh.close()
                    os.remove(self.path)
                except Exception:
                    pass

    def count(self) -> int:
        try:
            self.fh.flush()
            with open(self.path) as f:
                return sum(1 for _ in f)
        except Exception:
            return 0

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 10:
                    continue
                rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if self.bus_id:
            mine = [r for r in rows if r[1].lower().endswith(self.bus_id[-12:])]
            rows = mine or rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        idx = rows[0][0]
        rows = [r for r in rows if r[0] == idx]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[2]) for r in rows if num(r[2]) is not None]
        smax = max((num(r[3]) or 0.0) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower().startswith("active")})
        loaded = [s for s in sm if s >= 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max((num(r[4]) or 0.0) for r in rows)}


# ---------------------------------------------------------------- helpers
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured", "sm_max_mhz": float(d.get("sm_max_mhz", 2070))}
    except Exception:
        return {"hbm_gbs": 6800.0, "src": "fallback", "sm_max_mhz": 2070.0}


def blend_source_digest():
    """sha256 over what determines the blend kernel's memory traffic: the
    shared headers it includes, the kernel template itself and its launcher
    (render.cu's other kernels are not part of it)."""
    import hashlib

    csrc = os.path.join(ROOT, "paper_2412_00578_gb300", "csrc")
    h = hashlib.sha256()
    for name in ("blend_common.cuh", "gs_common.cuh"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    with open(os.path.join(csrc, "render.cu")) as f:
        r = f.read()
    a = r.index("struct BlendArgs {")
    h.update(r[a:r.index("};", a)].encode())
    a = r.index("template <int T, bool kStats, bool kMulti>")
    h.update(r[a:r.index("}  // namespace", a)].encode())
    h.update(r[r.index("gs_status launch_render("):].encode())
    return h.hexdigest()


def blend_traffic(keys):
    """DRAM bytes of one blend launch, from the ncu counters in
    profiles/dram_traffic.json scaled per key, or None if the blend's sources
    changed since those counters were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            rec = json.load(f)["blend_kernel"]
        if blend_source_digest() != rec["source_sha256"]:
            return None
        return rec["bytes_per_key"] * keys
    except Exception:
        return None


def workload(args):
    from paper_2412_00578_gb300 import synth

    scene, cam = synth.outdoor_workload(n=args.n, width=args.width, height=args.height)
    return scene, cam


def make_max_reduce(dist, device):
    """max over ranks of a float (identity without torch.distributed)."""
    import torch

    def red(x: float) -> float:
        if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
            return x
        t = torch.tensor([x], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    return red


def replica_rate(frames_per_rank: int, elapsed_ms_local: float, world: int, max_reduce):
    """Whole-job frames/s of N replicas: all ranks' frames over the slowest
    rank's elapsed time.  Returns (frames/s, ms per frame of one replica)."""
    ms = max_reduce(elapsed_ms_local)
    return world * frames_per_rank * 1e3 / ms, ms / frames_per_rank


def emit(obj):
    print(json.dumps(obj), flush=True)


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2412_00578_gb300 import synth

    oracle.build(omp=True)
    cores = os.cpu_count() or 1
    scene, cam = workload(args)
    H = cam.height

    def band_cam(y0, h):
        return synth.Camera(cam.width, h, cam.fx, cam.fy, cam.cx, cam.cy - y0, cam.tan_fovx, cam.tan_fovy,
                            cam.viewmat, cam.campos, cam.near_z)

    # first warm-up step: one full frame, which also sizes the band count so the
    # whole run stays within about 150 s
    t0 = time.perf_counter()
    oracle.render(scene, cam, args.tile, 2, prec64=False, omp=True)
    t_full = time.perf_counter() - t0
    extra_warmup = max(args.warmup - 1, 0)  # the full frame above counts as the first warm-up step
    steps = args.steps
    remaining = max(steps + extra_warmup, 1)
    bands = max(1, min(16, math.ceil(remaining * t_full / 150.0)))
    bh = math.ceil(H / bands)
    times = []
    for s in range(extra_warmup + steps):
        b = s % bands
        y0 = b * bh
        c = band_cam(y0, min(bh, H - y0))
        t0 = time.perf_counter()
        oracle.render(scene, c, args.tile, 2, prec64=False, omp=True)
        dt = time.perf_counter() - t0
        if s >= extra_warmup:
            times.append(dt)
    mean_band = sum(times) / len(times)
    fps = 1.0 / (bands * mean_band)
    sample = (f"CPU oracle (FP32, OpenMP over Gaussians and pixel rows, {cores} host threads), AccuTile, "
              f"{args.n} Gaussians; each step renders one of {bands} horizontal band(s) ({cam.width}x{bh}) of the "
              f"{cam.width}x{H} frame through the whole pipeline (every Gaussian preprocessed per band); first full "
              f"frame took {t_full:.2f} s")
    emit({"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": args.gpus,
          "steps": steps, "warmup": args.warmup, "ms_per_step": mean_band * 1e3,
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
          "config": config_dict(args, cam),
          "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle", "sample": sample},
          "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


# ---------------------------------------------------------------- our arm
def config_dict(args, cam):
    """The workload description both arms print (identical by construction)."""
    return {"workload": WORKLOAD, "gaussians": args.n, "width": cam.width, "height": cam.height, "tile": args.tile,
            "mode": "accutile", "l2": "inputs exceed L2 (708 MB scene), no flush",
            "parallelism": f"replicas x{args.gpus}"}


class ModeTimer:
    """Frames of one scene and camera in every tile mode, timed with CUDA
    events on the context's stream (forward, per stage, CUDA-graph replay)."""

    STAGES = ["preprocess", "intersect", "sort", "tile_ranges", "render"]

    def __init__(self, raster, renderer, scene, cam, tile, modes, barrier, max_over_ranks, world):
        self.raster, self.renderer, self.rast = raster, renderer, renderer.rast
        self.scene, self.cam, self.tile = scene, cam, tile
        self.barrier, self.max_over_ranks, self.world = barrier, max_over_ranks, world
        self.frames, self.keys = {}, {}
        for m in modes:  # size each mode's frame (one synchronising render)
            out = renderer.render(scene, cam, m, tile)
            self.keys[m] = out.num_keys
            self.frames[m] = out.frame

    def cfg(self, mode):
        return self.raster.cfg_struct(self.tile, mode)

    def check(self, mode):
        K, flags = self.rast.gs_read_status(self.frames[mode], raise_on_error=False)
        if flags:
            raise RuntimeError(f"device status flags {flags} ({mode})")

    def timed(self, mode, steps, warmup, sampler=None):
        import torch

        rast, cfg, f = self.rast, self.cfg(mode), self.frames[mode]
        for _ in range(warmup):
            rast.gs_forward(self.scene, self.cam, cfg, f)
        self.barrier()
        if sampler:
            sampler.start()
        l0 = rast.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(rast.stream)
        for _ in range(steps):
            rast.gs_forward(self.scene, self.cam, cfg, f)
        e1.record(rast.stream)
        launches = rast.launch_count() - l0  # kernels of the timed frames only
        self.barrier()
        if sampler:  # keep the same load running (untimed) until the sampler has >= 5 samples
            t_end = time.time() + 2.0
            while sampler.count() < 5 and time.time() < t_end:
                for _ in range(20):
                    rast.gs_forward(self.scene, self.cam, cfg, f)
                torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        _, ms = replica_rate(steps, e0.elapsed_time(e1), self.world, self.max_over_ranks)
        self.check(mode)
        return ms, launches, clocks

    def stages(self, mode, steps):
        import torch

        rast, cfg, f, scene, cam = self.rast, self.cfg(mode), self.frames[mode], self.scene, self.cam
        calls = [lambda: rast.gs_preprocess(scene, cam, cfg, f), lambda: rast.gs_intersect(cam, cfg, f),
                 lambda: rast.gs_sort(cam, cfg, f), lambda: rast.gs_tile_ranges(cam, cfg, f),
                 lambda: rast.gs_render(cam, cfg, f)]
        acc = [0.0] * 5
        for _ in range(max(steps, 1)):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
            ev[0].record(rast.stream)
            for k, c in enumerate(calls):
                c()
                ev[k + 1].record(rast.stream)
            torch.cuda.synchronize()
            for k in range(5):
                acc[k] += ev[k].elapsed_time(ev[k + 1])
        return {n: a / max(steps, 1) for n, a in zip(self.STAGES, acc)}

    def graph(self, mode, steps):
        """The same frame captured once as a CUDA graph and replayed."""
        import torch

        rast, cfg, f = self.rast, self.cfg(mode), self.frames[mode]
        stream = rast.stream
        side = torch.cuda.Stream(stream.device)
        side.wait_stream(stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            rast.set_stream(side)
            rast.gs_forward(self.scene, self.cam, cfg, f)
            side.synchronize()
            with torch.cuda.graph(g, stream=side):
                rast.gs_forward(self.scene, self.cam, cfg, f)
        rast.set_stream(stream)
        stream.wait_stream(side)
        for _ in range(3):
            g.replay()
        self.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            g.replay()
        e1.record(stream)
        self.barrier()
        _, ms = replica_rate(steps, e0.elapsed_time(e1), self.world, self.max_over_ranks)
        self.check(mode)
        return ms

    def pipelined(self, mode, steps, warmup, nstreams=2):
        """Whole-job rate with nstreams frames in flight: one context per
        stream, each with its own frame buffers, frames dealt out round robin
        over the streams so one frame's blend overlaps the next one's
        preprocess and sort.  Every stream's last image must equal the
        sequential frame's bit for bit."""
        import torch

        base, cfg = self.frames[mode], self.cfg(mode)
        streams = [torch.cuda.Stream(base.image.device) for _ in range(nstreams)]
        rasts = [self.raster.Rasterizer(base.image.device, s) for s in streams]
        frames = [self.raster.Frame(base.n, self.cam.width, self.cam.height, self.tile, base.key_capacity,
                                    base.image.device) for _ in streams]
        for _ in range(max(warmup, 1)):
            for r, f in zip(rasts, frames):
                r.gs_forward(self.scene, self.cam, cfg, f)
        torch.cuda.synchronize()
        self.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        cur = torch.cuda.current_stream(base.image.device)
        e0.record(cur)
        for st in streams:
            st.wait_event(e0)
        for i in range(steps):
            rasts[i % nstreams].gs_forward(self.scene, self.cam, cfg, frames[i % nstreams])
        for st in streams:
            cur.wait_stream(st)
        e1.record(cur)
        torch.cuda.synchronize()
        self.barrier()
        _, ms = replica_rate(steps, e0.elapsed_time(e1), self.world, self.max_over_ranks)
        self.rast.gs_forward(self.scene, self.cam, cfg, base)
        torch.cuda.synchronize()
        for r, f in zip(rasts, frames):
            K, flags = r.gs_read_status(f, raise_on_error=False)
            if flags or not torch.equal(f.image, base.image):
                raise RuntimeError(f"pipelined frame differs from the sequential one ({mode}, flags {flags})")
        return ms

    def table(self, steps, warmup, stage_steps):
        """ms/frame, frames/s, K and per-stage ms of every mode."""
        out = {}
        for m in self.frames:
            ms, _, _ = self.timed(m, steps, warmup)
            out[m] = {"ms_per_frame": ms, "fps": 1e3 / ms, "keys": self.keys[m],
                      "stages_ms": self.stages(m, stage_steps)}
        return out

    def image_diff(self, a, b):
        """Pixels where mode a's and mode b's images differ, and the max |difference|."""
        import torch

        for m in (a, b):
            self.rast.gs_forward(self.scene, self.cam, self.cfg(m), self.frames[m])
        torch.cuda.synchronize()
        d = (self.frames[a].image - self.frames[b].image).abs().amax(0)
        return {"pixels_differing": int((d > 0).sum().item()), "max_abs_diff": float(d.max().item()),
                "pixels": int(d.numel())}


def stage_work(st, n, n_counted, K, sh_bytes, hw, tiles, passes):
    """Algorithmic bytes per stage (the per-unit figures of the design notes
    times the units of this frame)."""
    return {
        # geometry (40 B) and opacity (4 B) read and a 4 B count written for
        # every Gaussian; SH read and the 48 B 2D state written for every
        # counted one
        "preprocess": n * (44 + 4) + n_counted * (sh_bytes + 48),
        # counts read twice (scan, emit); the 32 B of 2D state the tile function
        # needs (centre and depth; conic and threshold, or the 3-sigma radius)
        # read once per counted Gaussian; 12 B per key written
        "intersect": n * 8 + n_counted * 32 + K * 12,
        # lower bound: read and write every (key, value) pair once
        "sort": K * 24,
        # the onesweep design: one histogram read + 24 B per key and pass
        "sort_design": K * 8 + K * 24 * passes,
        "tile_ranges": K * 8 + tiles * 8,
        # blend: each key's 4 B value and each counted Gaussian's 48 B of 2D
        # state read once, 20 B per pixel written (image, final T, last index)
        "render": K * 4 + n_counted * 48 + hw * 20,
    }


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2412_00578_gb300 import build, raster, synth

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    scene_cpu, cam = workload(args)
    scene = scene_cpu.to(dev)
    renderer = raster.Renderer(dev)
    rast = renderer.rast
    stream = rast.stream

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    max_over_ranks = make_max_reduce(dist if world > 1 else None, dev)

    modes = [m for m in args.modes.split(",") if m]
    assert modes and modes[0] == "accutile", "the headline mode is accutile"
    T = ModeTimer(raster, renderer, scene, cam, args.tile, modes, barrier, max_over_ranks, world)
    keys = T.keys

    # --- headline: AccuTile, K timed frames
    sampler = ClockSampler(None)
    ms_acc, launches, clocks = T.timed("accutile", args.steps, args.warmup, sampler)
    per_mode = {"accutile": {"ms_per_frame": ms_acc, "fps": 1e3 / ms_acc, "keys": keys["accutile"]}}
    per_mode["accutile"]["ms_per_frame_cuda_graph"] = T.graph("accutile", args.steps)
    ms_pipe = T.pipelined("accutile", args.steps, args.warmup)
    per_mode["accutile"]["pipelined_two_streams"] = {
        "ms_per_frame": ms_pipe, "fps": 1e3 / ms_pipe,
        "how": "two frames in flight on two streams (own contexts and frame buffers), images equal to the "
               "sequential frame; value stays the sequential rate"}
    for m in modes[1:]:
        ms, _, _ = T.timed(m, max(10, args.steps // 2), args.warmup)
        per_mode[m] = {"ms_per_frame": ms, "fps": 1e3 / ms, "keys": keys[m]}
    stages = {m: T.stages(m, args.stage_steps) for m in modes} if args.stage_steps > 0 else {}
    diff_3sigma = T.image_diff("accutile", "3sigma") if "3sigma" in modes else None

    # --- roofline: the dominant kernel (blend, the render stage) and the whole frame
    pk = peaks()
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    cfg_acc = raster.cfg_struct(args.tile, "accutile")
    f_acc = T.frames["accutile"]
    rast.gs_forward(scene, cam, cfg_acc, f_acc)
    ev_pairs, contrib_pairs, exec_pairs = rast.gs_render_stats(cam, cfg_acc, f_acc)
    n = scene.n
    n_counted = int((f_acc.counts[:n] > 0).sum().item())
    K = keys["accutile"]
    hw = cam.width * cam.height
    tiles = f_acc.gx * f_acc.gy
    passes, digit_bits, depth_bits = rast.gs_read_sort_plan(cfg_acc, f_acc)
    st = stages["accutile"] if stages else T.stages("accutile", 3)
    work = stage_work(st, n, n_counted, K, 4 * 3 * (scene.sh_degree + 1) ** 2, hw, tiles, passes)
    hbm = pk["hbm_gbs"]
    stage_frac = {}
    for k in T.STAGES:
        gbs = work[k] / (st[k] * 1e-3) / 1e9
        stage_frac[k] = {"ms": st[k], "algorithmic_bytes": work[k], "gbs": gbs, "hbm_frac": gbs / hbm}
    stage_frac["sort"]["design_bytes"] = work["sort_design"]
    stage_frac["sort"]["plan"] = {"passes": passes, "digit_bits": digit_bits, "depth_bits_kept": depth_bits,
                                  "tile_bits": max(tiles - 1, 0).bit_length()}
    stage_frac["sort"]["design_hbm_frac"] = work["sort_design"] / (st["sort"] * 1e-3) / 1e9 / hbm
    # blend work per evaluated pair (dx, dy, 2b dy, c dy dy, two fma, compare):
    # 8 flop; per contributing pair about 10 more (alpha, T (1 - alpha), stop
    # test, alpha T, three colour fma) plus one exponential, counted apart
    blend_flops = 8 * ev_pairs + 10 * contrib_pairs
    fp32_peak = n_sm * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12
    achieved = blend_flops / (st["render"] * 1e-3) / 1e12
    roof = {"kernel": f"blend_kernel<{args.tile}>", "bound": "alu", "achieved": achieved, "peak": fp32_peak,
            "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": blend_traffic(K),
            "time_ms": st["render"], "time_src": "CUDA events around gs_render (the blend kernel alone)",
            "work": {"evaluated_pairs": ev_pairs, "contributing_pairs": contrib_pairs, "flops": blend_flops,
                     "flop_per_evaluated_pair": 8, "flop_per_contributing_pair": 10,
                     "exp_evaluations": contrib_pairs, "executed_pairs_after_culling": exec_pairs},
            "peak_src": f"{n_sm} SMs x 128 FP32 lanes x 2 flop x {pk['sm_max_mhz']:.0f} MHz (derived: "
                        "MEASURED_PEAKS.json has no FP32 figure); of derived peak"}
    # whole frame: the sum of the stages' lower-bound times over the frame time
    lb_ms = {k: work[k] / (hbm * 1e9) * 1e3 for k in ("preprocess", "intersect", "sort", "tile_ranges")}
    lb_ms["render"] = max(blend_flops / (fp32_peak * 1e12), work["render"] / (hbm * 1e9)) * 1e3
    frame_roof = {"lower_bound_ms": lb_ms, "sum_lower_bound_ms": sum(lb_ms.values()), "ms_per_frame": ms_acc,
                  "frac": sum(lb_ms.values()) / ms_acc,
                  "how": "HBM stages: algorithmic bytes / measured copy bandwidth (sort: 24 B per key); "
                         "blend: max(flops / FP32 peak, bytes / HBM)"}

    # --- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, scene, scene_cpu, cam, rast, cfg_acc, f_acc, stream, barrier, max_over_ranks, world)

    backward = None
    if not args.no_backward:
        backward = run_backward(args, raster, rast, scene, cam, cfg_acc, f_acc, stream, max_over_ranks, barrier)

    # --- the other configurations: 16k box at 320x240 and the 300k prune, all modes
    configs = None
    if not args.no_configs:
        configs = {}
        box, box_cam = synth.small_box_workload()
        Tb = ModeTimer(raster, raster.Renderer(dev), box.to(dev), box_cam, 16, modes, barrier, max_over_ranks, world)
        configs["box-16k-320x240"] = Tb.table(max(20, args.steps), args.warmup, max(args.stage_steps, 3))
        pr = synth.prune_random(scene_cpu, 300_000, seed=1).to(dev)
        Tp = ModeTimer(raster, raster.Renderer(dev), pr, cam, args.tile, modes, barrier, max_over_ranks, world)
        configs["outdoor-300k-prune-1280x840"] = Tp.table(max(20, args.steps), args.warmup, max(args.stage_steps, 3))
        del Tb, Tp, pr

    # --- CPU oracle baseline (rank 0, N = 1 only) and the FP64 error of the headline frame
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(args, scene_cpu, cam, f_acc)

    multiview = None
    if not args.no_multiview:
        multiview = run_multiview(args, dev, max_over_ranks, barrier)

    served = None
    if not args.no_serve and rank == 0:
        served = run_serving(args, dev, scene)

    pruning = None
    if not args.no_pruning and rank == 0:
        from paper_2412_00578_gb300 import prune

        sch = prune.Schedule(scale=args.prune_scale)
        task = prune.make_task(dev)
        pruning = {"task": "fit 16 seeded views (256x192) of a 20k-Gaussian box scene from a 40k-Gaussian "
                           "over-complete start; L1 + D-SSIM, Adam, 3D-GS densification and opacity resets; "
                           f"iteration counts x{args.prune_scale} of the paper's 30k",
                   "soft_hard": prune.run_schedule(dev, sch, task),
                   "pup_vs_efficient": prune.run_pup_vs_efficient(dev, sch, task)}

    if rank == 0:
        fps = world * 1e3 / ms_acc
        emit({"metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_acc, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_dict(args, cam),
              "ms_per_frame": ms_acc, "modes": per_mode,
              "speedup_vs_3sigma": (per_mode["3sigma"]["ms_per_frame"] / ms_acc) if "3sigma" in per_mode else None,
              "image_vs_3sigma": diff_3sigma,
              "speedup_vs_snugbox": (per_mode["snugbox"]["ms_per_frame"] / ms_acc) if "snugbox" in per_mode else None,
              "stages_ms": stages, "stage_roofline": stage_frac, "frame_roofline": frame_roof,
              "roofline": roof, "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
              "cpu_baseline": cpu, "backward": backward, "configs": configs, "multiview": multiview,
              "served": served, "pruning": pruning})
    if world > 1:
        dist.destroy_process_group()


def run_e2e(args, scene, scene_cpu, cam, rast, cfg, frame, stream, barrier, max_over_ranks, world):
    """The same frame through the public API with the scene uploaded from
    pinned host memory and the image read back every step."""
    import torch

    from paper_2412_00578_gb300 import synth

    dev = scene.means.device
    fields = ("means", "scales", "rotations", "opacities", "sh")
    host = {k: getattr(scene_cpu, k).pin_memory() for k in fields}
    img_host = torch.empty(3, cam.height, cam.width, dtype=torch.float32).pin_memory()
    h2d = sum(v.numel() * 4 for v in host.values())
    d2h = img_host.numel() * 4
    steps = min(args.steps, 20)

    # the host-to-device link, measured here: the scene's upload alone
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for k, v in host.items():
            getattr(scene, k).copy_(v, non_blocking=True)
    barrier()
    a0.record(stream)
    for _ in range(3):
        with torch.cuda.stream(stream):
            for k, v in host.items():
                getattr(scene, k).copy_(v, non_blocking=True)
    a1.record(stream)
    barrier()
    h2d_gbs = 3 * h2d / (a0.elapsed_time(a1) * 1e-3) / 1e9

    def e2e_step():
        with torch.cuda.stream(stream):
            for k, v in host.items():
                getattr(scene, k).copy_(v, non_blocking=True)
        rast.gs_forward(scene, cam, cfg, frame)
        with torch.cuda.stream(stream):
            img_host.copy_(frame.image, non_blocking=True)

    for _ in range(3):
        e2e_step()
    barrier()
    a0.record(stream)
    for _ in range(steps):
        e2e_step()
    a1.record(stream)
    barrier()
    ms_serial = max_over_ranks(a0.elapsed_time(a1)) / steps

    # Pipelined: two device copies of the scene; each step still uploads its
    # whole scene and reads back its image, but step i+1's upload (on a copy
    # stream) overlaps step i's render.
    bufs = [scene, synth.Scene(*[torch.empty_like(getattr(scene, k)) for k in fields], scene.sh_degree)]
    cstream = torch.cuda.Stream(dev)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    released = [torch.cuda.Event(), torch.cuda.Event()]
    for ev in released:
        ev.record(stream)

    def pipe_step(i):
        b = i % 2
        cstream.wait_event(released[b])
        with torch.cuda.stream(cstream):
            for k, v in host.items():
                getattr(bufs[b], k).copy_(v, non_blocking=True)
        copied[b].record(cstream)
        stream.wait_event(copied[b])
        rast.gs_forward(bufs[b], cam, cfg, frame)
        with torch.cuda.stream(stream):
            img_host.copy_(frame.image, non_blocking=True)
        released[b].record(stream)

    for i in range(3):
        pipe_step(i)
    barrier()
    a0.record(stream)
    cstream.wait_event(a0)
    for i in range(steps):
        pipe_step(i)
    a1.record(stream)
    barrier()
    ms_e2e = max_over_ranks(a0.elapsed_time(a1)) / steps

    # Scene resident (a renderer's usual case): per step a camera (the host
    # gs_camera struct, carried into the launch) and the image read back to
    # pinned host memory; two frames, so frame i's read-back (copy stream)
    # overlaps frame i+1's render.
    from paper_2412_00578_gb300 import raster

    frames = [frame, raster.Frame(frame.n, cam.width, cam.height, frame.tile, frame.key_capacity, dev)]
    imgs = [img_host, torch.empty_like(img_host).pin_memory()]
    rendered = [torch.cuda.Event(), torch.cuda.Event()]
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    for ev in copied:
        ev.record(cstream)

    def res_step(i):
        b = i % 2
        stream.wait_event(copied[b])  # the last read-back of this frame's image is done
        rast.gs_forward(scene, cam, cfg, frames[b])
        rendered[b].record(stream)
        cstream.wait_event(rendered[b])
        with torch.cuda.stream(cstream):
            imgs[b].copy_(frames[b].image, non_blocking=True)
        copied[b].record(cstream)

    for i in range(3):
        res_step(i)
    barrier()
    a0.record(stream)
    cstream.wait_event(a0)
    for i in range(steps):
        res_step(i)
    stream.wait_event(copied[(steps - 1) % 2])
    a1.record(stream)
    barrier()
    ms_res = max_over_ranks(a0.elapsed_time(a1)) / steps
    torch.cuda.synchronize(dev)
    if not torch.equal(imgs[0].to(dev), frames[0].image):
        raise RuntimeError("resident-scene read-back differs from the frame")
    cam_bytes = ctypes.sizeof(raster.GsCamera)
    resident = {"value": world * 1e3 / ms_res, "unit": "frames/s", "ms_per_frame": ms_res,
                "h2d_bytes_per_step": cam_bytes, "d2h_bytes_per_step": d2h,
                "path": "scene resident in HBM; per step the camera (host gs_camera struct, carried into the "
                        "launch) and gs_forward into one of two frames, whose image is read back to pinned host "
                        "memory on a copy stream while the next frame renders"}
    return {"value": world * 1e3 / ms_e2e, "unit": "frames/s", "ms_per_frame": ms_e2e,
            "resident_scene": resident,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "path": "per step: pinned host scene -> device copy (copy stream, into one of two device buffers), "
                    "gs_forward, image -> pinned host; step i+1's copy overlaps step i's render",
            "ms_per_frame_serial": ms_serial,
            "serial_path": "the same steps with no overlap (copy, render, read back in order on one stream)",
            "h2d_gbs_measured": h2d_gbs,
            "h2d_bound_ms": h2d / (h2d_gbs * 1e9) * 1e3}


def run_cpu_baseline(args, scene_cpu, cam, f_acc):
    """The oracle timed on the host cores: all cores (OpenMP build of the same
    code) and one thread, FP32, AccuTile, the full headline frame; and the FP64
    oracle's image error of the GPU frame beside the FP32 parity."""
    import oracle

    oracle.build()
    oracle.build(omp=True)
    cores = os.cpu_count() or 1
    img = f_acc.image.cpu().numpy().astype("float64")
    t0 = time.perf_counter()
    ref = oracle.render(scene_cpu, cam, args.tile, 2, prec64=False)
    t_single = time.perf_counter() - t0
    frames = 3
    t0 = time.perf_counter()
    for _ in range(frames):
        ref_omp = oracle.render(scene_cpu, cam, args.tile, 2, prec64=False, omp=True)
    t_omp = (time.perf_counter() - t0) / frames
    ref64 = oracle.render(scene_cpu, cam, args.tile, 2, prec64=True, omp=True)
    return {"value": 1.0 / t_omp, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"{frames} full {cam.width}x{cam.height} AccuTile frames of the {args.n}-Gaussian scene, FP32 "
                      f"oracle built with OpenMP over Gaussians and pixel rows on {cores} host threads "
                      f"({t_omp:.2f} s per frame)",
            "single_thread": {"value": 1.0 / t_single, "unit": "frames/s", "cores": 1,
                              "sample": f"one full frame, same oracle without OpenMP ({t_single:.2f} s)"},
            "image_max_abs_err_vs_gpu": float(abs(img - ref["image"]).max()),
            "image_max_abs_err_omp_vs_gpu": float(abs(img - ref_omp["image"]).max()),
            "image_max_abs_err_gpu_vs_fp64_oracle": float(abs(img - ref64["image"]).max())}


def run_backward(args, raster, rast, scene, cam, cfg, frame, stream, max_over_ranks, barrier):
    """gs_render_backward on the headline frame: dL/dimage ~ N(0, 1), all
    parameter gradients, the 2D-mean gradient and the pruning score."""
    import torch

    n = int(scene.means.shape[1])
    dev = scene.means.device
    grads = {k: torch.empty_like(getattr(scene, k)) for k in ("means", "scales", "rotations", "opacities", "sh")}
    grads["means2d"] = torch.empty(2, n, dtype=torch.float32, device=dev)
    grads["score"] = torch.zeros(n, dtype=torch.float32, device=dev)
    work = torch.empty(raster.backward_work_bytes(n) // 4, dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev).manual_seed(7)
    dL = torch.randn(3, cam.height, cam.width, device=dev, generator=gen)
    steps = min(args.steps, 50)

    def timed_loop(fn):
        for _ in range(3):
            fn()
        barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(steps):
            fn()
        a1.record(stream)
        barrier()
        return max_over_ranks(a0.elapsed_time(a1)) / steps

    rast.gs_forward(scene, cam, cfg, frame)  # the frame the backward walks
    ms_b = timed_loop(lambda: rast.gs_render_backward(scene, cam, cfg, frame, dL, grads, work))

    def step():
        rast.gs_forward(scene, cam, cfg, frame)
        rast.gs_render_backward(scene, cam, cfg, frame, dL, grads, work)

    ms_fb = timed_loop(step)
    # PUP's sensitivity for the same view (its 5x5 blend sums, Jacobian pass
    # and log det), against the efficient score that comes with the backward
    H = torch.zeros(21, n, dtype=torch.float32, device=dev)
    pwork = torch.empty(max(raster.pup_work_bytes(n) // 4, 4), dtype=torch.float32, device=dev)
    pscore = torch.empty(n, dtype=torch.float32, device=dev)
    rast.gs_forward(scene, cam, cfg, frame)

    def pup_step():
        rast.gs_pup_accumulate(scene, cam, cfg, frame, H, pwork)
        rast.gs_pup_score(H, n, pscore)

    ms_pup = timed_loop(pup_step)
    return {"workload": f"{WORKLOAD} AccuTile frame, dL/dimage ~ N(0, 1)", "steps": steps,
            "ms_backward": ms_b, "ms_forward_plus_backward": ms_fb,
            "ms_pup_sensitivity_one_view": ms_pup,
            "score_bytes_per_gaussian": {"efficient": 4, "pup_hessian": 84, "pup_work": 64, "backward_work": 48},
            "kernels": "memset, blend_backward<16>, preprocess_backward",
            "gaussians_with_score": int((grads["score"] > 0).sum().item())}


def run_multiview(args, dev, max_over_ranks, barrier):
    import torch

    from paper_2412_00578_gb300 import autotune, raster, synth

    scene = synth.blob_scene(args.mv_n, seed=5).to(dev)
    cams = synth.multiview_cameras(args.mv_cams, seed=6)
    tuned = autotune.tune(scene, cams, dev, reps=3)
    br = raster.BatchRenderer(dev, tile=tuned["tile"], sort_digit_bits=tuned["sort_digit_bits"])
    br.capture(scene, cams)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        br.replay()
    barrier()
    reps = max(5, min(args.steps, 50))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        br.replay()
    e1.record(stream)
    barrier()
    ms_batch = max_over_ranks(e0.elapsed_time(e1)) / reps
    K, flags = br.rast.gs_batch_status(br.frame, raise_on_error=False)
    # the same 64 views one by one through the single-view path (its tile 16 default)
    r = raster.Renderer(dev)
    for c in cams:
        r.render(scene, c, "accutile", 16)
    cfg = raster.cfg_struct(16, "accutile")
    frames = [r.frame(scene.n, c.width, c.height, 16) for c in cams]
    barrier()
    e0.record(stream)
    for _ in range(2):
        for c, f in zip(cams, frames):
            r.rast.gs_forward(scene, c, cfg, f)
    e1.record(stream)
    barrier()
    ms_seq = e0.elapsed_time(e1) / 2
    return {"workload": f"blob-{args.mv_n // 1000}k, {len(cams)} orbit cameras, resolutions from "
                        "{640x480, 980x545, 1332x876, 1920x1080}",
            "autotuned": {"tile": tuned["tile"], "sort_digit_bits": tuned["sort_digit_bits"] or 8,
                          "timings_ms": tuned["timings"], "cached": tuned["cached"]},
            "ms_per_batch_graph": ms_batch, "views_per_s": len(cams) * 1e3 / ms_batch,
            "ms_64_views_one_by_one": ms_seq, "speedup_vs_one_by_one": ms_seq / ms_batch,
            "keys": K, "status_flags": flags, "frame_gb": br.frame.nbytes() / 1e9}


def run_serving(args, dev, scene_3m):
    import torch

    from paper_2412_00578_gb300 import serve, synth

    scenes = {"300k": synth.blob_scene(300_000, seed=11).to(dev), "600k": synth.blob_scene(600_000, seed=12).to(dev),
              "1.5M": synth.blob_scene(1_500_000, seed=13).to(dev), "3M": scene_3m}
    res = synth.RESOLUTIONS

    def cam_fn(gen):
        w, h = res[int(torch.randint(len(res), (1,), generator=gen))]
        return synth.orbit_camera(gen, w, h)

    free, _ = torch.cuda.mem_get_info(dev)
    budget = int(0.5 * free)
    ex = serve.GpuExecutor(scenes, dev, slots=3, keep_results=False)
    warm = serve.poisson_requests(500.0, 0.05, list(scenes), cam_fn, seed=99)  # sizes the slot frames
    serve.serve(warm, serve.Scheduler({k: v.n for k, v in scenes.items()}, max_batch=16, memory_budget=budget), ex)
    out = {"scenes": {k: v.n for k, v in scenes.items()}, "slots": 3, "max_batch": 16,
           "memory_budget_gb": budget / 1e9, "arrivals_s": args.serve_duration, "rates": {}}
    for rate in [float(x) for x in args.serve_rates.split(",")]:
        reqs = serve.poisson_requests(rate, args.serve_duration, list(scenes), cam_fn, seed=7)
        sch = serve.Scheduler({k: v.n for k, v in scenes.items()}, max_batch=16, memory_budget=budget)
        _, st = serve.serve(reqs, sch, ex)
        out["rates"][str(int(rate))] = {k: st[k] for k in ("requests", "p50_ms", "p99_ms", "frames_per_s",
                                                            "mean_batch", "max_inflight_batches", "span_s")}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
