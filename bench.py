#!/usr/bin/env python
"""Throughput benchmark of the hybrid 3D-4D Gaussian rasterizer.

Metric: forward + backward views/s at 1352x1014 with 300k Gaussians (200k
static 3D + 100k dynamic 4D, the video workload), batched views with BF16
parameter storage, beside the plain per-view FP32 path on the same GPU.

A step is one full pass of the rasterizer over one batch of views: slice and
project, bin and sort, composite, L1 loss, compositing adjoint and projection
adjoint, replayed as one CUDA graph.  Inputs are resident in HBM when the
timed region starts (`value`); `e2e` adds the host->device copy of the step's
parameters and targets from pinned memory and the device->host read of the
loss.  L2 is flushed (a 512 MB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--views V] [--impl reference]

Under torchrun each rank renders its own batch of views (independent
replicas, weak scaling); rank 0 prints one JSON line.  On one GPU the line
also carries the training step (`train_step`), the other batched
configurations (`workloads`: an 8-view arc of 500k Gaussians at mixed
resolutions in FP32 and 1M Gaussians over 4 views at 2704x2028 in BF16) and
the FP64 oracle timed on the host cores (`cpu_baseline`).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd views/s at 1352×1014, 300k Gaussians: batched/BF16 vs plain FP32"
UNIT = "views/s"
N3, N4, W, H = 200_000, 100_000, 1352, 1014


# ---------------------------------------------------------------------------
# process group plumbing (barrier and max-over-ranks timing only)
# ---------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, local, world


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend, init_method="env://")
    return dist


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def reduce_max(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate(views_done: float, seconds: float, device=None):
    """Whole-job throughput of independent replicas: views of all ranks over the
    slowest rank's time.  Returns (views/s, total views, max seconds)."""
    total = reduce_sum(views_done, device)
    t_max = reduce_max(seconds, device)
    return total / t_max, total, t_max


def rank_seed(rank: int) -> int:
    """Each replica renders its own cameras / timestamps of the same scene."""
    return 100 + rank


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-i", str(gpu_index), "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        # nvidia-smi takes a moment to start: the timed region begins after its first sample
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = [n for j, n in enumerate(names) if any(r[5 + j].lower().startswith("active") for r in rows)]
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(pw) if pw else None}


class NvmlSampler:
    """SM clock, power and clock-event reasons read through NVML (the driver's
    management library, read only) about every millisecond from a thread, so
    that a timed region of tens of milliseconds still holds dozens of samples.
    The GPU is matched by its PCI address."""
    SW_POWER_CAP, HW_SLOWDOWN, SW_THERMAL, HW_THERMAL = 0x4, 0x8, 0x20, 0x40
    CLOCK_SM = 1

    def __init__(self, dev):
        import ctypes
        import threading

        import torch
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        props = torch.cuda.get_device_properties(dev)
        bus = b"%08X:%02X:%02X.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(self.h)) != 0:
            raise OSError("no NVML device at " + bus.decode())
        mx = ctypes.c_uint()
        self.max_mhz = mx.value if self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.CLOCK_SM, ctypes.byref(mx)) == 0 \
            else None
        try:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.samples = []
        self.done = threading.Event()
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()
        t0 = time.perf_counter()
        while not self.samples and time.perf_counter() - t0 < 2.0:
            time.sleep(0.001)

    def _run(self):
        ct = self.ct
        c, r, pw = ct.c_uint(), ct.c_ulonglong(), ct.c_uint()
        while not self.done.is_set():
            sm = c.value if self.lib.nvmlDeviceGetClockInfo(self.h, self.CLOCK_SM, ct.byref(c)) == 0 else None
            rs = r.value if self.reasons_fn(self.h, ct.byref(r)) == 0 else None
            w = pw.value / 1000.0 if self.lib.nvmlDeviceGetPowerUsage(self.h, ct.byref(pw)) == 0 else None
            self.samples.append((sm, rs, w))
            time.sleep(0.001)

    def stop(self):
        self.done.set()
        self.thread.join(timeout=5)
        rows = list(self.samples)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["no samples"], "source": "nvml"}
        sm = sorted(x[0] for x in rows if x[0] is not None)
        bits = 0
        for x in rows:
            bits |= x[1] or 0
        names = ((self.HW_SLOWDOWN, "hw_slowdown"), (self.HW_THERMAL, "hw_thermal_slowdown"),
                 (self.SW_THERMAL, "sw_thermal_slowdown"), (self.SW_POWER_CAP, "sw_power_cap"))
        pw = [x[2] for x in rows if x[2] is not None]
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": self.max_mhz,
                "reasons": [n for b, n in names if bits & b], "samples": len(rows),
                "power_w_max": max(pw) if pw else None, "source": "nvml"}


def clock_sampler(dev, index):
    """Clocks during a timed region: NVML when the driver's library loads, else nvidia-smi."""
    try:
        return NvmlSampler(dev)
    except (OSError, AttributeError, RuntimeError):
        return ClockSampler(index)


# ---------------------------------------------------------------------------
# roofline model
# ---------------------------------------------------------------------------

def param_bytes(n3, n4, elem):
    return elem * (n3 * (3 + 3 + 4 + 1 + 48) + n4 * (4 + 4 + 4 + 4 + 1 + 48))


def algorithmic_bytes(stage, n3, n4, V, pix, K, elem, K_super=0):
    """Bytes each stage must move to/from HBM once (inputs read once, outputs
    written once), per launch over the batch.  K: entries of the per-tile lists
    (after the footprint culling and the saturation cut); K_super: entries of
    the binned sort's super-tile lists (0 on the radix path)."""
    N = n3 + n4
    rows = V * N
    proj_row = 8 + 16 + 16 + 16 + 4 + 4       # xy, conic/opacity, rgb/depth, rect, radius, n_tiles
    if stage == "slice_project":
        return param_bytes(n3, n4, elem) + rows * proj_row
    if stage == "adjoint":
        return param_bytes(n3, n4, elem) + rows * (48 + 4) + param_bytes(n3, n4, 4)
    if stage == "composite_fwd":
        return K * 4 + rows * 36 + pix * (12 + 4 + 4)
    if stage == "composite_bwd":
        return K * 4 + rows * 36 + pix * (12 + 4 + 4) + rows * 48
    if stage == "loss":
        return pix * 12 * 3
    if stage == "bin_sort":
        if K_super:
            # depth keys of the rows; the super-tile lists written once and read
            # once with their coverage words; the per-tile lists written once
            return rows * (4 + 4 + 16) + K_super * (4 + 8) * 2 + K * 4
        # depth keys of the rows, instances written once by the duplication and
        # read once by the (tile-digit) sort, sorted ids and tile keys written once
        return rows * (4 + 4 + 16) + K * 8 * 2
    return 0


# FP32 operations per pixel-Gaussian pair on each path of the compositing
# kernels, counted from their source (FMA = 2, exp2 and reciprocal 1, compares
# and selects 0): evaluating -log2(alpha) (dy and two FMA) costs 5; a blended
# pair costs those 5 plus 9 in the forward (exp2, alpha T, transmittance, three
# colour FMA) and plus 25 in the backward (exp2, 1 - alpha, reciprocal,
# replayed T by one multiply, alpha T, three colour-gradient FMA, three FMA for
# <dL/dC, c> - Q, the Q update, dL/dpower and its three moments).
FLOPS_EVAL = 5
FLOPS_BLEND = {"composite_fwd": 5 + 9, "composite_bwd": 5 + 25}
# the round per-pair figures of the method's cost model: about 15 FP32
# operations and one exponential per evaluated pair forward, about 60 backward
COST_MODEL_OPS = {"composite_fwd": 15, "composite_bwd": 60}
KERNEL_SOURCES = {"composite_fwd": ["composite.cu", "splat_internal.cuh"],
                  "composite_bwd": ["composite.cu", "splat_internal.cuh"],
                  "slice_project": ["project.cu", "splat_internal.cuh"],
                  "adjoint": ["project.cu", "splat_internal.cuh"],
                  "adam": ["optim.cu", "splat_internal.cuh"]}


def source_digest(stage):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(stage, []):
        with open(os.path.join(ROOT, "paper_2505_13215_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(stage, views=None):
    """DRAM bytes per launch of `stage` from the committed ncu summary (per view,
    scaled to `views` views, or per launch); None when the kernel's source changed
    since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)[stage]
    except (OSError, ValueError, KeyError):
        return None
    if t.get("source_digest") != source_digest(stage):
        return None
    if "dram_bytes_per_view" in t:
        return int(t["dram_bytes_per_view"] * views)
    return int(t["dram_bytes_per_launch"])


# ---------------------------------------------------------------------------
# measured ceilings of the SM pipes the compositing kernels use
# ---------------------------------------------------------------------------

PROBE_ITERS = {0: 40000, 1: 20000, 2: 2500, 3: 2500}


def measure_pipe_peaks(dev, local, reps=12):
    """FP32 (scalar fma.rn.f32 and packed fma.rn.f32x2) and MUFU (ex2, rcp)
    throughput of this GPU, from splat_peak_probe launches of a few ms timed
    with CUDA events (best of `reps` after two warm-up launches), with the SM
    clock sampled while they run.  Returns TFLOP/s for the FMA probes and
    T operations/s for the MUFU probes."""
    import torch

    from paper_2505_13215_gb300 import abi
    props = torch.cuda.get_device_properties(dev)
    blocks = props.multi_processor_count * 8
    out = torch.zeros(256, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    res = {}
    clocks = clock_sampler(dev, local)
    for kind, name in ((0, "ffma"), (1, "ffma2"), (2, "ex2"), (3, "rcp")):
        for _ in range(2):
            abi.splat_peak_probe(kind, blocks, PROBE_ITERS[kind], out.data_ptr(), sp)
        best = None
        ops = 0.0
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ops = abi.splat_peak_probe(kind, blocks, PROBE_ITERS[kind], out.data_ptr(), sp)
            b.record(stream)
            torch.cuda.synchronize()
            if ops <= 0:
                raise RuntimeError("splat_peak_probe failed")
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        res[name] = round(ops / (best / 1e3) / 1e12, 3)
        res[name + "_ms"] = round(best, 3)
    clk = clocks.stop()
    res["fp32_peak_tflops"] = max(res["ffma"], res["ffma2"])
    res["mufu_peak_tops"] = min(res["ex2"], res["rcp"])
    res["clocks"] = clk
    res["how"] = ("splat_peak_probe: %d CTAs x 256 threads x 8 independent chains of one instruction, best of %d "
                  "launches (CUDA events); FMA counted as 2 FP32 operations, f32x2 as 4" % (blocks, reps))
    return res


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, rank, local, world):
    import numpy as np
    import torch

    from paper_2505_13215_gb300 import abi, autotune, raster, scenes

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the CUDA path has no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    init_dist(world, "nccl")
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    scene, base = scenes.video_scene(seed=1, n3=N3, n4=N4, W=W, H=H)
    views = scenes.jittered_views(base[0], args.views, seed=rank_seed(rank))
    V = len(views)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234 + rank)

    # ---- batched BF16 path (the headline) ----
    G = raster.Gaussians.from_scene(scene, dev, dtype=torch.bfloat16)
    R = raster.Rasterizer(G.n3, G.n4, views, device=dev, keep_keys=False)
    target = torch.rand(R.rgb.shape, generator=gen, device=dev)
    tune = autotune.tune(R, G, target)
    K_inst = R.instances()
    K_super = int(R.n_needed.item())  # binned sort: the larger of K and the super-tile list length
    # the timed graph records no events: an event recorded after each stage
    # inside the graph adds about 3.5 us per event to the step; the stage split
    # comes from separate replays of graphs that do record them
    gs = raster.GraphedStep(R, G, target, copies=1, with_marks=False)
    copies = min(args.steps, 8)
    try:
        gs_marked = raster.GraphedStep(R, G, target, copies=copies, with_marks=True)
        marks_ok = True
    except Exception as e:  # external events inside captures unsupported: stage times from an eager pass
        sys.stderr.write("graph with stage events failed (%s); stage times from eager steps\n" % e)
        gs_marked = None
        marks_ok = False
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for i in range(args.warmup):
        flush.zero_()
        gs.replay(i)
    torch.cuda.synchronize()
    R.check("warm-up")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = clock_sampler(dev, local)
    barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        gs.replay(k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    R.check("timed steps")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    value, views_total, t_max = aggregate(V * args.steps, total_s, dev)
    if marks_ok:
        for k in range(copies):  # the stage split, each replay after an L2 flush as above
            flush.zero_()
            gs_marked.replay(k)
        torch.cuda.synchronize()
        R.check("stage replays")
        per = [gs_marked.stage_ms(k) for k in range(copies)]
        stages = {s: sum(p[s] for p in per) / len(per) for s in raster.Rasterizer.STAGES}
        del gs_marked
    else:
        stages = eager_stage_ms(R, G, target, 5)
    launches = gs.launches_per_step * args.steps

    # ---- plain per-view FP32 path, same views ----
    G32 = raster.Gaussians.from_scene(scene, dev, dtype=torch.float32)
    plain = []
    for v in views:
        Rv = raster.Rasterizer(G32.n3, G32.n4, [v], device=dev, keep_keys=False)
        tv = torch.rand(Rv.rgb.shape, generator=gen, device=dev)
        Rv.autotune_capacity(G32)
        plain.append((Rv, tv))
    # the plain path gets its own tuned launch shape (pixels per lane of the
    # compositing kernels), chosen on its first view like the batched path's
    plain_tune = autotune.tune(plain[0][0], G32, plain[0][1])
    for Rv, _ in plain[1:]:
        Rv.set_options(ppl_fwd=plain_tune["ppl_fwd"], ppl_bwd=plain_tune["ppl_bwd"])
    plain_steps = max(2, args.steps // 2)
    for Rv, tv in plain:
        Rv.step(G32, tv)
    torch.cuda.synchronize()
    pe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(plain_steps)]
    for k in range(plain_steps):
        flush.zero_()
        pe[k][0].record(stream)
        for Rv, tv in plain:
            Rv.step(G32, tv)
        pe[k][1].record(stream)
    torch.cuda.synchronize()
    for Rv, _ in plain:
        Rv.check("plain FP32 path")
    plain_s = sum(a.elapsed_time(b) for a, b in pe) / 1e3
    plain_value = aggregate(V * plain_steps, plain_s, dev)[0]
    del plain

    # ---- end to end: pinned host inputs in, loss out, every step.  Two input sets
    # with a graph each: a copy stream uploads step k+1's inputs while step k runs ----
    host_params = {k: G.t[k].cpu().pin_memory() for k in G.t}
    host_target = target.cpu().pin_memory()
    loss_host = torch.zeros(1, dtype=torch.float32).pin_memory()
    status_host = torch.zeros(4, dtype=torch.int32).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host_params.values()) + host_target.numel() * 4
    d2h = 4 + 16
    G2 = raster.Gaussians({k: G.t[k].clone() for k in G.t}, G.n3, G.n4)
    target2 = target.clone()
    gs2 = raster.GraphedStep(R, G2, target2)
    sets = [(G, target, gs), (G2, target2, gs2)]
    copy_stream = torch.cuda.Stream(device=dev)
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    free = [torch.cuda.Event(), torch.cuda.Event()]

    def upload(b):
        copy_stream.wait_event(free[b])  # the step that last read set b has finished
        with torch.cuda.stream(copy_stream):
            for k, t in host_params.items():
                sets[b][0].t[k].copy_(t, non_blocking=True)
            sets[b][1].copy_(host_target, non_blocking=True)
        ready[b].record(copy_stream)

    def e2e_run(n):
        for b in (0, 1):
            free[b].record(stream)
        upload(0)
        for k in range(n):
            b = k % 2
            if k + 1 < n:
                upload(1 - b)
            stream.wait_event(ready[b])
            sets[b][2].replay(0)
            free[b].record(stream)
            loss_host.copy_(R.loss, non_blocking=True)
            status_host.copy_(R.status, non_blocking=True)

    e2e_run(2)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e2e_run(args.steps)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    if int(status_host[0]) != 0:
        raise abi.SplatError(int(status_host[0]), "e2e steps", int(status_host[1]))
    e2e_value = aggregate(V * args.steps, e2e_s, dev)[0]

    # ---- pair counts of the compositing kernels (one instrumented step, untimed) ----
    counters = torch.zeros(8, dtype=torch.int64, device=dev)
    R.set_options(stats=counters.data_ptr())
    try:
        R.step(G, target)
        torch.cuda.synchronize()
    finally:
        R.set_options(stats=None)
    fe, fb, be, bb = [int(x) for x in counters.cpu().tolist()[:4]]  # the compositing pair counts
    pairs = {"fwd_evaluated": fe, "fwd_blended": fb, "bwd_evaluated": be, "bwd_blended": bb}
    flops = {"composite_fwd": FLOPS_EVAL * fe + (FLOPS_BLEND["composite_fwd"] - FLOPS_EVAL) * fb,
             "composite_bwd": FLOPS_EVAL * be + (FLOPS_BLEND["composite_bwd"] - FLOPS_EVAL) * bb}

    # ---- roofline of the dominant stage ----
    pix = int(sum(R.pix))
    # every stage interval carries one in-graph event, whose cost the empty
    # "loss" interval (the loss is computed inside the forward) measures; the
    # rooflines take the stages' kernel time as the interval less that cost
    ev_over = stages.get("loss", 0.0) if (marks_ok and raster.Rasterizer.fuse_loss) else 0.0
    net = {s: max(1e-6, ms - ev_over) for s, ms in stages.items() if not (s == "loss" and ev_over > 0.0)}
    dom = max(net, key=lambda s: net[s])
    pipes = measure_pipe_peaks(dev, local)
    fp32_peak = pipes["fp32_peak_tflops"]
    # operation counts per pair: the kernels' own source (FLOPS_EVAL / FLOPS_BLEND)
    # and the method's cost model in round figures (about 15 FP32 operations per evaluated pair
    # in the forward, about 60 in the backward)
    model_flops = {"composite_fwd": COST_MODEL_OPS["composite_fwd"] * fe, "composite_bwd": COST_MODEL_OPS["composite_bwd"] * be}
    # MUFU work: one base-2 exponential per evaluated pair in both kernels, plus
    # one reciprocal per evaluated pair in the backward, each at its own
    # measured rate; mufu_frac is the share of the kernel's time the unit needs
    mufu_ops = {"composite_fwd": (fe, 0), "composite_bwd": (be, be)}

    def alu_entry(st, ms):
        a = flops[st] / (ms / 1e3) / 1e12
        a_s = model_flops[st] / (ms / 1e3) / 1e12
        n_ex2, n_rcp = mufu_ops[st]
        mufu_s = n_ex2 / (pipes["ex2"] * 1e12) + n_rcp / (pipes["rcp"] * 1e12)
        return {"bound": "alu", "achieved": round(a, 2), "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": round(a / fp32_peak, 4), "achieved_cost_model": round(a_s, 2),
                "frac_cost_model": round(a_s / fp32_peak, 4),
                "mufu_tops": round((n_ex2 + n_rcp) / (ms / 1e3) / 1e12, 3),
                "mufu_frac": round(mufu_s / (ms / 1e3), 4)}

    if dom in flops:
        roofline = dict(alu_entry(dom, net[dom]), kernel=dom, traffic=measured_traffic(dom, V),
                        peak_source="measured: splat_peak_probe, max of fma.rn.f32 and fma.rn.f32x2 chains",
                        algorithmic_flops=flops[dom], algorithmic_flops_cost_model=model_flops[dom])
    else:
        alg = algorithmic_bytes(dom, G.n3, G.n4, V, pix, K_inst, 2)
        ach = alg / (net[dom] / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(ach / hbm_peak, 4), "traffic": measured_traffic(dom, V),
                    "peak_source": peak_src + " (copy bandwidth)", "algorithmic_bytes": alg}

    # every stage against its own bound: the compositing kernels in FP32
    # operations against the measured FP32 ceiling, the others in algorithmic
    # HBM bytes (inputs read once, outputs written once) against the measured
    # copy bandwidth
    stage_roof = {}
    for st, ms in net.items():
        if ms <= 0:
            continue
        if st == "loss" and raster.Rasterizer.fuse_loss:
            stage_roof[st] = {"fused": "computed inside composite_fwd's pixel epilogue (splat_composite_fwd_l1)"}
            continue
        if st in flops:
            stage_roof[st] = alu_entry(st, ms)
        else:
            alg = algorithmic_bytes(st, G.n3, G.n4, V, pix, K_inst, 2, K_super if K_super > K_inst else 0)
            a = alg / (ms / 1e3) / 1e9
            stage_roof[st] = {"bound": "hbm", "achieved": round(a, 1), "unit": "GB/s", "frac": round(a / hbm_peak, 4),
                              "algorithmic_bytes": int(alg)}
    if raster.Rasterizer.fuse_loss and "loss" not in stage_roof:
        stage_roof["loss"] = {"fused": "computed inside composite_fwd's pixel epilogue (splat_composite_fwd_l1)"}

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 storage, f32 compute", "data": "synthetic",
        "config": {"workload": "video scene 200k 3D + 100k 4D Gaussians, %d views/step at %dx%d, BF16 storage, "
                               "one CUDA graph per step" % (V, W, H),
                   "views_per_step": V, "gaussians": N3 + N4, "resolution": [W, H], "l2": "flushed before each step",
                   "instances_K": K_inst, "capacity_needed": K_super, "autotune": {k: tune[k] for k in ("ppl_fwd", "ppl_bwd", "capacity")},
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "mpixel_per_s": round(value * W * H / 1e6, 1),
        "plain_fp32": {"value": round(plain_value, 2), "unit": UNIT, "path": "per-view launches, FP32 storage, eager",
                       "autotune": {k: plain_tune[k] for k in ("ppl_fwd", "ppl_bwd")}},
        "stage_ms": {k: round(v, 4) for k, v in stages.items()},
        "stage_event_ms": round(ev_over, 4),
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": d2h,
                "pipeline": "pinned host parameters and targets copied on a second stream one step ahead; "
                            "loss and status read back after every step"},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "stage_roofline": stage_roof,
        "composite_pairs": pairs,
        "pipe_peaks": pipes,
        "error_vs_oracle": workload_errors("headline"),
        "fp32_peak_measured": {"tflops": fp32_peak, "sm_mhz": pipes["clocks"].get("sm_mhz"),
                               "ffma_tflops": pipes["ffma"], "ffma2_tflops": pipes["ffma2"]},
        "clocks": clk,
    }
    if not args.no_train:
        del gs, gs2, sets, R, G, G2, target2, G32, flush
        torch.cuda.empty_cache()
        out["train_step"] = run_train(args, hbm_peak, peak_src, dev, rank)
    if rank == 0 and world == 1 and not args.no_extra:
        out["workloads"] = run_workloads(dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(scene, views, samples=args.cpu_samples)
    if rank == 0:
        print(json.dumps(out), flush=True)


# The other batched configurations, reported beside the headline (their
# parity is checked by the workload tests): a 500k-Gaussian arc of 8 cameras
# at mixed resolutions in FP32, and 1M Gaussians over 4 views at 2704x2028 with
# BF16 and with FP16 storage.
WORKLOADS = (
    ("arc 500k (70% 3D), 8 views at 1352x1014 / 676x507, FP32",
     dict(seed=2, n=500_000, frac4=0.3, n_views=8), "float32"),
    ("arc 1M (60% 3D), 4 views at 2704x2028, BF16",
     dict(seed=3, n=1_000_000, frac4=0.4, n_views=4, full=(2704, 2028, 2920.0), half=(2704, 2028, 2920.0)),
     "bfloat16"),
    ("arc 1M (60% 3D), 4 views at 2704x2028, FP16",
     dict(seed=3, n=1_000_000, frac4=0.4, n_views=4, full=(2704, 2028, 2920.0), half=(2704, 2028, 2920.0)),
     "float16"),
)


def workload_errors(name):
    """The errors against the FP64 oracle that the GPU parity test of this
    workload measured (profiles/precision_workloads.json, written from its
    report): per view RGB max-abs and per tensor gradient rel-L2 on the stored
    values, and for half storage also against the FP32 originals."""
    try:
        with open(os.path.join(ROOT, "profiles", "precision_workloads.json")) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    return d.get("workloads", {}).get(name)


def run_workloads(dev, steps=20, warmup=3):
    """Each WORKLOADS entry autotuned and timed as its graphed training step
    (forward, L1 loss, backward) with the L2 flushed before every step."""
    import torch

    from paper_2505_13215_gb300 import autotune, raster, scenes
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    res = {}
    for name, kw, dt in WORKLOADS:
        scene, views = scenes.arc_scene(**kw)
        G = raster.Gaussians.from_scene(scene, dev, dtype=getattr(torch, dt))
        R = raster.Rasterizer(G.n3, G.n4, views, device=dev, keep_keys=False)
        target = torch.rand(R.rgb.shape, device=dev)
        tune = autotune.tune(R, G, target)
        gs = raster.GraphedStep(R, G, target, copies=1)
        for _ in range(warmup):
            flush.zero_()
            gs.replay(0)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            gs.replay(0)
            b.record(stream)
        torch.cuda.synchronize()
        R.check("workload: " + name)
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        res[name] = {"views_per_s": round(R.V / (ms / 1e3), 2),
                     "mpixel_per_s": round(sum(R.pix) / (ms / 1e3) / 1e6, 1), "ms_per_step": round(ms, 3),
                     "views": R.V, "gaussians": G.n, "storage": dt, "instances_K": R.instances(),
                     "autotune": {"ppl_fwd": tune["ppl_fwd"], "ppl_bwd": tune["ppl_bwd"]},
                     "l2": "flushed before each step", "steps": steps,
                     "error_vs_oracle": workload_errors(name)}
        del gs, R, G, target
        torch.cuda.empty_cache()
    return res


TRAIN_N = 300_000
TRAIN_VIEWS = 16
TRAIN_STEPS = 100


def run_train(args, hbm_peak, peak_src, dev, rank):
    """The training step at scale: 300k Gaussians that start 4D, 16 random arc
    views per step at 1352x1014 from a 300-frame sequence, BF16 storage, L1
    loss, fused Adam, and the 4D -> 3D conversion every 100 steps with its
    optimizer state.  One conversion pass runs after the warm-up (the first
    classification, which moves the wide-time-scale Gaussians to 3D); the timed
    steps include the next one."""
    import numpy as np
    import torch

    from paper_2505_13215_gb300 import scenes, train
    rng = np.random.default_rng(500 + rank)
    scene = scenes.training_scene(seed=4, n=TRAIN_N, frac_static=0.7)
    views0 = scenes.random_arc_views(rng, TRAIN_VIEWS)
    # densification statistics gather every step (as in the paper's first 15k iterations);
    # one densification pass is timed after the steps
    tr = train.Trainer(scene, views0, dtype=torch.bfloat16, tau=1.0, convert_every=TRAIN_STEPS,
                       densify_every=10 ** 9, densify_until=10 ** 9)
    gen = torch.Generator(device=dev)
    gen.manual_seed(77 + rank)
    target = torch.rand(tr.R.rgb.shape, generator=gen, device=dev)
    batches = [scenes.random_arc_views(rng, TRAIN_VIEWS) for _ in range(8)]
    for i in range(3):
        tr.step(batches[i % len(batches)], target)
    moved0 = tr.convert()  # the first classification
    for i in range(2):
        tr.step(batches[i % len(batches)], target)
    torch.cuda.synchronize()
    tr.R.check("training warm-up")
    stream = torch.cuda.current_stream()
    steps = TRAIN_STEPS
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    adam_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t_before = tr.t
    ev0.record(stream)
    import ctypes as C

    from paper_2505_13215_gb300 import abi
    from paper_2505_13215_gb300.raster import _ptr
    for k in range(steps):
        tr.R.set_views(batches[k % len(batches)])
        tr.R.step(tr.store, target)
        abi.check(abi.splat_densify_stats(C.byref(tr.R.cproj), tr.R.cviews, tr.R.V, _ptr(tr.R.dproj),
                                          _ptr(tr.accum), _ptr(tr.count), None), "splat_densify_stats")
        adam_ev[k][0].record(stream)
        tr.adam()
        adam_ev[k][1].record(stream)
        if tr.t % tr.convert_every == 0:
            tr.convert()
    ev1.record(stream)
    torch.cuda.synchronize()
    tr.R.check("training steps")
    total_ms = ev0.elapsed_time(ev1)
    n_before = (tr.n3, tr.n4)
    k_before = tr.R.instances()
    t0 = time.perf_counter()
    n_after = tr.densify()
    torch.cuda.synchronize()
    densify_ms = (time.perf_counter() - t0) * 1e3
    adam_ms = sum(a.elapsed_time(b) for a, b in adam_ev) / steps
    conversions = (tr.t // tr.convert_every) - (t_before // tr.convert_every)
    floats = n_before[0] * (3 + 3 + 4 + 1 + 48) + n_before[1] * (4 + 4 + 4 + 4 + 1 + 48)
    adam_bytes = floats * (4 + 12 + 12 + 2)  # gradient in; master, m, v in and out; BF16 copy out
    ach = adam_bytes / (adam_ms / 1e3) / 1e9
    return {
        "workload": "%d Gaussians starting 4D, %d random arc views/step at 1352x1014 over a 300-frame sequence, "
                    "BF16 storage, L1 loss, densification statistics, fused Adam, 4D->3D conversion every %d steps" % (TRAIN_N, TRAIN_VIEWS,
                                                                                          TRAIN_STEPS),
        "steps": steps, "ms_per_step": round(total_ms / steps, 3),
        "steps_per_s": round(1e3 * steps / total_ms, 2), "views_per_s": round(1e3 * steps * TRAIN_VIEWS / total_ms, 1),
        "conversions_timed": int(conversions), "moved_first_pass": int(moved0), "moved_total": int(tr.moved_total),
        "n3": n_before[0], "n4": n_before[1], "share_4d": round(n_before[1] / sum(n_before), 4),
        "instances_K": k_before,
        "densify": {"ms": round(densify_ms, 2), "n3_after": n_after[0], "n4_after": n_after[1],
                    "includes": "clone/split/prune of both sets, storage cast, a rasterizer for the new counts "
                                "and its capacity tuning (one forward)"},
        "adam_ms": round(adam_ms, 4),
        "adam_roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                          "frac": round(ach / hbm_peak, 4), "algorithmic_bytes": int(adam_bytes),
                          "traffic": measured_traffic("adam"),
                          "peak_source": peak_src + " (copy bandwidth)"},
        "data": "synthetic",
    }


def eager_stage_ms(R, G, target, reps):
    import torch
    from paper_2505_13215_gb300 import raster
    acc = {s: 0.0 for s in raster.Rasterizer.STAGES}
    for _ in range(reps):
        m = raster.stage_events()
        R.step(G, target, marks=m)
        torch.cuda.synchronize()
        names = ("start",) + raster.Rasterizer.STAGES
        for a, b in zip(names[:-1], names[1:]):
            acc[b] += m[a].elapsed_time(m[b]) / reps
    return acc


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, as it stands, on a bounded sample
# ---------------------------------------------------------------------------

def _oracle_sample(scene, v, samples, seed):
    """Oracle forward at `samples` random pixels of view v plus the backward of
    a loss on those pixels; returns (seconds, sampled fraction of the view)."""
    import numpy as np

    import oracle as O
    rng = np.random.default_rng(seed)
    npix = v.W * v.H
    pix = rng.choice(npix, size=min(samples, npix), replace=False)
    t0 = time.perf_counter()
    ref = O.render(scene, v, pixels=pix)
    g = np.zeros((3, npix))
    g[:, pix] = np.sign(ref["rgb"] - 0.5)
    O.render_bwd(scene, v, g.reshape(3, v.H, v.W))
    return time.perf_counter() - t0, len(pix) / npix


def _oracle_full_small():
    """The 128x128 workload (3,072 3D + 1,024 4D Gaussians, one view) rendered in
    full by the oracle: seconds of the forward and of forward + backward (L1
    sign gradient against 0.5)."""
    import numpy as np

    import oracle as O
    from paper_2505_13215_gb300 import scenes
    scene, views = scenes.small_scene(seed=0)
    v = views[0]
    t0 = time.perf_counter()
    O.render(scene, v)
    t1 = time.perf_counter()
    ref = O.render(scene, v)
    O.render_bwd(scene, v, np.sign(ref["rgb"] - 0.5).reshape(3, v.H, v.W))
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1


def cpu_baseline(scene, views, samples=1500, seed=0, full_small=True):
    """The FP64 oracle as it stands on the host cores.  Headline value: the
    1352x1014 video workload, forward at `samples` random pixels of view 0 plus
    the backward of a loss on them, all threads, scaled to views/s by the
    sampled fraction.  Also: the same sample single-threaded (fewer pixels),
    and the 128x128 workload rendered in full, forward and forward + backward,
    single-threaded and on all threads."""
    import oracle as O
    v = views[0]
    n_all = O.num_threads()
    dt, frac = _oracle_sample(scene, v, samples, seed)
    out = {"value": round(frac / dt, 6), "unit": UNIT, "cores": n_all, "kind": "oracle",
           "sample": "FP64 oracle forward at %d random pixels of one %dx%d view (of %d Gaussians) plus the "
                     "backward of a loss on them: %.1f s on %d threads; scaled by the sampled fraction %.2e of a view"
                     % (int(round(frac * v.W * v.H)), v.W, v.H, scene.n, dt, n_all, frac)}
    if not full_small:
        return out
    configs = {}
    O.set_num_threads(1)
    try:
        dt1, frac1 = _oracle_sample(scene, v, max(100, samples // 5), seed + 1)
        f1, fb1 = _oracle_full_small()
    finally:
        O.set_num_threads(n_all)
    fN, fbN = _oracle_full_small()
    configs["%dx%d, %d Gaussians, fwd+bwd, sampled pixels" % (v.W, v.H, scene.n)] = {
        "views_per_s": {"1": round(frac1 / dt1, 6), str(n_all): out["value"]},
        "sample": "%d / %d pixels (1 thread), %d (%d threads)" % (int(round(frac1 * v.W * v.H)), v.W * v.H,
                                                                   int(round(frac * v.W * v.H)), n_all)}
    configs["128x128, 4096 Gaussians, full image"] = {
        "fwd_views_per_s": {"1": round(1.0 / f1, 3), str(n_all): round(1.0 / fN, 3)},
        "fwd_bwd_views_per_s": {"1": round(1.0 / fb1, 3), str(n_all): round(1.0 / fbN, 3)},
        "seconds": {"fwd_1": round(f1, 3), "fwd_bwd_1": round(fb1, 3), "fwd_%d" % n_all: round(fN, 3),
                    "fwd_bwd_%d" % n_all: round(fbN, 3)}}
    out["configs"] = configs
    return out


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, rank, local, world):
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="gloo", init_method="env://")
        dist.barrier()
        if rank != 0:
            return
    from paper_2505_13215_gb300 import scenes
    scene, base = scenes.video_scene(seed=1, n3=N3, n4=N4, W=W, H=H)
    views = scenes.jittered_views(base[0], args.views, seed=rank_seed(0))
    for i in range(args.warmup):
        cpu_baseline(scene, views, samples=args.ref_samples // 4, seed=1000 + i, full_small=False)
    vals, total, cores, sample = [], 0.0, None, None
    for k in range(args.steps):
        r = cpu_baseline(scene, [views[k % len(views)]], samples=args.ref_samples, seed=k, full_small=False)
        vals.append(r["value"])
        cores, sample = r["cores"], r["sample"]
    value = len(vals) / sum(1.0 / x for x in vals)  # views per total second
    step_s = sum(1.0 / x for x in vals) / len(vals) * (args.ref_samples / (W * H))
    out = {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "impl": "reference", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * step_s, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "video scene 200k 3D + 100k 4D Gaussians at %dx%d, oracle on a pixel sample" % (W, H),
                      "views_per_step": 1, "gaussians": N3 + N4, "resolution": [W, H]},
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_profile(args):
    """Untimed eager steps of the workload, for profilers (ncu); prints K."""
    import torch

    from paper_2505_13215_gb300 import abi, raster, scenes
    torch.cuda.set_device(0)
    scene, base = scenes.video_scene(seed=1, n3=N3, n4=N4, W=W, H=H)
    views = scenes.jittered_views(base[0], args.views, seed=rank_seed(0))
    dt = torch.bfloat16 if args.dtype == "bf16" else torch.float32
    G = raster.Gaussians.from_scene(scene, "cuda", dtype=dt)
    R = raster.Rasterizer(G.n3, G.n4, views, keep_keys=False)
    ppl_f, ppl_b = (int(x) for x in args.ppl.split(","))
    R.set_options(ppl_fwd=ppl_f, ppl_bwd=ppl_b)
    R.autotune_capacity(G)
    target = torch.rand(R.rgb.shape, device="cuda")
    for _ in range(args.profile):
        R.step(G, target)
    torch.cuda.synchronize()
    R.check("profile steps")
    print("K", R.instances())


def run_profile_train(args):
    """Untimed training steps of the training workload (for profilers); prints the counts."""
    import numpy as np
    import torch

    from paper_2505_13215_gb300 import scenes, train
    torch.cuda.set_device(0)
    rng = np.random.default_rng(500)
    scene = scenes.training_scene(seed=4, n=TRAIN_N, frac_static=0.7)
    tr = train.Trainer(scene, scenes.random_arc_views(rng, TRAIN_VIEWS), dtype=torch.bfloat16, tau=1.0,
                       convert_every=0)
    tr.convert()
    target = torch.rand(tr.R.rgb.shape, device="cuda")
    for _ in range(args.profile_train):
        tr.step(scenes.random_arc_views(rng, TRAIN_VIEWS), target)
    torch.cuda.synchronize()
    tr.R.check("profile training steps")
    print("n3", tr.n3, "n4", tr.n4)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--views", type=int, default=4, help="views per batched step (<= 16)")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--cpu-samples", type=int, default=1500)
    ap.add_argument("--ref-samples", type=int, default=600)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-train", action="store_true", help="skip the training-step measurement")
    ap.add_argument("--no-extra", action="store_true", help="skip the other batched workloads")
    ap.add_argument("--profile", type=int, default=0, help="run this many untimed eager steps (for ncu) and exit")
    ap.add_argument("--profile-train", type=int, default=0,
                    help="run this many untimed steps of the training workload (for ncu) and exit")
    ap.add_argument("--dtype", choices=("bf16", "f32"), default="bf16", help="storage dtype of --profile")
    ap.add_argument("--ppl", default="2,4", help="pixels per lane (forward,backward) of --profile")
    args = ap.parse_args(argv)
    if args.profile:
        return run_profile(args)
    if args.profile_train:
        return run_profile_train(args)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    rank, local, world = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, local, world)
    else:
        run_ours(args, rank, local, world)


if __name__ == "__main__":
    main()
