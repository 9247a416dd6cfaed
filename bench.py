"""Benchmark of the occlusion-point reuse hot path on GB300.

Workload (one step = one frame): 1920x1080 ambient occlusion, 1 cosine ray per pixel,
radius 0.5, over the seeded ~1M-triangle terrain scene (512^2 heightfield + 300
icospheres + 8000 boxes, seed 2), then biased occluder reuse with K = 8 (the receiver
plus 7 shared random offsets in a 15-pixel disk).  Metric: reuse-pass neighbour-samples/s
= pixels * K / reuse time, summed over the timed steps; ms_per_step is the whole frame
(trace + reuse), and frame_neighbour_samples_per_s = pixels * K / frame time beside it.

  python bench.py [--gpus N --steps K --warmup W]    this library (CUDA, sm_103a)
  python bench.py --impl reference ...               the FP64 CPU oracle on host cores
  OCC_LIB_VARIANT=counters python bench.py --count-touch
                                                     traversal counters of the trace
                                                     (instrumented library)

N > 1 runs one independent replica per GPU (the path needs no exchange between GPUs); run
without torchrun, --gpus N relaunches itself as N ranks on this node.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W, H, K, RADIUS, SEED_SCENE, SEED_OFF, DISK_R = 1920, 1080, 8, 0.5, 2, 3, 15.0
METRIC = "reuse-pass neighbour-samples/s and ms/frame (1080p AO, biased K=8 reuse)"
UNIT = "neighbour-samples/s"
WORKLOAD = ("1920x1080 AO, 1 spp, R=0.5, ~1M-tri terrain (seed 2); biased occluder reuse, "
            "K=8 (receiver + 7 shared offsets in a 15-px disk), FP32 records")
FLOPS_PER_PAIR_AO = 21     # d (3), r^2 (5), n_x.d (5), n_z.d (5), product, r^4, divide
L2_FLUSH_BYTES = 512 << 20


class L2Flush:
    """Evicts the step's data from L2 before a timed call: writes a buffer four times the
    L2 size, then reads it back so the lines left behind are clean (otherwise the timed
    kernel would also pay for writing the flush buffer's dirty lines back to HBM)."""

    def __init__(self, device):
        import torch
        self.buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
        self.sink = torch.empty((), dtype=torch.float32, device=device)

    def zero_(self):
        import torch
        self.buf.zero_()
        torch.sum(self.buf, dim=0, out=self.sink)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-quality", action="store_true")
    ap.add_argument("--no-uhd", action="store_true",
                    help="skip the 4K packed K = 16 leg (~4M-triangle scene)")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--count-touch", action="store_true",
                    help="with OCC_LIB_VARIANT=counters: node visits, triangle tests and the "
                         "distinct BVH bytes touched by the 1080p AO and shadow traces")
    ap.add_argument("--profile-step", action="store_true",
                    help="launch the hot kernels once each (1080p: AO trace, window reuse, "
                         "4x2 group reuse, shadow trace, fused AO and shadow trace + 4x2 "
                         "group reuse, then an AO trace and unbiased 4x2 group reuse) and "
                         "exit: the case profiled with ncu")
    return ap.parse_args()


def max_over_ranks(x: float, device) -> float:
    """The largest x over the ranks of the default process group (x itself on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_step: float, steps: int, t_max: float) -> float:
    """Whole-job rate: every rank processed units_per_step per step; the job took the
    slowest rank's time."""
    return world * units_per_step * steps / t_max


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def bench_config(world: int, tris: int) -> dict:
    """The workload description both arms print (the same dict, key for key)."""
    return {"workload": WORKLOAD, "W": W, "H": H, "K": K, "radius": RADIUS, "tris": tris,
            "pattern": "offsets", "estimator": "biased",
            "l2": f"GPU arm: flushed before every step ({L2_FLUSH_BYTES >> 20} MB written, then "
                  "read back)",
            "parallelism": f"replicas x{world}"}


def relaunch_as_ranks(n: int) -> int:
    """Runs this script as n ranks on this node (torchrun), when started without it."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__),
           *sys.argv[1:]]
    return subprocess.call(cmd)


def scene_inputs():
    import synth
    scene = synth.scene_terrain(grid=512, n_spheres=300, n_boxes=8000, seed=SEED_SCENE)
    offs = synth.disk_offsets(K, DISK_R, seed=SEED_OFF)
    return scene, synth.camera_c2(), offs


# ----------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------
# our implementation
# ----------------------------------------------------------------------------------------

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured", d
    return 6800.0, "fallback", {}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def cpu_baseline(scene, cam, offs, budget_s: float = 12.0) -> dict:
    """The FP64 oracle, as it stands, on this host: trace + reuse of square pixel blocks
    (plus the halo their neighbour sets reach) until ~budget_s of work is done, on all the
    cores this process may use, then on one core for a quarter of the time; trace and
    reuse timed separately."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    oracle.set_num_threads(cores)
    osc = oracle.OracleScene(scene.tris)
    pos, nrm, _ = oracle.gbuffer(osc, cam.as_array(), W, H, scene.eps)
    rec = np.zeros((H, W, 8))
    rec[..., 7] = -1.0
    mg = np.full((H, W), np.inf)
    out = np.zeros((H, W))
    omg = np.zeros((H, W))
    pat = (2, 0, 0, offs)
    hx0, hx1 = max(0, -offs[:, 0].min()), max(0, offs[:, 0].max())
    hy0, hy1 = max(0, -offs[:, 1].min()), max(0, offs[:, 1].max())
    rng = np.random.default_rng(11)

    def run(B, budget):
        receivers, t_tr, t_ru, blocks = 0, 0.0, 0.0, 0
        while t_tr + t_ru < budget and blocks < 100000:
            x0 = int(rng.integers(hx0, W - B - hx1))
            y0 = int(rng.integers(hy0, H - B - hy1))
            t0 = time.perf_counter()
            oracle.trace(osc, 0, pos, nrm, radius=RADIUS, seed=1, sample=0,
                         region=(x0 - hx0, y0 - hy0, B + hx0 + hx1, B + hy0 + hy1), out=(rec, mg))
            t1 = time.perf_counter()
            oracle.reuse(None, 0, pos, nrm, rec, pat, oracle.EST_BIASED, radius=RADIUS,
                         region=(x0, y0, B, B), out=(out, omg))
            t2 = time.perf_counter()
            t_tr += t1 - t0
            t_ru += t2 - t1
            receivers += B * B
            blocks += 1
        return receivers, t_tr, t_ru, blocks

    n, t_tr, t_ru, blocks = run(48, budget_s)
    oracle.set_num_threads(1)
    n1, t_tr1, t_ru1, blocks1 = run(48, budget_s / 4)
    oracle.set_num_threads(cores)
    return {"value": n * K / t_ru, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle", "cpu_model": cpu_model(),
            "frame_neighbour_samples_per_s": n * K / (t_tr + t_ru),
            "trace_rays_per_s": n / t_tr * ((48 + hx0 + hx1) * (48 + hy0 + hy1)) / (48 * 48),
            "trace_s": t_tr, "reuse_s": t_ru,
            "reuse_neighbour_samples_per_s": n * K / t_ru,
            "single_core": {"value": n1 * K / t_ru1, "unit": UNIT, "cores": 1,
                            "frame_neighbour_samples_per_s": n1 * K / (t_tr1 + t_ru1),
                            "trace_s": t_tr1, "reuse_s": t_ru1,
                            "sample": f"{blocks1} random 48x48 blocks with their halos"},
            "sample": (f"{blocks} random 48x48 receiver blocks of the 1080p frame: trace of "
                       f"each block plus its {hx0}/{hx1}/{hy0}/{hy1}-px halo, then biased "
                       f"K=8 reuse of the block ({t_tr + t_ru:.1f} s)")}


GROUP_BYTES_PER_PX = 52   # x 12, n 12, z 12, n_z 12, out 4
# DRAM bytes (read + write) per launch from one `ncu --set full` capture of
# `bench.py --profile-step` (cold L2); None once a kernel changes
NCU_TRAFFIC = {"k_trace_dyn<AO>": 72.004352e6 + 28.321792e6,
               "k_reuse_tile<AO,8>": 132.7616e6 + 7.310336e6,
               "k_reuse_group<AO,biased,4,2>": 114.169088e6 + 5.264384e6}
NCU_TRACE_ISSUE_ACTIVE = 0.6522   # smsp__issue_active of k_trace_dyn<AO> in its capture
NCU_TRACE_WARP_INSTR = 255.203861e6   # smsp__inst_executed.sum of k_trace_dyn<AO>, same capture
# What the 1080p AO trace (seed 1, sample 0) traverses, from the instrumented library:
# OCC_LIB_VARIANT=counters python bench.py --count-touch
TRACE_TOUCH = {"rays": 1409214, "node_visits": 21643959, "triangle_tests": 5850259,
               "distinct_nodes": 44564, "distinct_triangles": 122825, "distinct_bytes": 11599792}


def fp32_peak(occ, ctx, dev, stream) -> dict:
    """Measured FP32 peak: the library's FMA-chain probe over 8 CTAs of 256 threads per SM
    (scalar fma.rn.f32 and paired fma.rn.f32x2), best of 10 CUDA-event timings each, with
    the SM clock sampled during the runs."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, iters = 8 * sms, 4096
    sink = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    clk = ClockSampler(dev.index)
    clk.start()
    res = {}
    for paired in (False, True):
        flop = occ.occ_debug_fp32_peak(ctx, paired, iters, blocks, sink, stream=stream)
        best = None
        for _ in range(10):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            occ.occ_debug_fp32_peak(ctx, paired, iters, blocks, sink, stream=stream)
            b.record(stream)
            b.synchronize()
            t = a.elapsed_time(b) * 1e-3
            best = t if best is None else min(best, t)
        res["paired_f32x2" if paired else "scalar"] = flop / best / 1e12
    c = clk.stop()
    ctx.sync()
    res.update(unit="TFLOP/s", sm_mhz=c["sm_mhz"], sm_max_mhz=c["sm_max_mhz"],
               probe=f"{blocks} CTAs x 256 threads x 16 FMA chains x {iters} iterations")
    res["peak"] = max(res["scalar"], res["paired_f32x2"])
    return res


def time_kernel(fn, flush, stream, iters: int) -> dict:
    """Mean CUDA-event time of fn(stream) with the L2 flushed before every call."""
    import torch
    for _ in range(3):
        fn(stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(iters)]
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        fn(stream)
        b.record(stream)
    torch.cuda.synchronize()
    t = np.array([a.elapsed_time(b) for a, b in ev]) * 1e-3
    return {"s": float(t.mean()), "ms": float(t.mean() * 1e3), "ms_min": float(t.min() * 1e3)}


def shadow_frame(occ, ctx, gb, bvh, pat, rec, out, flush, stream) -> dict:
    """1080p area-light shadow frame on the same scene: trace, biased K=8 reuse, and the
    no-reuse and light-sample box-mean (Light(8)) baselines on the same records."""
    import synth
    light = synth.light_c3().as_array()
    tr = time_kernel(lambda st: occ.occ_trace_shadow(ctx, gb, bvh, light, 1, 0, out=rec, stream=st),
                     flush, stream, 100)
    ru = time_kernel(lambda st: occ.occ_reuse_shadow(ctx, gb, rec, pat, K, occ.OCC_EST_BIASED,
                                                     out=out, stream=st), flush, stream, 100)
    lb = time_kernel(lambda st: occ.occ_reuse_shadow(ctx, gb, rec, pat, K, occ.OCC_EST_BOXMEAN,
                                                     out=out, stream=st), flush, stream, 100)
    gr = time_kernel(lambda st: occ.occ_reuse_shadow(ctx, gb, rec, occ.Pattern.group(4, 2), 8,
                                                     occ.OCC_EST_BIASED, out=out, stream=st),
                     flush, stream, 100)
    return {"trace_ms": tr["ms"], "reuse_offsets_k8_ms": ru["ms"], "light8_boxmean_ms": lb["ms"],
            "reuse_group4x2_ms": gr["ms"], "ms_per_frame": tr["ms"] + ru["ms"],
            "light": "1 x 0.5 rectangle at z=4 facing down"}


def fused_frame(occ, ctx, gb, bvh, rec, out, flush, stream) -> dict:
    """Steps 1-3 with 4x2 shared groups (K = 8, biased) on the same frame: the separate
    trace + group-reuse launches against the fused kernel that keeps the occluders on chip
    (AO on both of its launch paths, and shadows)."""
    import synth
    light = synth.light_c3().as_array()
    g, B = occ.Pattern.group(4, 2), occ.OCC_EST_BIASED

    def ao_separate(st):
        occ.occ_trace_ao(ctx, gb, bvh, RADIUS, 1, 0, out=rec, stream=st)
        occ.occ_reuse_ao(ctx, gb, rec, g, 8, B, out=out, stream=st)

    def sh_separate(st):
        occ.occ_trace_shadow(ctx, gb, bvh, light, 1, 0, out=rec, stream=st)
        occ.occ_reuse_shadow(ctx, gb, rec, g, 8, B, out=out, stream=st)

    res = {"ao_separate_ms": time_kernel(ao_separate, flush, stream, 100)["ms"]}
    try:
        for path in (1, 2):
            occ.occ_set_tuning(ctx, fused_ao_path=path)
            res[f"ao_fused_path{path}_ms"] = time_kernel(
                lambda st: occ.occ_trace_reuse_ao(ctx, gb, bvh, RADIUS, 1, 0, g, 8, B, out=out,
                                                  stream=st), flush, stream, 100)["ms"]
    finally:
        occ.occ_set_tuning(ctx)
    res["shadow_separate_ms"] = time_kernel(sh_separate, flush, stream, 100)["ms"]
    res["shadow_fused_ms"] = time_kernel(
        lambda st: occ.occ_trace_reuse_shadow(ctx, gb, bvh, light, 1, 0, g, 8, B, out=out,
                                              stream=st), flush, stream, 100)["ms"]
    return res


def uhd_frame(occ, flush, stream) -> dict:
    """The 4K configuration: ~4M-triangle scene (1024^2 heightfield, 1,200 spheres, 30,000
    boxes, seed 4), 3840 x 2160, packed G-buffer and records, K = 16 in 4x4 groups and in a
    16-member disk (window tuning picked by the autotuner), AO and shadows."""
    import tempfile

    import torch

    import synth
    from paper_2607_23122_gb300 import autotune
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = occ.Context(dev.index)
    t0 = time.perf_counter()
    scene = synth.scene_terrain(grid=1024, n_spheres=1200, n_boxes=30000, seed=4)
    bvh = occ.BVH(ctx, scene.tris)
    build_s = time.perf_counter() - t0
    Wu, Hu = 3840, 2160
    P = Wu * Hu
    gb = occ.occ_gbuffer_pinhole(ctx, bvh, synth.camera_c2().as_array(), scene.eps, Wu, Hu,
                                 packed=True)
    rec = occ.Occluders.empty(Hu, Wu, dev, packed=True)
    out = torch.empty((Hu, Wu), dtype=torch.float32, device=dev)
    light = synth.light_c3().as_array()
    g16 = occ.Pattern.group(4, 4)
    d16 = occ.Pattern.offsets_of(synth.disk_offsets(16, 15.0, seed=3))
    res = {"W": Wu, "H": Hu, "tris": scene.num_tris, "scene_and_bvh_s": build_s,
           "formats": "packed G-buffer and records (16 + 16 B/px)"}
    old_cache = os.environ.get("OCC_TUNE_CACHE")
    with tempfile.TemporaryDirectory() as tmp:
        os.environ["OCC_TUNE_CACHE"] = os.path.join(tmp, "tuning.json")
        try:
            for name, eff in (("ao", occ.OCC_EFFECT_AO), ("shadow", occ.OCC_EFFECT_SHADOW)):
                if eff == occ.OCC_EFFECT_AO:
                    def trace(st):
                        occ.occ_trace_ao(ctx, gb, bvh, RADIUS, 1, 0, out=rec, stream=st)
                    fn = occ.occ_reuse_ao
                else:
                    def trace(st):
                        occ.occ_trace_shadow(ctx, gb, bvh, light, 1, 0, out=rec, stream=st)
                    fn = occ.occ_reuse_shadow
                tr = time_kernel(trace, flush, stream, 30)["ms"]
                trace(stream)
                ctx.sync()
                tuned = autotune.tune_reuse(ctx, gb, rec, d16, occ.OCC_EST_BIASED, out,
                                            use_cache=False)
                gr = time_kernel(lambda st: fn(ctx, gb, rec, g16, 16, occ.OCC_EST_BIASED, out=out,
                                               stream=st), flush, stream, 30)["ms"]
                dk = time_kernel(lambda st: fn(ctx, gb, rec, d16, 16, occ.OCC_EST_BIASED, out=out,
                                               stream=st), flush, stream, 30)["ms"]
                occ.occ_set_tuning(ctx)
                res[name] = {"trace_ms": tr, "reuse_group4x4_ms": gr, "reuse_disk16_ms": dk,
                             "disk16_tuning": tuned["best"],
                             "ms_per_frame_group4x4": tr + gr, "ms_per_frame_disk16": tr + dk,
                             "neighbour_samples_per_s_group4x4": P * 16 / ((tr + gr) * 1e-3),
                             "neighbour_samples_per_s_disk16": P * 16 / ((tr + dk) * 1e-3)}
        finally:
            if old_cache is None:
                os.environ.pop("OCC_TUNE_CACHE", None)
            else:
                os.environ["OCC_TUNE_CACHE"] = old_cache
    ctx.sync()
    return res


# frames in flight in the end-to-end leg (1080p: 1 -> 0.90 ms, 2 -> 0.62, 3 -> 0.51,
# 4 -> 0.57 ms per frame)
E2E_DEPTH = 3
PACKED_GROUP_BYTES_PER_PX = 30   # x 12, octahedral n 4, offsets 6, octahedral n_z 4, out 4


def packed_frame(occ, ctx, gb, bvh, pat, out, flush, stream) -> dict:
    """The same AO frame with packed G-buffer and records (16 + 16 bytes per pixel)."""
    pgb = occ.occ_pack_gbuffer(ctx, gb)
    prec = occ.Occluders.empty(H, W, gb.pos4.device, packed=True)
    tr = time_kernel(lambda st: occ.occ_trace_ao(ctx, pgb, bvh, RADIUS, 1, 0, out=prec, stream=st),
                     flush, stream, 100)
    ru = time_kernel(lambda st: occ.occ_reuse_ao(ctx, pgb, prec, pat, K, occ.OCC_EST_BIASED,
                                                 out=out, stream=st), flush, stream, 100)
    gr = time_kernel(lambda st: occ.occ_reuse_ao(ctx, pgb, prec, occ.Pattern.group(4, 2), 8,
                                                 occ.OCC_EST_BIASED, out=out, stream=st),
                     flush, stream, 100)
    return {"trace_ms": tr["ms"], "reuse_offsets_k8_ms": ru["ms"], "reuse_group4x2_ms": gr["ms"],
            "ms_per_frame": tr["ms"] + ru["ms"], "bytes_per_px_stored": 16 + 16 + 4}


def quality_leg(occ, ctx, gb, bvh, pat) -> dict:
    """Equal-time RelMSE (eps 1e-3) against a 4096-spp no-reuse reference on this frame:
    AO at 2 ms and area-light shadows at 5 ms per image, the paper's 1080p budgets."""
    import synth

    from paper_2607_23122_gb300 import quality as Q
    light = synth.light_c3().as_array()
    out = {"reference": "no-reuse mean over 4096 spp (samples 0..4095); estimates use "
                        "independent samples; frames per method = floor(budget / frame time)"}
    for eff, budget, key in ((occ.OCC_EFFECT_AO, 2.0, "ao_2ms"), (occ.OCC_EFFECT_SHADOW, 5.0, "shadow_5ms")):
        ref = Q.reference(ctx, gb, bvh, eff, radius=RADIUS, light=light, spp=4096)
        out[key] = Q.equal_time(ctx, gb, bvh, eff, budget, ref, radius=RADIUS, light=light,
                                extra=[("Occ(8) disk", pat, occ.OCC_EST_BIASED),
                                       ("Occ(8)U", occ.Pattern.group(4, 2), occ.OCC_EST_UNBIASED)]
                                + ([("Light(8U)", occ.Pattern.group(4, 2), occ.OCC_EST_LIGHT_UNBIASED)]
                                   if eff == occ.OCC_EFFECT_SHADOW else []))
    return out


SERVE_RES = [(640, 360), (1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)]


def serving_mix(n: int, seed: int = 5) -> list:
    """The request mix: resolution uniform over SERVE_RES, AO / shadow 50/50, K uniform in
    {4, 8, 16} (groups 2x2, 15-px disk offsets, groups 4x4), one of 8 preset cameras."""
    rng = np.random.default_rng(seed)
    return [(SERVE_RES[int(rng.integers(5))], int(rng.random() < 0.5), (4, 8, 16)[int(rng.integers(3))],
             int(rng.integers(8))) for _ in range(n)]


class _OutPool:
    """Pinned host output buffers by resolution, recycled when their request completes."""

    def __init__(self):
        self.free, self.lock = {}, threading.Lock()

    def take(self, w, h):
        import torch
        with self.lock:
            lst = self.free.setdefault((w, h), [])
            if lst:
                return lst.pop()
        return torch.empty((h, w), dtype=torch.float32, pin_memory=True)

    def give(self, t):
        with self.lock:
            self.free.setdefault((t.shape[1], t.shape[0]), []).append(t)


def serving(occ, ctx, bvh, scene, n_req: int) -> dict:
    """Continuous-batching serving loop on the request mix, FP32 and packed formats, with
    the G-buffer either rendered on the device per request ("device_gbuffer") or sent from
    pinned host memory by the client ("host_gbuffer": 32 B/px FP32, 16 B/px packed,
    copied inside the request).  Per mode: the saturated rate of each format (median of
    3 bursts of n_req requests after one untimed burst), then Poisson arrivals of 4 n_req
    requests at 0.8x the slowest burst of either format (same arrival times for both); for
    the device mode also a saturated run under a 2 GB budget (admission by memory).
    Latency = submit -> estimate in pinned host memory, on the server's own clock."""
    import torch

    import synth
    n_poi = 4 * n_req
    mix = serving_mix(n_poi)
    cams = [c.as_array() for c in synth.serving_views(8)]
    light = synth.light_c3().as_array()
    pats = {4: occ.Pattern.group(2, 2), 8: occ.Pattern.offsets_of(synth.disk_offsets(8, DISK_R, 3)),
            16: occ.Pattern.group(4, 4)}
    pool = _OutPool()
    px = [w * h for (w, h), _, _, _ in mix]
    # client-side G-buffers (4 of the cameras x 5 resolutions), rendered once
    host_gb = {}
    for c in range(4):
        for (w, h) in SERVE_RES:
            g = occ.occ_gbuffer_pinhole(ctx, bvh, cams[c], scene.eps, w, h)
            gp = occ.occ_gbuffer_pinhole(ctx, bvh, cams[c], scene.eps, w, h, packed=True)
            ctx.sync()
            host_gb[(c, w, h)] = (g.pos4.cpu().pin_memory(), g.nrm4.cpu().pin_memory(),
                                  gp.pos4.cpu().pin_memory())
            del g, gp

    def run(srv, idx, packed, host, gaps=None):
        res, outs, lock, stop = {}, {}, threading.Lock(), threading.Event()

        def collect():
            while not stop.is_set() or len(res) < len(idx):
                for r in srv.poll(timeout_us=5000):
                    with lock:
                        res[r["id"]] = r
                        pool.give(outs.pop(r["id"]))

        th = threading.Thread(target=collect, daemon=True)
        th.start()
        due = time.perf_counter()
        for n, i in enumerate(idx):
            if gaps is not None:
                due += gaps[n]
                while True:
                    left = due - time.perf_counter()
                    if left <= 0:
                        break
                    time.sleep(left if left > 2e-4 else 0)
            (w, h), eff, k, c = mix[i]
            o = pool.take(w, h)
            kw = {}
            if host:
                pos, nrm, ppos = host_gb[(c % 4, w, h)]
                kw = {"pos4_host": ppos} if packed else {"pos4_host": pos, "nrm4_host": nrm}
            else:
                kw = {"camera": cams[c], "eps": scene.eps}
            with lock:
                rid = srv.submit(w, h, eff, pats[k], occ.OCC_EST_BIASED, o, radius=RADIUS,
                                 light=light if eff else None, seed=9, sample=i, packed=packed, **kw)
                outs[rid] = o
        stop.set()
        th.join(timeout=600)
        t_first = min(r["t_submit_ns"] for r in res.values())
        lat = np.array([r["t_done_ns"] - r["t_submit_ns"] for r in res.values()]) * 1e-6
        span = (max(r["t_done_ns"] for r in res.values()) - t_first) * 1e-9
        return {"requests": len(idx), "requests_per_s": len(idx) / span,
                "Mpx_per_s": sum(px[i] for i in idx) / span / 1e6,
                "p50_ms": float(np.median(lat)), "p99_ms": float(np.quantile(lat, 0.99)),
                "mean_batch_views": float(np.mean([r["batch_views"] for r in res.values()])),
                "all_ok": all(r["status"] == 0 for r in res.values())}

    out = {"mix": "640x360..3840x2160 uniform, AO/shadow 50/50, K in {4 (group 2x2), "
                  "8 (15-px disk), 16 (group 4x4)}, 8 cameras, biased; estimate copied to "
                  "pinned host memory"}
    for mode in ("device_gbuffer", "host_gbuffer"):
        host = mode == "host_gbuffer"
        m = {}
        servers = {}
        for packed in (False, True):
            srv = occ.Server(ctx, bvh, max_views_per_batch=32, max_inflight=2)
            # warm-up: a whole burst, so that the server's memory pool has grown to the
            # mix's working set before the timed bursts
            run(srv, list(range(n_req)), packed, host)
            bursts = [run(srv, list(range(n_req)), packed, host) for _ in range(3)]
            bursts.sort(key=lambda b: b["requests_per_s"])
            m["packed" if packed else "fp32"] = {"saturated": bursts[1],
                                                 "saturated_runs_req_s": [b["requests_per_s"] for b in bursts]}
            servers[packed] = srv
        # 0.8x the slower format's slowest burst: bursts of the same requests vary by up to
        # ~1.6x on this host (submission thread, pinned copies), and a rate above the
        # sustained one measures queue growth, not latency
        rate = 0.8 * min(min(m["fp32"]["saturated_runs_req_s"]),
                         min(m["packed"]["saturated_runs_req_s"]))
        gaps = np.random.default_rng(55).exponential(1.0 / rate, size=n_poi)
        for packed in (False, True):
            srv = servers[packed]
            key = "packed" if packed else "fp32"
            m[key]["poisson"] = run(srv, list(range(n_poi)), packed, host, gaps)
            st = srv.stats()
            m[key]["peak_reserved_MB"] = st["peak_reserved_bytes"] / 2**20
            m[key]["views_batched"], m[key]["views_single"] = st["views_batched"], st["views_single"]
            srv.close()
            if not host:
                srv = occ.Server(ctx, bvh, budget_bytes=2 << 30, max_views_per_batch=32,
                                 max_inflight=2)
                small = run(srv, list(range(n_req)), packed, host)
                m[key]["budget_2GB_saturated"] = dict(
                    small, peak_reserved_MB=srv.stats()["peak_reserved_bytes"] / 2**20)
                srv.close()
        m["poisson_rate_req_s"] = rate
        out[mode] = m
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2607_23122_gb300 import occ

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = occ.Context(local)
    scene, cam, offs = scene_inputs()
    bvh = occ.BVH(ctx, scene.tris)
    gb = occ.occ_gbuffer_pinhole(ctx, bvh, cam.as_array(), scene.eps, W, H)
    ctx.sync()
    pat = occ.Pattern.offsets_of(offs)
    rec = occ.Occluders.empty(H, W, dev)
    out = torch.empty((H, W), dtype=torch.float32, device=dev)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()

    def step():
        occ.occ_trace_ao(ctx, gb, bvh, RADIUS, 1, 0, out=rec, stream=stream)
        occ.occ_reuse_ao(ctx, gb, rec, pat, K, occ.OCC_EST_BIASED, out=out, stream=stream)

    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        flush.zero_()
        step()
    ctx.sync()
    P = W * H
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()                        # L2 flush outside the step's events
        ev[i][0].record(stream)
        occ.occ_trace_ao(ctx, gb, bvh, RADIUS, 1, i, out=rec, stream=stream)
        ev[i][1].record(stream)
        occ.occ_reuse_ao(ctx, gb, rec, pat, K, occ.OCC_EST_BIASED, out=out, stream=stream)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    ctx.sync()
    t_trace = np.array([ev[i][0].elapsed_time(ev[i][1]) for i in range(args.steps)]) * 1e-3
    t_reuse = np.array([ev[i][1].elapsed_time(ev[i][2]) for i in range(args.steps)]) * 1e-3
    t_step = max_over_ranks(float((t_trace + t_reuse).sum()), dev)
    t_reuse_all = max_over_ranks(float(t_reuse.sum()), dev)
    value = job_throughput(world, P * K, args.steps, t_reuse_all)

    # end to end through the C ABI with host buffers (pinned), copies inside the region:
    # every frame uploads its G-buffer and downloads its estimate.  Pipelined: E2E_DEPTH
    # frames in flight (one context and one stream each), so the copies of some frames overlap
    # the kernels of another; serial: occ_frame_host, one frame at a time.
    pos_h = gb.pos4.cpu().pin_memory()
    nrm_h = gb.nrm4.cpu().pin_memory()
    outs_h = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(E2E_DEPTH)]
    e2e_steps = max(3, args.steps // 2)
    ctxs = [ctx] + [occ.Context(local) for _ in range(E2E_DEPTH - 1)]
    streams = [torch.cuda.Stream(dev) for _ in range(E2E_DEPTH)]

    def e2e_pipelined(n):
        for i in range(n):
            j = i % E2E_DEPTH
            if i >= E2E_DEPTH:
                ctxs[j].sync(streams[j])         # frame i - E2E_DEPTH done: its context is free
            occ.occ_frame_host_async(ctxs[j], bvh, occ.OCC_EFFECT_AO, pos_h, nrm_h, RADIUS, None,
                                     1, i, pat, K, occ.OCC_EST_BIASED, outs_h[j], stream=streams[j])
        for j in range(E2E_DEPTH):
            ctxs[j].sync(streams[j])

    e2e_pipelined(4)
    for i in range(2):
        occ.occ_frame_host(ctx, bvh, occ.OCC_EFFECT_AO, pos_h, nrm_h, RADIUS, None, 1, i, pat, K,
                           occ.OCC_EST_BIASED, outs_h[0], stream=stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_pipelined(e2e_steps)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0, dev)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        occ.occ_frame_host(ctx, bvh, occ.OCC_EFFECT_AO, pos_h, nrm_h, RADIUS, None, 1, i, pat, K,
                           occ.OCC_EST_BIASED, outs_h[0], stream=stream)
    torch.cuda.synchronize()
    t_e2e_serial = max_over_ranks(time.perf_counter() - t0, dev)

    # the paper's own layout: 4x2 shared groups (K = 8) on warp lanes, HBM bound
    extra = {}
    if rank == 0:
        g42 = occ.Pattern.group(4, 2)
        extra["reuse_group4x2"] = time_kernel(
            lambda st: occ.occ_reuse_ao(ctx, gb, rec, g42, 8, occ.OCC_EST_BIASED, out=out,
                                        stream=st), flush, stream, 200)
        # the group kernel's L2 prefetch choices (tuning group_prefetch 1 / 2 / 3)
        pf = {}
        try:
            for c in (1, 2, 3):
                occ.occ_set_tuning(ctx, group_prefetch=c)
                pf[c] = time_kernel(lambda st: occ.occ_reuse_ao(ctx, gb, rec, g42, 8,
                                                                occ.OCC_EST_BIASED, out=out,
                                                                stream=st), flush, stream, 200)
        finally:
            occ.occ_set_tuning(ctx)
        extra["reuse_group4x2"]["prefetch_choices_ms"] = {
            {1: "none", 2: "gbuffer+rec0", 3: "gbuffer+rec0+rec1"}[c]: v["ms"] for c, v in pf.items()}
        # the same loads and stores with no arithmetic: what the kernel's bytes cost alone
        extra["reuse_group4x2"]["stream_ceiling"] = time_kernel(
            lambda st: occ.occ_debug_stream_ceiling(ctx, gb, rec, out, stream=st), flush, stream, 200)
        # the trace's launch choices on this frame (autotuner candidates, bit-identical records)
        from paper_2607_23122_gb300 import autotune
        tt = autotune.tune_trace(ctx, gb, bvh, occ.OCC_EFFECT_AO, rec, radius=RADIUS, iters=10,
                                 use_cache=False)
        occ.occ_set_tuning(ctx)
        extra["trace_tuning"] = {"best": tt["best"],
                                 "ms": {json.dumps(t["config"], sort_keys=True): t["ms"]
                                        for t in tt["timings"]}}
        # the G-buffer layout (row-major or 8 x 8 tiles in Morton order), per frame
        lay = {}
        for pname, lpat in (("group4x2", occ.Pattern.group(4, 2)), ("disk8", pat)):
            lt = autotune.tune_layout(ctx, gb, bvh, occ.OCC_EFFECT_AO, lpat, occ.OCC_EST_BIASED,
                                      rec, out, radius=RADIUS, iters=20, use_cache=False)
            lay[pname] = {"best": lt["best"]["gbuffer_layout"],
                          "frame_ms": {t["config"]["gbuffer_layout"]: t["ms"] for t in lt["timings"]}}
        extra["layout_tuning"] = lay
        extra["shadow"] = shadow_frame(occ, ctx, gb, bvh, pat, rec, out, flush, stream)
        extra["packed"] = packed_frame(occ, ctx, gb, bvh, pat, out, flush, stream)
        extra["fused"] = fused_frame(occ, ctx, gb, bvh, rec, out, flush, stream)
        # serving before the 4K and quality legs: their large allocations made the saturated
        # bursts vary by up to 1.6x when they ran first
        if not args.no_serving:
            extra["serving"] = serving(occ, ctx, bvh, scene, args.serve_requests)
        if not args.no_uhd:
            extra["uhd"] = uhd_frame(occ, flush, stream)
        if not args.no_quality:
            extra["quality"] = quality_leg(occ, ctx, gb, bvh, pat)

    if rank == 0:
        fp32 = fp32_peak(occ, ctx, dev, stream)
        hbm, peak_kind, peaks = measured_peaks()
        st = bvh.stats
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        tr, ru = float(t_trace.mean()), float(t_reuse.mean())
        # trace: compulsory bytes = G-buffer read + record write + the distinct BVH nodes and
        # triangles the traversal touches (instrumented-library count)
        trace_bytes = P * (32 + 32) + TRACE_TOUCH["distinct_bytes"]
        # reuse (offset window, K^2 pair densities): FP32 ALU bound
        pairs = P * K * K
        issue_mhz = clk["sm_max_mhz"] or peaks.get("sm_max_mhz", 2070.0)
        alu_peak = fp32["peak"] * 1e12
        # the trace is bound by instruction issue and dependent-fetch latency, not by bytes:
        # its roofline is the warp-instruction issue rate (4 schedulers per SM, one warp
        # instruction per cycle each, at the max SM clock), with the byte roofline beside it
        issue_peak = sms * 4 * issue_mhz * 1e6
        winstr = NCU_TRACE_WARP_INSTR
        trace_roof = {"kernel": "k_trace_dyn<AO>", "bound": "alu",
                      "achieved": winstr / tr / 1e9 if winstr else None, "peak": issue_peak / 1e9,
                      "unit": "G warp-instructions/s",
                      "frac": winstr / tr / issue_peak if winstr else None,
                      "traffic": NCU_TRAFFIC["k_trace_dyn<AO>"],
                      "peak_source": f"{sms} SMs x 4 schedulers x 1 warp-instruction per cycle x "
                                     f"{issue_mhz:.0f} MHz max SM clock",
                      "algorithmic": ("warp instructions per launch (ncu smsp__inst_executed.sum "
                                      f"{winstr:.4g}); issue slots "
                                      f"{NCU_TRACE_ISSUE_ACTIVE:.0%} busy under ncu") if winstr
                                     else "warp instructions per launch: not captured for this build",
                      "hbm": {"algorithmic_bytes": trace_bytes, "achieved": trace_bytes / tr / 1e9,
                              "peak": hbm, "unit": "GB/s", "frac": trace_bytes / tr / 1e9 / hbm,
                              "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                              "bytes": "G-buffer 32 B/px + records 32 B/px + distinct BVH bytes "
                                       f"touched {TRACE_TOUCH['distinct_bytes']} (of "
                                       f"{st['bytes']})"},
                      "traversal": {k: TRACE_TOUCH[k] / TRACE_TOUCH["rays"]
                                    for k in ("node_visits", "triangle_tests")}}
        reuse_roof = {"kernel": "k_reuse_tile<AO,8> (TMA-staged window)", "bound": "alu",
                      "achieved": pairs * FLOPS_PER_PAIR_AO / ru / 1e12,
                      "peak": alu_peak / 1e12, "unit": "TFLOP/s",
                      "frac": pairs * FLOPS_PER_PAIR_AO / ru / alu_peak,
                      "traffic": NCU_TRAFFIC["k_reuse_tile<AO,8>"],
                      "peak_source": "measured: FP32 FMA-chain probe (fp32_peak)"}
        dominant = trace_roof if tr >= ru else reuse_roof
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_step / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(world, scene.num_tris),
            "frame_neighbour_samples_per_s": job_throughput(world, P * K, args.steps, t_step),
            "reuse_pass": {"neighbour_samples_per_s": P * K / ru, "ms": ru * 1e3},
            "trace_pass": {"rays_per_s": P / tr, "ms": tr * 1e3},
            "fp32_peak": fp32,
            "roofline": dominant, "roofline_other": reuse_roof if dominant is trace_roof else trace_roof,
            "e2e": {"value": job_throughput(world, P * K, e2e_steps, t_e2e), "unit": UNIT,
                    "h2d_bytes_per_step": 2 * 16 * P, "d2h_bytes_per_step": 4 * P,
                    "ms_per_step": t_e2e / e2e_steps * 1e3,
                    "api": f"occ_frame_host_async, {E2E_DEPTH} frames in flight (a context and a "
                           "stream each)",
                    "serial": {"value": job_throughput(world, P * K, e2e_steps, t_e2e_serial),
                               "ms_per_step": t_e2e_serial / e2e_steps * 1e3,
                               "api": "occ_frame_host, one frame at a time"}},
            "gpu_launches": 2 * args.steps,
            "clocks": clk, "wall_s": wall,
            "reuse_group4x2": dict(extra["reuse_group4x2"], kernel="k_reuse_group<AO,biased,4,2>",
                                   traffic=NCU_TRAFFIC["k_reuse_group<AO,biased,4,2>"],
                                   algorithmic_bytes=P * GROUP_BYTES_PER_PX,
                                   achieved_gbs=P * GROUP_BYTES_PER_PX / extra["reuse_group4x2"]["s"] / 1e9,
                                   frac_hbm=P * GROUP_BYTES_PER_PX / extra["reuse_group4x2"]["s"] / 1e9 / hbm,
                                   neighbour_samples_per_s=P * 8 / extra["reuse_group4x2"]["s"]),
            "trace_tuning_ao": extra["trace_tuning"],
            "layout_tuning_ao": extra["layout_tuning"],
            "shadow_frame": extra["shadow"],
            "packed_frame": dict(extra["packed"],
                                 group_frac_hbm=P * PACKED_GROUP_BYTES_PER_PX
                                 / (extra["packed"]["reuse_group4x2_ms"] * 1e-3) / 1e9 / hbm),
            "fused_group4x2_frame": extra["fused"],
            "bvh": {"nodes": st["num_nodes"], "depth": st["depth"], "bytes": st["bytes"],
                    "build_s": st["build_seconds"]},
        }
        if "uhd" in extra:
            line["uhd_packed_k16_frame"] = extra["uhd"]
        for key in ("quality", "serving"):
            if key in extra:
                line[key] = extra[key]
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(scene, cam, offs)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ----------------------------------------------------------------------------------------
# reference arm: the FP64 oracle
# ----------------------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    scene, cam, offs = scene_inputs()
    osc = oracle.OracleScene(scene.tris)
    pos, nrm, _ = oracle.gbuffer(osc, cam.as_array(), W, H, scene.eps)
    rec = np.zeros((H, W, 8))
    rec[..., 7] = -1.0
    mg = np.full((H, W), np.inf)
    out = np.zeros((H, W))
    omg = np.zeros((H, W))
    pat = (2, 0, 0, offs)
    hx0, hx1 = max(0, -offs[:, 0].min()), max(0, offs[:, 0].max())
    hy0, hy1 = max(0, -offs[:, 1].min()), max(0, offs[:, 1].max())
    B = 32
    rng = np.random.default_rng(5)

    t_reuse = [0.0]

    def step(i):
        x0 = int(rng.integers(hx0, W - B - hx1))
        y0 = int(rng.integers(hy0, H - B - hy1))
        oracle.trace(osc, 0, pos, nrm, radius=RADIUS, seed=1, sample=i,
                     region=(x0 - hx0, y0 - hy0, B + hx0 + hx1, B + hy0 + hy1), out=(rec, mg))
        t1 = time.perf_counter()
        oracle.reuse(None, 0, pos, nrm, rec, pat, oracle.EST_BIASED, radius=RADIUS,
                     region=(x0, y0, B, B), out=(out, omg))
        t_reuse[0] += time.perf_counter() - t1

    for i in range(args.warmup):
        step(i)
    t_reuse[0] = 0.0
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    t = time.perf_counter() - t0
    # the same metric as the GPU arm: neighbour-samples over the reuse time; the frame rate
    # (trace + reuse) beside it
    value = B * B * K * args.steps / t_reuse[0]
    sample = (f"each step: one random {B}x{B} receiver block of the 1080p frame, traced with "
              f"its {hx0}/{hx1}/{hy0}/{hy1}-px halo, then biased K=8 reuse")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": bench_config(world, scene.num_tris),
        "frame_neighbour_samples_per_s": B * B * K * args.steps / t,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def count_touch():
    """Traversal counters of the 1080p AO trace (the bench step's) and shadow trace, from the
    instrumented library: node visits and triangle tests per ray, and the distinct nodes and
    triangles touched (their bytes are the BVH part of the trace's compulsory traffic)."""
    from paper_2607_23122_gb300 import _native
    if _native.variant() != "counters":
        raise SystemExit("--count-touch needs OCC_LIB_VARIANT=counters")
    import synth
    from paper_2607_23122_gb300 import occ
    ctx = occ.Context(0)
    scene, cam, _ = scene_inputs()
    bvh = occ.BVH(ctx, scene.tris)
    gb = occ.occ_gbuffer_pinhole(ctx, bvh, cam.as_array(), scene.eps, W, H)
    rec = occ.Occluders.empty(H, W, gb.pos4.device)
    ctx.sync()
    occ.occ_debug_bvh_counters(ctx, bvh, reset=True)
    res = {"bvh_bytes": bvh.stats["bytes"], "bvh_nodes": bvh.stats["num_nodes"], "tris": scene.num_tris}
    valid = int((gb.pos4[..., 3] != 0).sum())
    for name, fn in (("ao", lambda: occ.occ_trace_ao(ctx, gb, bvh, RADIUS, 1, 0, out=rec)),
                     ("shadow", lambda: occ.occ_trace_shadow(ctx, gb, bvh, synth.light_c3().as_array(),
                                                             1, 0, out=rec))):
        fn()
        ctx.sync()
        c = occ.occ_debug_bvh_counters(ctx, bvh, reset=True)
        c["rays"] = valid
        c["node_visits_per_ray"] = c["node_visits"] / valid
        c["triangle_tests_per_ray"] = c["triangle_tests"] / valid
        res[name] = c
    print(json.dumps(res), flush=True)


def profile_step():
    """One launch of each hot kernel on the 1080p AO frame, untimed (ncu captures)."""
    import torch

    import synth
    from paper_2607_23122_gb300 import occ
    ctx = occ.Context(0)
    scene, cam, offs = scene_inputs()
    bvh = occ.BVH(ctx, scene.tris)
    gb = occ.occ_gbuffer_pinhole(ctx, bvh, cam.as_array(), scene.eps, W, H)
    rec = occ.Occluders.empty(H, W, gb.pos4.device)
    out = torch.empty((H, W), dtype=torch.float32, device=gb.pos4.device)
    occ.occ_trace_ao(ctx, gb, bvh, RADIUS, 1, 0, out=rec)
    occ.occ_reuse_ao(ctx, gb, rec, occ.Pattern.offsets_of(offs), K, occ.OCC_EST_BIASED, out=out)
    occ.occ_reuse_ao(ctx, gb, rec, occ.Pattern.group(4, 2), 8, occ.OCC_EST_BIASED, out=out)
    occ.occ_trace_shadow(ctx, gb, bvh, synth.light_c3().as_array(), 1, 0, out=rec)
    occ.occ_trace_reuse_ao(ctx, gb, bvh, RADIUS, 1, 0, occ.Pattern.group(4, 2), 8,
                           occ.OCC_EST_BIASED, out=out)
    occ.occ_trace_reuse_shadow(ctx, gb, bvh, synth.light_c3().as_array(), 1, 0,
                               occ.Pattern.group(4, 2), 8, occ.OCC_EST_BIASED, out=out)
    # unbiased 4x2 groups on the AO records: collect pass, k_validate, final pass
    occ.occ_trace_ao(ctx, gb, bvh, RADIUS, 1, 0, out=rec)
    occ.occ_reuse_ao(ctx, gb, rec, occ.Pattern.group(4, 2), 8, occ.OCC_EST_UNBIASED, bvh=bvh, out=out)
    ctx.sync()
    print(json.dumps({"profile_step": "ok", "checksum": float(out.double().sum())}))


def main():
    args = parse()
    if args.profile_step:
        profile_step()
        return
    if args.count_touch:
        count_touch()
        return
    _, world, _ = dist_env()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(relaunch_as_ranks(args.gpus))
    if world != args.gpus:
        raise SystemExit(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={world}")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
