#!/usr/bin/env python3
"""Throughput of the neural visibility cache hot path on synthetic frames.

One step = one frame of the 1080p workload: an online training step (8192
positions x 32 shadow rays against 64 occluders, forward, loss, backward,
Adam over all 16.8M parameters) followed by inference + WRS + Neural DI of
all 1920x1080 pixels, replayed as one CUDA graph.  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank renders and trains its own view (weak
scaling, no data-path collective); rank 0 prints the max-over-ranks time.
--impl reference times the CPU oracle (float64 numpy) on a bounded sample
of the same frame, extrapolated to the whole frame.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("Mpixels/s encode+MLP+WRS and ms/frame incl. train step at 1080p/32 lights; "
          "% roofline")
WORKLOAD = "frame_1080p"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, help="override the inference precision")
    ap.add_argument("--pretrain", type=int, default=500)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return dict(hbm=p["hbm_gbs"], bf16=p["bf16_tflops"],
                    bf16_sustained=p["bf16_tflops_sustained"], src="measured")
    except Exception:
        return dict(hbm=6800.0, bf16=1900.0, bf16_sustained=1700.0, src="fallback")


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region:
    sampled every 10 ms with nvidia-smi's own timestamps; `ready` waits for
    the first sample, `begin` / `stop` bracket the region on the host clock.
    The samples inside the region are kept; a region shorter than the
    sampling interval keeps the last sample before it and the first after
    it instead (`window` says which)."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int, interval_ms: int = 10):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.t0 = self.t1 = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(gpu_index), "-lms", str(interval_ms)],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def ready(self, timeout_s: float = 5.0):
        end = time.time() + timeout_s
        while self.p is not None and time.time() < end:
            if os.path.getsize(self.f.name) > 0:
                return
            time.sleep(0.02)

    def begin(self):
        self.t0 = time.time()

    @classmethod
    def parse(cls, text):
        """(timestamp, sm MHz, max MHz, active reasons) per sample line."""
        rows = []
        for line in text.splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(c[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                sm, mx = float(c[2]), float(c[3])
            except ValueError:
                continue
            reasons = {n for n, v in zip(cls.NAMES, c[6:10]) if v.lower().startswith("active")}
            rows.append((ts, sm, mx, reasons))
        return rows

    @staticmethod
    def summarise(rows, t0, t1):
        inside = [r for r in rows if t0 <= r[0] <= t1]
        window = "inside"
        if not inside:
            before = [r for r in rows if r[0] < t0]
            after = [r for r in rows if r[0] > t1]
            inside = before[-1:] + after[:1]
            window = "edges"
        if not inside:
            return None
        reasons = set().union(*(r[3] for r in inside))
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": inside[-1][2],
                "reasons": sorted(reasons), "samples": len(inside), "window": window}

    def stop(self):
        self.t1 = time.time()
        if self.p is None:
            return None
        time.sleep(0.05)                 # let the sample after the end land
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = self.parse(self.f.read())
        os.unlink(self.f.name)
        return self.summarise(rows, self.t0, self.t1)


# ------------------------------------------------------- multi-rank logic --

def rank_stream(rank: int):
    """Seed and view id of a rank: every rank renders and trains its own
    view (weak scaling), so their random streams must differ."""
    return 1234 + rank, rank


def max_over_ranks(x: float, device) -> float:
    """The slowest rank's time (a no-op on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, pixels_per_rank: int, ms_per_frame: float) -> float:
    """Whole-job Mpixels/s: all ranks' pixels over the slowest rank's frame time."""
    return world * pixels_per_rank / (ms_per_frame * 1e-3) / 1e6


# --------------------------------------------------------------- workload --

_WORKLOAD_CACHE = {}


def workload(precision=None):
    import nvc_synth as S
    if "base" not in _WORKLOAD_CACHE:
        cfg = S.config_by_name(WORKLOAD)
        sc = S.scene_heightfield(seed=1, n_lights=32, n_spheres=32, n_boxes=32)
        gb = S.gbuffer_heightfield(seed=1, width=1920, height=1080)
        _WORKLOAD_CACHE["base"] = (cfg, sc, gb)
    cfg, sc, gb = _WORKLOAD_CACHE["base"]
    if precision:
        cfg = cfg.with_(precision=precision)
    return cfg, sc, gb


def workload_config(world, pixels_per_gpu, positions_per_frame):
    """The bench line's `config`, the same for both arms."""
    return {"workload": "frame_1080p: 1920x1080 heightfield+boxes view, 32 point lights, "
                        "32 spheres + 32 boxes; hash grid 16 levels x 2 features x 2^19 (FP32 "
                        "master, FP16 copy for inference), MLP 32-64-64-64-32; training 8192 "
                        "positions x 32 lights per frame",
            "global_batch": world * pixels_per_gpu, "pixels_per_gpu": pixels_per_gpu,
            "train_positions_per_frame": positions_per_frame, "parallelism": f"replica{world}",
            "l2": "no flush: per-frame working set (G-buffer 50 MB, table+Adam state 270 MB) "
                  "exceeds L2"}


# Algorithmic work of one pixel, counted from the method's definition (each
# arithmetic operation once, a fused multiply-add as one):
#   normalise: 3 x (sub, div, two clamps)                                12
#   per level: cell 3 x (mul, floor, min, sub) 12; 1 - f 3; hash 2 mul +
#     3 add + 8 x (2 xor + and) 29; corner weights 12; blend 8 F; 8
#     addresses 8 (the 8 row loads are load/store-unit work, not counted) 64 + 8F
#   per hidden value: leaky ReLU 2 + conversion to the operand type 0.5  2.5
#   per light: sigmoid 4; contribution 15 (3 sub, two 3-term dots, rsqrt,
#     4 mul, clamp); weight 2; max / sum / Neural DI 3; reservoir 8
#     (quantise 3, running sum, mulhi, compare, 2 selects); Philox 10
#     (10 rounds x 4 ops per block of 4 lights)                          42
ALU_OPS = dict(normalise=12, level_base=64, level_per_feature=8, hidden_value=2.5, light=42)


def algorithmic(cfg, n_pixels):
    """Algorithmic work of the stages (the roofline numerators)."""
    F, Lv, L = cfg.n_features, cfg.n_levels, cfg.n_outputs
    dims = [cfg.n_inputs, *cfg.hidden, L]
    macs = sum(a * b for a, b in zip(dims[:-1], dims[1:]))
    n_table = cfg.n_levels * cfg.table_size * F
    n_params = n_table + macs
    # the half-precision feature copy the fused inference reads is rewritten
    # by the same Adam pass, 2 B per table parameter
    table16 = cfg.table_precision != "fp32" and cfg.precision != "fp32"
    alu_px = (ALU_OPS["normalise"]
              + Lv * (ALU_OPS["level_base"] + ALU_OPS["level_per_feature"] * F)
              + ALU_OPS["hidden_value"] * sum(cfg.hidden)
              + ALU_OPS["light"] * L)
    return dict(
        shade_alu_ops=alu_px * n_pixels,
        shade_flops=2.0 * macs * n_pixels,                  # MLP contraction
        shade_hbm_bytes=40.0 * n_pixels,                    # pos+nrm in, idx/pdf/wsum/DI out
        shade_gather_bytes=Lv * 8 * F * 4.0 * n_pixels,     # useful table bytes gathered
        # read theta,m,v,g; write theta,m,v; clear touched g; the FP16 copy
        adam_bytes=28.5 * n_params + (2.0 * n_table if table16 else 0.0),
        n_params=n_params, macs_per_px=macs, alu_ops_per_px=alu_px)


def alu_peak_ops(sm_mhz=2070.0, n_sms=152, lanes=128):
    """Peak ALU rate: every FP32/INT32 lane of every SM, one op per clock."""
    return n_sms * lanes * sm_mhz * 1e6


# Clustered sampler (Section 3.6), per pixel: per light a contribution (15)
# and its add to the cluster sum (1); per cluster weight 2, sum 1, reservoir
# 8, Philox 10; the RIS step: 4 candidates x (pick 2, contribution 15,
# reservoir 8), Philox 20, the contribution weight 8.
CLUSTER_OPS = dict(light=16, cluster=21, ris=128)


def clustered_alu_ops(n_lights, k, n_pixels):
    return (CLUSTER_OPS["light"] * n_lights + CLUSTER_OPS["cluster"] * k
            + CLUSTER_OPS["ris"]) * n_pixels


# Per-launch DRAM traffic of the dominant kernel from the ncu capture named in
# profiles/ (None once the kernel has changed since that capture); the fused
# shading kernel's by variant (the 1080p frame's launch).
KERNEL_TRAFFIC = {"fused_shade": {6: 78.75e6, 7: 83.04e6}, "adam": 460.4e6,
                  # 1080p launch with the shadow ray (light, W and estimate written)
                  "sample_clustered": 336.78e6}


# ------------------------------------------------------------- our arm ----

def measure_tiny(stream, use_graph):
    """The launch-bound tiny workload (64x64 points, 4 lights, FP32): one
    frame = a training step on 1024 positions x 4 lights, then inference,
    WRS and Neural DI of the 4096 points, as one captured CUDA graph.
    Reported in microseconds per frame (200 frames after 10 warm-up)."""
    import torch
    from paper_2506_05930_gb300 import nvc
    import nvc_synth as S
    cfg = S.config_by_name("tiny_fp32")
    sc = S.scene_unit_cube(seed=0)
    gb = S.gbuffer_points(0, 64, 64)
    cache = nvc.VisibilityCache(cfg)
    cache.set_params(S.init_params(cfg, seed=0))
    scene = nvc.Scene.from_synth(sc)
    n = gb.n
    view = nvc.View(torch.from_numpy(gb.pos).cuda(), torch.from_numpy(gb.nrm).cuda(), 0,
                    torch.empty(n, dtype=torch.int32, device="cuda"),
                    torch.empty(n, device="cuda"), torch.empty(n, device="cuda"),
                    torch.empty(n, device="cuda"))
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    for f in range(10):
        nvc.nvc_frame(cache.handle, scene, [view], 0, 3, f, loss, use_graph=use_graph)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for f in range(200):
        nvc.nvc_frame(cache.handle, scene, [view], 0, 3, 10 + f, loss, use_graph=use_graph)
    e1.record(stream)
    torch.cuda.synchronize()
    cache.close()
    return {"workload": "tiny_fp32: 64x64 points, 4 lights, 4 spheres; training 1024 "
                        "positions x 4 lights; FP32", "us_per_frame": e0.elapsed_time(e1) / 200 * 1e3,
            "cuda_graph": use_graph}


def measure_gather_peak(stream, table_mib=64, rows_per_thread=256, reps=7):
    """The random-row gather rate from an L2-resident table: the encode's
    roofline denominator (nvc_gather_bench: 8 independent row loads in
    flight per thread, rows of 8 and 16 bytes at uniformly random places of
    a 64 MiB float32 table, the size of the 1080p workload's master table).
    Two untimed launches bring the table into L2; the best of `reps` timed
    launches is reported, as useful bytes and as 32-byte L2 sectors."""
    import torch
    from paper_2506_05930_gb300 import nvc
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    table = torch.rand(table_mib * (1 << 20) // 4, device="cuda")
    n_threads = sms * 2048
    sink = torch.empty(n_threads, device="cuda")
    out = {"table_mib": table_mib, "threads": n_threads, "rows_per_thread": rows_per_thread}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for rb in (8, 16):
        for _ in range(2):
            nvc.nvc_gather_bench(table, rb, n_threads, rows_per_thread, sink, seed=1, stream=stream)
        best = None
        for r in range(reps):
            e0.record(stream)
            nvc.nvc_gather_bench(table, rb, n_threads, rows_per_thread, sink, seed=2 + r,
                                 stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        rows = n_threads * rows_per_thread
        out[f"row{rb}"] = {"ms": best, "useful_gbs": rows * rb / (best * 1e-3) / 1e9,
                           "sector_gbs": rows * 32 / (best * 1e-3) / 1e9,
                           "grows_per_s": rows / (best * 1e-3) / 1e9}
    del table
    return out


def measure_phases(cache, scene, pos, nrm, view, seed, frame, shade_ms, cfg, gather_peak,
                   pk, sm_mhz):
    """Where the fused shading kernel's time goes, by phase (nvc_shade_phases:
    SM-clock stamps at the phase boundaries of every tile), and the two
    per-phase rooflines this attributes: the encode's useful gather bytes
    over its share of the kernel time against the measured random-gather
    rate, and the MLP's flops over its share against the tensor peak.  The
    time attribution charges phase p with share_p x kernel time, share_p =
    the groups' summed cycles in p over their summed tile-loop cycles."""
    from paper_2506_05930_gb300 import nvc
    try:
        cyc = nvc.nvc_shade_phases(cache.handle, scene, pos, nrm, seed, frame, view.idx, view.pdf,
                                   view.wsum, view.radiance)
    except Exception as e:          # the chosen variant is not a tile-stream kernel
        return {"unavailable": str(e)}
    alg = algorithmic(cfg, pos.shape[0])
    total = cyc[3]
    share = {k: cyc[i] / total for i, k in enumerate(("encode", "mlp", "sampler"))}
    t = shade_ms * 1e-3
    enc_gbs = alg["shade_gather_bytes"] / (share["encode"] * t) / 1e9
    mlp_tf = alg["shade_flops"] / (share["mlp"] * t) / 1e12
    g8 = gather_peak["row8"]["useful_gbs"] if gather_peak else None
    # per-tile view of the MLP phase: a tile's tensor work at one SM's peak
    # over the mean wall time a tile spends in its MLP phase
    n_sms = 152
    tiles = -(-pos.shape[0] // 128)
    mlp_tile_s = cyc[1] / tiles / (sm_mhz * 1e6)
    tile_tensor_s = alg["shade_flops"] / tiles / (pk["bf16_sustained"] * 1e12 / n_sms)
    return {
        "cycles": {"encode": cyc[0], "mlp": cyc[1], "sampler": cyc[2], "tile_loop": cyc[3]},
        "share": share,
        "encode": {"useful_gather_gbs": enc_gbs, "l2_gather_peak_gbs": g8,
                   "frac_of_l2_gather": enc_gbs / g8 if g8 else None,
                   "gather_bytes_per_px": alg["shade_gather_bytes"] / pos.shape[0]},
        "mlp": {"tflops": mlp_tf, "peak_tflops": pk["bf16_sustained"],
                "frac_of_tensor_peak": mlp_tf / pk["bf16_sustained"],
                "per_tile_phase_us": mlp_tile_s * 1e6,
                "per_tile_tensor_us_at_sm_peak": tile_tensor_s * 1e6,
                "per_tile_frac": tile_tensor_s / mlp_tile_s},
        "note": "phase p is charged share_p x the kernel time; per_tile_frac = a tile's MLP "
                "flops at one SM's sustained tensor peak over the mean time a tile spends in "
                "its MLP phase (other tile streams of the SM run meanwhile)"}


def measure_mlp_only(cache, cfg, n_px, stream, pk):
    """The network alone on the tensor cores (nvc_mlp_infer_features: the
    shading point's tile-stream kernel with its encode replaced by a read of
    given layer-0 operands) over the frame's pixel count, random 16-bit
    operands (133 MB at 1080p, more than L2) and sigmoid visibilities out;
    flops over the CUDA-event time against the sustained tensor peak."""
    import torch
    from paper_2506_05930_gb300 import nvc
    k0 = (cfg.n_levels * cfg.n_features + 15) // 16 * 16
    dtype = torch.bfloat16 if cfg.precision == "bf16" else torch.float16
    g = torch.Generator(device="cuda").manual_seed(5)
    feat = (torch.rand((n_px, k0), device="cuda", generator=g) - 0.5).to(dtype)
    vis = torch.empty((n_px, cfg.n_outputs), device="cuda")
    try:
        ms = _timed(stream, lambda k: nvc.nvc_mlp_infer_features(cache.handle, feat, vis), 20)
    except Exception as e:
        return {"unavailable": str(e)}
    flops = 2 * algorithmic(cfg, n_px)["macs_per_px"] * n_px
    tf = flops / (ms * 1e-3) / 1e12
    del feat, vis
    # operands in and float32 visibilities out: at the copy peak this I/O
    # takes longer than the contraction at the tensor peak, so HBM bounds
    # the launch
    io = n_px * (k0 * 2 + cfg.n_outputs * 4)
    io_gbs = io / (ms * 1e-3) / 1e9
    return {"workload": f"{n_px} pixels x {k0} 16-bit operands, MLP of the frame's network, "
                        "sigmoid visibilities out",
            "ms": ms, "tflops": tf, "peak_tflops": pk["bf16_sustained"],
            "frac_of_tensor_peak": tf / pk["bf16_sustained"],
            "io_bytes": io, "io_gbs": io_gbs, "peak_hbm_gbs": pk["hbm"],
            "frac_of_hbm": io_gbs / pk["hbm"],
            "bound": "hbm" if io / pk["hbm"] > flops / (pk["bf16_sustained"] * 1e3) else "tensor"}


def _timed(stream, fn, n, warm=3):
    """Mean milliseconds of fn(k) over n calls on `stream` (CUDA events),
    after `warm` untimed calls."""
    import torch
    for w in range(warm):
        fn(w)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(n):
        fn(warm + k)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def shade_views(cfg, n_pixels, seconds):
    """The fused shading kernel's ALU roofline view for `n_pixels` pixels of
    configuration `cfg` shaded in `seconds`."""
    alg = algorithmic(cfg, n_pixels)
    pk = peaks()
    return {"alu_frac": alg["shade_alu_ops"] / seconds / alu_peak_ops(),
            "tensor_frac_of_sustained": alg["shade_flops"] / seconds / 1e12 / pk["bf16_sustained"],
            "alu_ops_per_px": alg["alu_ops_per_px"], "mlp_flop_per_px": 2 * alg["macs_per_px"]}


def measure_training_data_fusion(cache, scene, screen, seed, frame0, stream, n=20):
    """The 1080p training step with its batch made by a launch of its own
    and made inside the tensor-core training kernel (Section 4.4 fuses
    them): milliseconds per step (positions + shadow-ray targets, forward,
    loss, backward, Adam) for each, on the bench's own cache; the handle's
    setting is restored afterwards."""
    from paper_2506_05930_gb300 import nvc
    import torch
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    s = stream.cuda_stream
    out = {}
    for fused in (False, True):
        nvc.nvc_set_training_data_fused(cache.handle, fused)
        out["fused_ms" if fused else "separate_ms"] = _timed(
            stream, lambda f: nvc.nvc_train_step(cache.handle, scene, screen, seed, frame0 + f, loss,
                                                 stream=s), n)
    nvc.nvc_set_training_data_fused(cache.handle, False)
    out["note"] = ("training step incl. Adam; separate: positions + targets in their own "
                   "launch over all SMs; fused: inside the 64 training CTAs, traced while the "
                   "forward MMAs run")
    return out


def measure_multiview(stream):
    """The batched multi-view workload: four views of the unit-cube scene at
    1280x720, 1920x1080, 2560x1440 and 3840x2160 (14,976,000 pixels), 128
    lights, MLP 32-64-64-64-128, every view shaded by one persistent launch
    of the variant the project's autotuner picks; the frame (a training step
    on 8,192 positions x 128 lights, then the shading) replayed as one CUDA
    graph, and the shading alone.  10 frames after 3 warm-up."""
    import torch
    from paper_2506_05930_gb300 import nvc
    import nvc_synth as S
    cfg = S.config_by_name("multiview")
    sc = S.scene_unit_cube(seed=0, n_lights=128)
    gbs = S.multiview_gbuffers(seed=0)
    P = sum(g.n for g in gbs)
    cache = nvc.VisibilityCache(cfg)
    cache.set_params(S.init_params(cfg, seed=0))
    scene = nvc.Scene.from_synth(sc)
    views = []
    for v, gb in enumerate(gbs):
        n = gb.n
        views.append(nvc.View(torch.from_numpy(gb.pos).cuda(), torch.from_numpy(gb.nrm).cuda(), v,
                              torch.empty(n, dtype=torch.int32, device="cuda"),
                              torch.empty(n, device="cuda"), torch.empty(n, device="cuda"),
                              torch.empty(n, device="cuda")))
    big = views[-1]
    chosen, tried = nvc.nvc_autotune_shade_plan(cache.handle, scene, big.pos, big.nrm, big.idx,
                                                big.pdf, big.wsum, big.radiance, reps=3)
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    s = stream.cuda_stream
    frame_ms = _timed(stream, lambda f: nvc.nvc_frame(cache.handle, scene, views, 1, 11, f, loss,
                                                      use_graph=True, stream=s), 10)
    shade_ms = _timed(stream, lambda f: nvc.nvc_frame(cache.handle, scene, views, nvc.NO_TRAINING,
                                                      11, 100 + f, use_graph=True, stream=s), 10)
    cache.close()
    return {"workload": "multiview: 1280x720 + 1920x1080 + 2560x1440 + 3840x2160 views "
                        "(14,976,000 pixels), 128 lights, MLP 32-64-64-64-128, one launch",
            "pixels": P, "frame_ms": frame_ms, "value": P / (frame_ms * 1e-3) / 1e6,
            "unit": "Mpixels/s", "shade_ms": shade_ms,
            "shade_mpixels_s": P / (shade_ms * 1e-3) / 1e6,
            "autotune": {"chosen": {"variant": chosen[0], "ctas_per_sm": chosen[1]},
                         "points_ms_4k_view": {f"{v}/{c}": round(m, 4) for (v, c), m in tried}},
            "roofline": shade_views(cfg, P, shade_ms * 1e-3)}


def measure_online_training(stream):
    """The online-training workload: the tiny scene seen along its camera
    path, 16,384 positions x 4 lights = 65,536 shadow-ray samples per frame,
    BCE, FP16 tensor-core forward/backward, loss scale 128, Adam; one frame =
    the training step + inference, WRS and Neural DI of the 64x64 view, as a
    CUDA graph.  100 frames of the path after 5 warm-up (their G-buffers made
    on the host beforehand and uploaded once)."""
    import torch
    from paper_2506_05930_gb300 import nvc
    import nvc_synth as S
    cfg = S.config_by_name("online_train")
    sc = S.scene_unit_cube(seed=0)
    cache = nvc.VisibilityCache(cfg)
    cache.set_params(S.init_params(cfg, seed=0))
    scene = nvc.Scene.from_synth(sc)
    n_frames = 105
    gbs = [S.gbuffer_camera_path(seed=0, frame=f) for f in range(n_frames)]
    n = gbs[0].n
    views = [nvc.View(torch.from_numpy(g.pos).cuda(), torch.from_numpy(g.nrm).cuda(), 0,
                      torch.empty(n, dtype=torch.int32, device="cuda"),
                      torch.empty(n, device="cuda"), torch.empty(n, device="cuda"),
                      torch.empty(n, device="cuda")) for g in gbs]
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    s = stream.cuda_stream
    frame_ms = _timed(stream, lambda f: nvc.nvc_frame(cache.handle, scene, [views[f]], 0, 2, f,
                                                      loss, use_graph=True, stream=s), 100, warm=5)
    train_ms = _timed(stream, lambda f: nvc.nvc_train_step(cache.handle, scene, views[f % n_frames].pos,
                                                           2, 1000 + f, loss, stream=s), 100, warm=5)
    samples = cfg.batch_positions * cfg.n_outputs
    cache.close()
    return {"workload": "online_train: unit-cube scene, 64x64 view on the camera path, 16,384 "
                        "positions x 4 lights per frame, FP16 training with loss scale 128",
            "us_per_frame": frame_ms * 1e3, "train_step_us": train_ms * 1e3,
            "training_samples_per_s": samples / (train_ms * 1e-3),
            "training_positions_per_s": cfg.batch_positions / (train_ms * 1e-3),
            "note": "a launch-latency-bound workload; frame = training step + shading in one graph"}


def measure_precisions(stream):
    """The 4K precision workload: 3840x2160 pixels of the heightfield scene
    with 256 lights and 256 occluders, T = 2^21 with half-precision table
    features for the tensor-core paths; inference + WRS + Neural DI per
    MLP precision (FP32 on the CUDA cores with the float32 table, FP16, BF16
    and E4M3 on the tensor cores), each with the variant the autotuner
    picks.  5 launches after 2 warm-up per precision."""
    import torch
    from paper_2506_05930_gb300 import nvc
    import nvc_synth as S
    base = S.config_by_name("precision_4k")
    sc = S.scene_heightfield(seed=5, n_lights=256, n_spheres=128, n_boxes=128)
    gb = S.gbuffer_heightfield(seed=5, width=3840, height=2160)
    scene = nvc.Scene.from_synth(sc)
    pos = torch.from_numpy(gb.pos).cuda()
    nrm = torch.from_numpy(gb.nrm).cuda()
    P = gb.n
    p = S.init_params(base, seed=0)
    out = dict(idx=torch.empty(P, dtype=torch.int32, device="cuda"),
               pdf=torch.empty(P, device="cuda"), wsum=torch.empty(P, device="cuda"),
               radiance=torch.empty(P, device="cuda"))
    s = stream.cuda_stream
    res = {}
    for prec in ("fp32", "fp16", "bf16", "fp8"):
        cfg = base.with_(precision=prec, train_precision="fp32",
                         table_precision="fp32" if prec == "fp32" else "fp16")
        cache = nvc.VisibilityCache(cfg)
        cache.set_params(p)
        fused = prec != "fp32"
        chosen = None
        if prec == "fp8":
            nvc.nvc_calibrate(cache.handle, pos[::4096][:1024].contiguous())
        if not fused:
            nvc.nvc_set_staging(cache.handle, P)
        else:
            chosen, _ = nvc.nvc_autotune_shade_plan(cache.handle, scene, pos, nrm, reps=2, **out)
        ms = _timed(stream, lambda f: nvc.nvc_shade(cache.handle, scene, pos, nrm, 3, f, 0, 0,
                                                    fused=fused, stream=s, **out), 5, warm=2)
        r = {"ms": ms, "mpixels_s": P / (ms * 1e-3) / 1e6, "variant": chosen}
        if fused:
            r["roofline"] = shade_views(cfg, P, ms * 1e-3)
        res[prec] = r
        cache.close()
    return {"workload": "precision_4k: 3840x2160 heightfield view, 256 lights, 256 occluders, "
                        "T = 2^21, MLP 32-64-64-64-256; inference + WRS + Neural DI",
            "precisions": res}


CLUSTERED_LIGHTS = 1024
PAPER_SCALE_LIGHTS = 59000      # the light count of the paper's many-lights scene


def measure_clustered(args, gb, stream):
    """The clustered cache (Section 3.6) on the same G-buffer: the 16-room
    scene with 1024 lights in k = 32 k-means clusters, one frame = a
    clustered training step (49,152 positions), inference of the cluster
    visibilities, and the two-step sampler with its one shadow ray.  Timed
    with CUDA events over 20 frames after 3 warm-up frames."""
    import torch
    from paper_2506_05930_gb300 import nvc
    import nvc_synth as S
    cfg = S.config_by_name("clustered_1080p")
    sc = S.scene_rooms(seed=1, n_lights=CLUSTERED_LIGHTS)
    k = cfg.n_outputs
    assign, _ = nvc.nvc_kmeans_lights(sc.lights, S.kmeans_init(CLUSTERED_LIGHTS, k, seed=0), 10)
    cl = nvc.Clusters(assign, k)
    cl_vis = nvc.Clusters(assign, k, weights="visibility")
    scene = nvc.Scene.from_synth(sc)
    P = gb.n
    pos = torch.from_numpy(gb.pos).cuda()
    nrm = torch.from_numpy(gb.nrm).cuda()
    cache = nvc.VisibilityCache(cfg)
    cache.set_params(S.init_params(cfg, seed=0))
    nvc.nvc_set_staging(cache.handle, P)
    vis = torch.empty((P, k), device="cuda")
    infer_variant, _ = nvc.nvc_autotune_infer(cache.handle, pos, vis, reps=3)
    light = torch.empty(P, dtype=torch.int32, device="cuda")
    W = torch.empty(P, device="cuda")
    est = torch.empty(P, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else None

    def frame(f, parts=("train", "infer", "sample")):
        if "train" in parts:
            nvc.nvc_train_step_clustered(cache.handle, scene, cl, pos, 5, f, loss, stream=s)
        if "infer" in parts:
            nvc.nvc_infer(cache.handle, pos, vis, stream=s)
        if "sample" in parts:
            nvc.nvc_sample_clustered(scene, cl, vis, pos, nrm, 7, f, light=light, weight=W,
                                     estimate=est, stream=s)
        if "sample_only" in parts:
            nvc.nvc_sample_clustered(scene, cl, vis, pos, nrm, 7, f, light=light, weight=W,
                                     stream=s)
        if "sample_vis" in parts:
            nvc.nvc_sample_clustered(scene_v, cl_v, vis, pos, nrm, 7, f, light=light,
                                     weight=W, estimate=est, stream=s)

    def timed(parts, n=20):
        for w in range(3):
            frame(w, parts)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for f in range(n):
            frame(100 + f, parts)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    frame_ms = timed(("train", "infer", "sample"))
    train_ms = timed(("train",))
    infer_ms = timed(("infer",))
    sample_ms = timed(("sample",))
    sampler_ms = timed(("sample_only",))
    # the visibility-only first-step weights: cost independent of the light
    # count, timed at 1024 lights and at the paper's many-lights scale
    scene_v, cl_v = scene, cl_vis
    sample_vis_ms = timed(("sample_vis",))
    frame_vis_ms = timed(("train", "infer", "sample_vis"))
    sc_big = S.scene_rooms(seed=1, n_lights=PAPER_SCALE_LIGHTS)
    assign_big, _ = nvc.nvc_kmeans_lights(sc_big.lights,
                                          S.kmeans_init(PAPER_SCALE_LIGHTS, k, seed=0), 10)
    scene_v = nvc.Scene.from_synth(sc_big)
    cl_v = nvc.Clusters(assign_big, k, weights="visibility")
    sample_vis_big_ms = timed(("sample_vis",))
    # the summed-contribution weights at the same scale: one contribution per
    # light and pixel, the lights staged through shared memory in tiles
    cl_v = nvc.Clusters(assign_big, k, weights="sum")
    sample_sum_big_ms = timed(("sample_vis",), n=3)
    cache.close()
    ops = clustered_alu_ops(CLUSTERED_LIGHTS, k, P)
    peak = alu_peak_ops()
    return {
        "workload": f"16-room scene, {CLUSTERED_LIGHTS} lights in k = {k} clusters, "
                    f"{gb.width}x{gb.height} heightfield G-buffer, 49,152 training positions",
        "value": P / (frame_ms * 1e-3) / 1e6, "unit": "Mpixels/s", "frame_ms": frame_ms,
        "train_ms": train_ms, "infer_ms": infer_ms, "infer_variant": infer_variant,
        "sample_with_shadow_ray_ms": sample_ms,
        f"sample_with_shadow_ray_ms_at_{PAPER_SCALE_LIGHTS}_lights": sample_sum_big_ms,
        "sampler_ms": sampler_ms,
        "visibility_weights": {
            "frame_ms": frame_vis_ms, "value": P / (frame_vis_ms * 1e-3) / 1e6,
            "sample_with_shadow_ray_ms": sample_vis_ms,
            f"sample_with_shadow_ray_ms_at_{PAPER_SCALE_LIGHTS}_lights": sample_vis_big_ms,
            "note": "first-step weights max(v, 0.001) alone (NVC_CLUSTER_WEIGHT_VISIBILITY)"},
        "roofline": {"kernel": "sample_clustered_kernel (no shadow ray)", "bound": "alu",
                     "achieved": ops / (sampler_ms * 1e-3) / 1e12, "peak": peak / 1e12,
                     "unit": "Tops/s", "frac": ops / (sampler_ms * 1e-3) / peak,
                     "ops_per_pixel": ops / P,
                     "traffic": KERNEL_TRAFFIC["sample_clustered"] if P == 1920 * 1080 else None,
                     "traffic_launch": "ncu, 1080p launch with the shadow ray",
                     "peak_source": "152 SMs x 128 lanes x 2070 MHz (max SM clock)"},
    }



def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2506_05930_gb300.build import build
    build()
    from paper_2506_05930_gb300 import nvc
    import nvc_synth as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    cfg, sc, gb = workload(args.precision)
    P = gb.n
    seed, view_id = rank_stream(rank)
    scene = nvc.Scene.from_synth(sc)
    pos = torch.from_numpy(gb.pos).cuda()
    nrm = torch.from_numpy(gb.nrm).cuda()
    cache = nvc.VisibilityCache(cfg)
    cache.set_params(S.init_params(cfg, seed=0))
    fused = cfg.precision != "fp32"
    if not fused:
        nvc.nvc_set_staging(cache.handle, P)
    view = nvc.View(pos, nrm, view_id, torch.empty(P, dtype=torch.int32, device="cuda"),
                    torch.empty(P, device="cuda"), torch.empty(P, device="cuda"),
                    torch.empty(P, device="cuda"))
    tune = None
    if fused:
        # the project's autotuner picks the fused kernel's point -- layout
        # (tile streams per CTA, levels split across threads, warp
        # specialisation) x resident CTAs per SM -- for this frame (untimed)
        chosen, tried = nvc.nvc_autotune_shade_plan(cache.handle, scene, pos, nrm, view.idx,
                                                    view.pdf, view.wsum, view.radiance, reps=5)
        tune = {"chosen": {"variant": chosen[0], "ctas_per_sm": chosen[1]},
                "points_ms": {f"{v}/{c}": round(m, 4) for (v, c), m in tried}}
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    use_graph = not args.no_graph
    # pretraining (untimed): 500 frames of online training on this view
    for f in range(args.pretrain):
        nvc.nvc_train_step(cache.handle, scene, pos, seed, f, loss)
    torch.cuda.synchronize()
    frame0 = args.pretrain

    def frame(f):
        nvc.nvc_frame(cache.handle, scene, [view], 0, seed, f, loss, use_graph=use_graph)

    for w in range(args.warmup):
        frame(frame0 + w)
    nvc.nvc_stage_times(cache.handle)        # reset counters
    stream = torch.cuda.current_stream()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.ready()
        clocks.begin()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        frame(frame0 + args.warmup + k)
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms_total = t0.elapsed_time(t1)
    clk = clocks.stop() if clocks else None
    _, launches = nvc.nvc_stage_times(cache.handle)
    ms_total = max_over_ranks(ms_total, "cuda")
    ms_frame = ms_total / args.steps
    value = job_throughput(world, P, ms_frame)

    # per-stage attribution with CUDA events around each stage (eager frames)
    nvc.nvc_set_profiling(cache.handle, True)
    nvc.nvc_stage_times(cache.handle)
    f0 = frame0 + args.warmup + args.steps
    ta = torch.cuda.Event(enable_timing=True)
    tb = torch.cuda.Event(enable_timing=True)
    ta.record(stream)
    for k in range(args.steps):
        nvc.nvc_frame(cache.handle, scene, [view], 0, seed, f0 + k, loss, use_graph=False)
    tb.record(stream)
    torch.cuda.synchronize()
    eager_ms = ta.elapsed_time(tb) / args.steps
    stage_ms, _ = nvc.nvc_stage_times(cache.handle)
    nvc.nvc_set_profiling(cache.handle, False)
    stage_ms = [m / args.steps for m in stage_ms]

    # the encode's and the MLP's own rooflines: the random-gather rate of an
    # L2-resident table, and the fused kernel's time split by phase
    gather = measure_gather_peak(stream) if rank == 0 else None
    phases = None
    if rank == 0 and fused:
        sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
        phases = measure_phases(cache, scene, pos, nrm, view, seed, f0 + args.steps, stage_ms[3],
                                cfg, gather, peaks(), sm_mhz)
    mlp_only = measure_mlp_only(cache, cfg, P, stream, peaks()) if rank == 0 and fused else None

    # end to end through the public API with host buffers
    pin_pos = torch.from_numpy(gb.pos).pin_memory()
    pin_nrm = torch.from_numpy(gb.nrm).pin_memory()
    out_h = [torch.empty(P, dtype=torch.int32).pin_memory()] + \
        [torch.empty(P).pin_memory() for _ in range(3)]
    h2d = pin_pos.numel() * 4 + pin_nrm.numel() * 4
    d2h = sum(t.numel() * 4 for t in out_h)

    # the library's host-buffer frame: every step uploads its G-buffer from
    # pinned memory and reads its four outputs back, on the library's copy
    # streams, pipelined so a frame's compute overlaps the next upload and
    # the previous read-back; the timed region ends after the last read-back
    host_view = nvc.View(pin_pos, pin_nrm, view_id, *out_h)

    def e2e_step(f):
        nvc.nvc_frame_host(cache.handle, scene, [host_view], 0, seed, f, loss,
                           use_graph=use_graph)

    f1 = f0 + args.steps
    for w in range(2):
        e2e_step(f1 + w)
    nvc.nvc_host_frames_wait(cache.handle, stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e_steps = max(5, args.steps // 2)
    if world > 1:
        dist.barrier()
    e0.record(stream)
    for k in range(e_steps):
        e2e_step(f1 + 2 + k)
    nvc.nvc_host_frames_wait(cache.handle, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e_ms = e0.elapsed_time(e1) / e_steps
    e_ms = max_over_ranks(e_ms, "cuda")

    # the plain float32 separate-kernel path, same frame (the baseline to beat)
    base = None
    if fused and rank == 0:
        cache32 = nvc.VisibilityCache(cfg.with_(precision="fp32"))
        cache32.set_params(cache.state()[0])
        nvc.nvc_set_staging(cache32.handle, P)
        for w in range(3):
            nvc.nvc_frame(cache32.handle, scene, [view], 0, seed, f1 + w, loss, use_graph=use_graph)
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for k in range(args.steps):
            nvc.nvc_frame(cache32.handle, scene, [view], 0, seed, f1 + 3 + k, loss,
                          use_graph=use_graph)
        b1.record(stream)
        torch.cuda.synchronize()
        bm = b0.elapsed_time(b1) / args.steps
        base = {"ms_per_step": bm, "value": P / (bm * 1e-3) / 1e6}
        cache32.close()

    # the shading pass (Section 3.1: one shadow ray per pixel to the picked
    # light, running mean) and the all-lights exact DI that Section 4.4
    # compares the cache's inference with; reported beside the frame
    shading = None
    if rank == 0:
        acc = torch.zeros(P, device="cuda")
        exact = torch.empty(P, device="cuda")
        nvc.nvc_shade_estimate(scene, pos, nrm, view.idx, view.pdf, accum=acc, count=1)
        nvc.nvc_exact_di(scene, pos, nrm, exact)
        torch.cuda.synchronize()
        x0 = torch.cuda.Event(enable_timing=True)
        x1 = torch.cuda.Event(enable_timing=True)
        x0.record(stream)
        for k in range(20):
            nvc.nvc_shade_estimate(scene, pos, nrm, view.idx, view.pdf, accum=acc, count=k + 2)
        x1.record(stream)
        torch.cuda.synchronize()
        pass_ms = x0.elapsed_time(x1) / 20
        x0.record(stream)
        for k in range(5):
            nvc.nvc_exact_di(scene, pos, nrm, exact)
        x1.record(stream)
        torch.cuda.synchronize()
        exact_ms = x0.elapsed_time(x1) / 5
        shading = {"shade_pass_ms": pass_ms, "exact_di_ms": exact_ms,
                   "exact_di_over_inference": exact_ms / stage_ms[3] if stage_ms[3] > 0 else None,
                   "note": "shade pass: one shadow ray per pixel to the sampled light, V c / p, "
                           "running mean; exact DI: a shadow ray to every light from every pixel"}

    fusion = (measure_training_data_fusion(cache, scene, pos, seed, 10_000, stream)
              if rank == 0 and cfg.train_precision == "fp16" else None)
    clustered = measure_clustered(args, gb, stream) if rank == 0 else None
    tiny = measure_tiny(stream, use_graph) if rank == 0 else None
    multiview = measure_multiview(stream) if rank == 0 else None
    online = measure_online_training(stream) if rank == 0 else None
    precisions = measure_precisions(stream) if rank == 0 else None

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    pk = peaks()
    alg = algorithmic(cfg, P)
    shade_s = stage_ms[3] * 1e-3
    adam_s = stage_ms[2] * 1e-3
    # the dominant stage sets the reported roofline; the others ride along
    peak_alu = alu_peak_ops()
    shade_view = {"kernel": "fused_shade (encode + tcgen05 MLP + WRS + Neural DI)",
                  "bound": "alu", "achieved": alg["shade_alu_ops"] / shade_s / 1e12,
                  "peak": peak_alu / 1e12, "unit": "Tops/s",
                  "peak_source": "152 SMs x 128 lanes x 2070 MHz (max SM clock)",
                  "traffic": KERNEL_TRAFFIC["fused_shade"].get(
                      tune["chosen"]["variant"] if tune else None)}
    if not fused:
        shade_view["kernel"] = "shade (encode, MLP, WRS+DI kernels)"
        shade_view["traffic"] = None
    adam_view = {"kernel": "adam", "bound": "hbm",
                 "achieved": alg["adam_bytes"] / adam_s / 1e9 if adam_s > 0 else None,
                 "peak": pk["hbm"], "unit": "GB/s", "peak_source": pk["src"] + " (MEASURED_PEAKS hbm_gbs)",
                 "traffic": KERNEL_TRAFFIC["adam"]}
    tensor_view = {"kernel": "fused_shade MLP share", "bound": "tensor",
                   "achieved": alg["shade_flops"] / shade_s / 1e12, "peak": pk["bf16_sustained"],
                   "unit": "TFLOP/s", "peak_source": pk["src"] + " bf16 sustained (fp16 same rate)"}
    for v in (shade_view, adam_view, tensor_view):
        if v.get("achieved") is not None:
            v["frac"] = v["achieved"] / v["peak"]
    # the fused kernel's three views: ALU issue (the bound), the encode's
    # gathers against the measured L2 random-gather rate, the MLP against the
    # tensor peak (both over their phase's share of the kernel time)
    shade_view["views"] = {"alu_whole_kernel": {"achieved": shade_view["achieved"],
                                                "frac": shade_view.get("frac"),
                                                "ops_per_px": alg["alu_ops_per_px"]},
                           "tensor_whole_kernel": {"achieved": tensor_view["achieved"],
                                                   "frac": tensor_view["frac"]}}
    if phases and "share" in phases:
        shade_view["views"]["encode_vs_l2_gather"] = {
            "achieved_gbs": phases["encode"]["useful_gather_gbs"],
            "peak_gbs": phases["encode"]["l2_gather_peak_gbs"],
            "frac": phases["encode"]["frac_of_l2_gather"], "phase_share": phases["share"]["encode"]}
        shade_view["views"]["mlp_vs_tensor"] = {
            "achieved_tflops": phases["mlp"]["tflops"], "peak_tflops": pk["bf16_sustained"],
            "frac": phases["mlp"]["frac_of_tensor_peak"], "phase_share": phases["share"]["mlp"],
            "per_tile_frac": phases["mlp"]["per_tile_frac"]}
    if mlp_only and "tflops" in mlp_only:
        shade_view["views"]["mlp_only_launch_vs_tensor"] = {
            "achieved_tflops": mlp_only["tflops"], "peak_tflops": pk["bf16_sustained"],
            "frac": mlp_only["frac_of_tensor_peak"], "ms": mlp_only["ms"],
            "bound": mlp_only["bound"], "io_frac_of_hbm": mlp_only["frac_of_hbm"]}
    roof = shade_view if stage_ms[3] >= stage_ms[2] else adam_view
    line = {
        "metric": METRIC, "value": value, "unit": "Mpixels/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_frame,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": cfg.precision, "data": "synthetic",
        "config": workload_config(world, P, cfg.batch_positions),
        "cuda_graph": use_graph,
        "roofline": roof,
        "roofline_other": [v for v in (shade_view, adam_view, tensor_view) if v is not roof],
        "stages_ms": {"train_data": stage_ms[0], "train_fwd_bwd": stage_ms[1],
                      "adam": stage_ms[2], "shade": stage_ms[3], "eager_frame": eager_ms},
        "infer_mpixels_s": P / shade_s / 1e6 if shade_s > 0 else None,
        "train_ms": stage_ms[0] + stage_ms[1] + stage_ms[2],
        "train_rates": {
            "positions_per_s": cfg.batch_positions / ((stage_ms[0] + stage_ms[1] + stage_ms[2]) * 1e-3),
            "targets_per_s": cfg.batch_positions * cfg.n_outputs
                             / ((stage_ms[0] + stage_ms[1] + stage_ms[2]) * 1e-3),
            "note": "training step = positions + shadow-ray targets, forward/backward, Adam"},
        "e2e": {"value": job_throughput(world, P, e_ms), "unit": "Mpixels/s",
                "ms_per_step": e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "autotune": tune,
        "clocks": clk,
        "l2_gather_peak_gbs": gather["row8"]["useful_gbs"] if gather else None,
        "gather_bench": gather,
        "shade_phases": phases,
        "mlp_only": mlp_only,
    }
    if base:
        line["fp32_unfused_baseline"] = base
    if shading:
        line["shading_pass"] = shading
    if clustered:
        line["clustered"] = clustered
    if tiny:
        line["tiny_frame"] = tiny
    if fusion:
        line["training_data_fusion"] = fusion
    if multiview:
        line["multiview"] = multiview
    if online:
        line["online_training"] = online
    if precisions:
        line["precision_4k"] = precisions
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(threads=1, parts=4)
        line["cpu_baseline_all_cores"] = cpu_baseline(threads=oracle_processes())
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------- the oracle on the CPU --

def oracle_frame_sample(n_pixels=16384, n_positions=1024, seed=0, adam_params=None, fixed=None):
    """Time the oracle on a sample of the frame and extrapolate to the whole
    frame.  Each part is modelled as a fixed cost plus a per-unit cost: the
    oracle's calls carry work proportional to the whole parameter vector
    (splitting and joining it, a full-size gradient) whatever the sample, so
    `fixed` holds the times of the same calls on one pixel / one position
    (oracle_fixed_costs) and only the rest is scaled: shading by pixels,
    training forward/backward by positions, the dense Adam update by
    parameters (all of them when adam_params is None)."""
    import numpy as np
    from oracle import nvc as O
    import nvc_synth as S
    cfg, sc, gb = workload()
    if "oracle_state" not in _WORKLOAD_CACHE:      # parameters and Adam state, made once
        p0 = S.init_params(cfg, seed=0)
        _WORKLOAD_CACHE["oracle_state"] = (p0, O.TrainState.fresh(p0))
    p, st = _WORKLOAD_CACHE["oracle_state"]
    rng = np.random.default_rng(seed)
    pick = rng.choice(gb.n, n_pixels, replace=False)
    t0 = time.perf_counter()
    O.shade(cfg, p, gb.pos[pick], gb.nrm[pick], sc.lights, seed=1, frame=0)
    t1 = time.perf_counter()
    pos = O.training_positions(n_positions, sc.world_min, sc.world_max, gb.pos, 1, 0)
    y = O.visibility(pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    _, g = O.gradients(cfg, p, pos, y)
    t2 = time.perf_counter()
    k = len(p) if adam_params is None else min(int(adam_params), len(p))
    O.adam_update(st.params[:k], g[:k], st.m[:k], st.v[:k], 1, cfg.lr, cfg.beta1, cfg.beta2,
                  cfg.eps)
    t3 = time.perf_counter()
    f_shade, f_train = fixed if fixed else (0.0, 0.0)

    def scaled(t, f, n, total):
        return f + max(t - f, 0.0) * (total - 1) / max(n - 1, 1) if n > 1 else t * total

    frame_s = (scaled(t1 - t0, f_shade, n_pixels, gb.n)
               + scaled(t2 - t1, f_train, n_positions, cfg.batch_positions)
               + (t3 - t2) * len(p) / k)
    return frame_s, t3 - t0, gb.n


def oracle_fixed_costs(reps=2):
    """The oracle's shading call on one pixel and its training forward/
    backward on one position: the per-call costs the sample times carry."""
    import numpy as np
    from oracle import nvc as O
    import nvc_synth as S
    cfg, sc, gb = workload()
    p = S.init_params(cfg, seed=0)
    fs, ft = [], []
    for _ in range(reps):
        t0 = time.perf_counter()
        O.shade(cfg, p, gb.pos[:1], gb.nrm[:1], sc.lights, seed=1, frame=0)
        t1 = time.perf_counter()
        pos = O.training_positions(1, sc.world_min, sc.world_max, gb.pos, 1, 0)
        y = O.visibility(pos, sc.lights, sc.spheres, sc.boxes, np.float32)
        O.gradients(cfg, p, pos, y)
        t2 = time.perf_counter()
        fs.append(t1 - t0)
        ft.append(t2 - t1)
    return min(fs), min(ft)


def oracle_processes(per_process_bytes=2e9):
    """One oracle process per host core, but no more than fit in half the
    memory that is free now (a process peaks near 1.5 GB)."""
    cores = os.cpu_count() or 1
    try:
        free = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError, AttributeError):
        return 1
    return max(1, min(cores, int(0.5 * free // per_process_bytes)))


def oracle_frame_part(k, n_parts, chunk=32768):
    """Part k of n_parts of one 1080p frame on the oracle, timed directly:
    inference + WRS + Neural DI of pixels [k P / n, (k + 1) P / n), the
    training forward/backward on positions [k B / n, (k + 1) B / n) of the
    frame's batch, and the Adam update of parameters [k N / n, (k + 1) N / n).
    Returns the part's pixel count; the caller times it."""
    import numpy as np
    from oracle import nvc as O
    import nvc_synth as S
    cfg, sc, gb = workload()
    if "oracle_state" not in _WORKLOAD_CACHE:
        p0 = S.init_params(cfg, seed=0)
        _WORKLOAD_CACHE["oracle_state"] = (p0, O.TrainState.fresh(p0))
    p, st = _WORKLOAD_CACHE["oracle_state"]

    def span(total):
        return total * k // n_parts, total * (k + 1) // n_parts

    def work():
        a, b = span(gb.n)
        for c in range(a, b, chunk):
            e = min(c + chunk, b)
            O.shade(cfg, p, gb.pos[c:e], gb.nrm[c:e], sc.lights, seed=1, frame=0,
                    pixel_offset=c)
        pos = O.training_positions(cfg.batch_positions, sc.world_min, sc.world_max, gb.pos, 1, 0)
        a2, b2 = span(cfg.batch_positions)
        y = O.visibility(pos[a2:b2], sc.lights, sc.spheres, sc.boxes, np.float32)
        _, g = O.gradients(cfg, p, pos[a2:b2], y)
        a3, b3 = span(len(p))
        O.adam_update(st.params[a3:b3], g[a3:b3], st.m[a3:b3], st.v[a3:b3], 1, cfg.lr, cfg.beta1,
                      cfg.beta2, cfg.eps)
        return b - a
    return work


def cpu_baseline(threads=1, parts=None):
    """The oracle's 1080p frame on the host, timed directly: the frame is
    split into `parts` disjoint parts (oracle_frame_part; default one per
    process) and `threads` single-threaded oracle processes (one BLAS
    thread each) run parts 0 .. threads - 1.  Each sets up, reports ready
    and waits; all start together on one signal, and the time is the span
    from the earliest start to the latest end.  With parts > threads only
    that share of the frame runs, and the frame time is the span times
    parts / threads (every part holds the same share of pixels, positions
    and parameters).  The training step's partial gradients are not summed
    across processes (each updates its own slice of the parameters)."""
    n = max(int(threads), 1)
    parts = max(int(parts or n), n)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, sys, time; sys.path.insert(0, %r); import bench; "
            "work = bench.oracle_frame_part(int(sys.argv[1]), int(sys.argv[2])); "
            "print('ready', flush=True); sys.stdin.readline(); "
            "t0 = time.time(); px = work(); t1 = time.time(); "
            "print(json.dumps([t0, t1, px]), flush=True)" % ROOT)
    procs = [subprocess.Popen([sys.executable, "-c", code, str(k), str(parts)], stdin=subprocess.PIPE,
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
             for k in range(n)]

    def abandon(msg):
        for q in procs:
            if q.poll() is None:
                q.kill()
            q.wait()
        return {"error": msg[-300:]}

    for pr in procs:
        if pr.stdout.readline().strip() != "ready":
            return abandon(pr.stderr.read() if pr.poll() is not None else "no ready line")
    for pr in procs:
        pr.stdin.write("go\n")
        pr.stdin.flush()
    results = []
    for pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            return abandon(err)
        results.append(json.loads(out.strip().splitlines()[-1]))
    t0 = min(r[0] for r in results)
    t1 = max(r[1] for r in results)
    span = t1 - t0
    frame_s = span * parts / n
    P = sum(r[2] for r in results) * parts // n
    share = "the whole 1080p frame" if parts == n else "%d/%d of the 1080p frame" % (n, parts)
    return {"value": P / frame_s / 1e6, "unit": "Mpixels/s", "cores": n, "kind": "oracle",
            "ms_per_frame": frame_s * 1e3, "wall_s": span,
            "sample": ("%s timed directly: %d disjoint equal parts run by %d concurrent "
                       "single-threaded oracle processes started together: inference + WRS + "
                       "Neural DI of the part's pixels, the training forward/backward on its "
                       "share of the 8,192 positions and the Adam update of its share of the "
                       "parameters (partial gradients not summed across processes)%s"
                       % (share, n, n, "" if parts == n else
                          "; frame time = the span x %d/%d" % (parts, n)))}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg, _, _ = workload()
    fixed = oracle_fixed_costs()
    sample = dict(n_pixels=2048, n_positions=128, adam_params=1 << 19, fixed=fixed)
    for _ in range(args.warmup):
        oracle_frame_sample(**sample)
    frames, walls = [], []
    t0 = time.perf_counter()
    for k in range(args.steps):
        f, w, P = oracle_frame_sample(seed=k, **sample)
        frames.append(f)
        walls.append(w)
    frame_s = sum(frames) / len(frames)
    value = P / frame_s / 1e6
    line = {
        "metric": METRIC, "value": value, "unit": "Mpixels/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": frame_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": workload_config(world, P, cfg.batch_positions),
        "cpu_baseline": {"value": value, "unit": "Mpixels/s", "cores": 1, "kind": "oracle",
                         "sample": "per step 2,048 pixels shaded, training forward/backward on "
                                   "128 positions, Adam over 2^19 of the 16.8M parameters; each "
                                   "part extrapolated to the 1080p frame as a fixed per-call cost "
                                   "(timed once on one pixel / one position) plus a linear rest",
                         "wall_s_per_step": sum(walls) / len(walls)},
        "e2e": {"value": value, "unit": "Mpixels/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
