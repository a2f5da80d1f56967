#!/usr/bin/env python
"""Benchmark of the SSGI hot path on GB300: one step = one inverse-rendering iteration of the
1600x900, 16 spp workload (environment mips -> Hi-Z -> direct shading -> Monte-Carlo screen-
space trace -> L2 loss -> backward), every stage a libssgi.so call.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  `value` is indirect rays per second through the whole step
(V*H*W*spp rays / step time), all ranks together; each rank renders its own frame (weak
scaling, no collective on the data path).  `--impl reference` times the FP64 CPU oracle on
the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "indirect rays/s & fwd+bwd ms at 1600x900x16spp; serving p50/p99 ms vs plain"
UNIT = "rays/s"
L2_FLUSH_BYTES = 512 << 20  # > 126 MB L2: flushed between timed steps, outside the event-timed region
OPS_PER_STEP = 40           # FP32/INT ops of one march iteration (algorithmic count)
OPS_PER_SAMPLE = 150        # ops of one traced sample outside the march (RNG, GGX, setup, gather)
SM_COUNT, FP32_LANES_PER_SM = 152, 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def workload():
    import ssgi_inputs as si
    return si.config3()


def config_dict(wl, extra=None):
    V, H, W = wl.depth.shape
    p = wl.params
    d = {"workload": f"{W}x{H} {p.spp}spp forward+backward, ground + 40 boxes + 2 tilted mirrors, "
                     f"env {wl.env.shape[0]}x{wl.env.shape[1]} log-normal, L2 loss to a U[0,1] target",
         "views": V, "height": H, "width": W, "spp": p.spp, "max_steps": p.max_steps, "hiz_levels": p.hiz_levels,
         "thickness": p.thickness, "rays_per_step": V * H * W * p.spp,
         "step": "env mips + Hi-Z + direct shade + trace (hits stored) + L2 loss + backward",
         "l2": "flushed between timed steps (512 MiB write outside the event-timed region)"}
    if extra:
        d.update(extra)
    return d


# ----------------------------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if s > 0.5 * (max(mx) if mx else 1)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------------------------
# peaks and profile summaries
# ----------------------------------------------------------------------------------------------
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("k_trace.cu", "ssgi_device.cuh", "ssgi_internal.h"):
        with open(os.path.join(ROOT, "paper_2504_01358_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """dram bytes per trace launch from the committed ncu summary, if taken on this source."""
    path = os.path.join(ROOT, "profiles", "k_trace_1600x900x16spp.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith(" "):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != kernel_source_hash():
            return None
        return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


# ----------------------------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ----------------------------------------------------------------------------------------------
def oracle_step(wl, lut):
    import oracle as O
    r = O.forward(wl, lut=lut)
    g_final = 2.0 * (r["final"] - wl.target) / r["final"].size
    He, We = wl.env.shape[:2]
    O.backward(wl.depth, wl.normal, wl.albedo, wl.rough, wl.metal, wl.cams, r["mips"], He, We, lut, r["c1"],
               r["hit_idx"], g_final, wl.params.spp, wl.params.seed, wl.params.flags)
    return r


def cpu_baseline(wl):
    import oracle as O
    lut = O.build_lut()
    t0 = time.perf_counter()
    oracle_step(wl, lut)
    dt = time.perf_counter() - t0
    V, H, W = wl.depth.shape
    rays = V * H * W * wl.params.spp
    return {"value": rays / dt, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
            "sample": f"one whole step of the same workload ({rays} rays: FP64 direct shading, Hi-Z, trace, "
                      f"Monte-Carlo sum and adjoint, OpenMP over pixels), {dt:.2f} s wall"}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle as O
    wl = workload()
    lut = O.build_lut()
    V, H, W = wl.depth.shape
    rays = V * H * W * wl.params.spp
    for _ in range(args.warmup):
        oracle_step(wl, lut)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_step(wl, lut)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = rays / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(wl, {"parallelism": "host cores (OpenMP)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
                             "sample": f"each step one whole fwd+bwd step of the workload ({rays} rays)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2504_01358_gb300 as S

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if world > 1:
            dist.barrier()

    wl = workload()
    V, H, W = wl.depth.shape
    p = S.params_of(wl.params)
    p.seed = p.seed + 1000 * rank  # each rank renders its own frame
    pipe = S.FramePipeline((V, H, W), wl.env.shape[:2], p, wl.cams)
    pipe.load(wl)
    rays = V * H * W * p.spp
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda", dtype=torch.float32)

    for _ in range(max(args.warmup, 3)):
        pipe.step()
    torch.cuda.synchronize()

    names = [n for n, _ in pipe.stages()]
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)] for _ in range(args.steps)]
    sampler = ClockSampler(torch.cuda.current_device())
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev = evs[k]
        ev[0].record(stream)
        for i, (_, fn) in enumerate(pipe.stages()):
            fn()
            ev[i + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()

    step_ms = [ev[0].elapsed_time(ev[-1]) for ev in evs]
    stage_ms = {n: statistics.mean(ev[i].elapsed_time(ev[i + 1]) for ev in evs) for i, n in enumerate(names)}
    ms = statistics.mean(step_ms)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * rays / (ms / 1e3)
    trace_ms = stage_ms["trace"]

    # march iterations of one trace launch (counted by the kernel itself, untimed)
    counter = torch.zeros(1, device="cuda", dtype=torch.int64)
    pipe.trace(step_count=counter)
    torch.cuda.synchronize()
    iters = int(counter.item())
    hit = pipe.hit_idx
    valid = int((hit >= -1).sum().item())

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        host = {n: torch.from_numpy(np.ascontiguousarray(getattr(wl, n))).pin_memory()
                for n in ("depth", "normal", "albedo", "rough", "metal", "env", "target")}
        out_final = torch.empty_like(pipe.final, device="cpu").pin_memory()
        out_loss = torch.empty(1).pin_memory()
        dst = {"depth": pipe.g.depth, "normal": pipe.g.normal, "albedo": pipe.g.albedo, "rough": pipe.g.rough,
               "metal": pipe.g.metal, "env": pipe.env, "target": pipe.target}
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        d2h = out_final.numel() * 4 + 4
        e_ms = []
        for k in range(args.warmup + args.steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for n, t in host.items():
                dst[n].copy_(t, non_blocking=True)
            pipe.step()
            out_final.copy_(pipe.final, non_blocking=True)
            out_loss.copy_(pipe.loss, non_blocking=True)
            b.record(stream)
            b.synchronize()
            if k >= args.warmup:
                e_ms.append(a.elapsed_time(b))
        em = statistics.mean(e_ms)
        if world > 1:
            t = torch.tensor([em], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            em = float(t.item())
        e2e = {"value": world * rays / (em / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": em}

    peaks, peak_src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = SM_COUNT * FP32_LANES_PER_SM * sm_max * 1e6 / 1e9  # Gop/s
    alg_ops = OPS_PER_STEP * iters + OPS_PER_SAMPLE * valid
    achieved = alg_ops / (trace_ms / 1e3) / 1e9
    traffic = profiled_traffic()
    roofline = {"kernel": "k_trace (ssgi_trace_indirect)", "bound": "alu", "achieved": achieved, "peak": alu_peak,
                "unit": "Gop/s", "frac": achieved / alu_peak, "traffic": traffic,
                "peak_source": f"derived: {SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_max:.0f} MHz "
                               f"({peak_src} max SM clock)",
                "work": f"{OPS_PER_STEP} ops x {iters} march iterations + {OPS_PER_SAMPLE} ops x {valid} traced samples",
                "trace_ms": trace_ms, "march_iterations": iters, "traced_samples": valid,
                "hbm_algorithmic_gbs": (V * H * W * (36 + 12 + 12) + 4 * V * H * W * p.spp) / (trace_ms / 1e3) / 1e9,
                "hbm_peak_gbs": float(peaks.get("hbm_gbs", 6800.0))}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(wl, {"parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}),
                "fwd_bwd_ms": ms, "trace_rays_per_s": rays / (trace_ms / 1e3),
                "stage_ms": stage_ms, "wall_s": t_wall,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": pipe.kernels_per_step() * args.steps, "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
