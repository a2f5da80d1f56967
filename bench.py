#!/usr/bin/env python
"""Benchmark of the SSGI hot path on GB300: one step = one inverse-rendering iteration of the
1600x900, 16 spp workload (environment mips -> Hi-Z -> direct shading -> Monte-Carlo screen-
space trace -> L2 loss -> backward), every stage a libssgi.so call.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  `value` is indirect rays per second through the whole step
(V*H*W*spp rays / step time), all ranks together; each rank renders its own frame (weak
scaling, no collective on the data path).  The line also carries the trace kernel's roofline
(ALU-bound; L2 and HBM figures from the committed ncu summary and the library's own bandwidth
probe), the end-to-end rate from pinned host buffers, the CPU oracle, the fused 8-view step
(ssgi_step_fused, one launch) next to its per-stage equivalent, and the serving run.
`--impl reference` times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import dataclasses
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
# The march is bound by the integer/logic ALU pipe (integer add/logic/shift, compares, min/max,
# selects): 16 lanes per SM sub-partition per clock, 64 per SM.  Its work is counted in ALU-pipe
# operations of the source: 29 per march iteration (15 in the cell test every iteration, 21 more
# on the 64 % of iterations that leave a cell, 1 on the rest that refine) and 100 per traced
# sample outside the march (Philox's 40, the sampler's and the ray set-up's compares and selects,
# the lookup's octant selection and texel indexing).
ALU_OPS_PER_ITER = 29
ALU_OPS_PER_SAMPLE = 100
SM_COUNT, ALU_LANES_PER_SM = 152, 64
SERVE_SUSTAINED_RATE, SERVE_SUSTAINED_REQUESTS = 250.0, 5000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rate", type=float, default=400.0)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-fused", action="store_true")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest of every rank's x (the slowest rank sets the job's time); x itself on one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Units all ranks processed per second when each rank does units_per_rank in ms (weak scaling)."""
    return world * units_per_rank / (ms / 1e3)


def rank_seed(seed: int, rank: int) -> int:
    """Each rank renders its own frame: a different sample sequence per rank."""
    return seed + 1000 * rank


def workload():
    import ssgi_inputs as si
    return si.config3()


def alu_peak_gops(sm_mhz: float) -> float:
    """ALU-pipe lane operations per second of the GPU (Gop/s)."""
    return SM_COUNT * ALU_LANES_PER_SM * sm_mhz * 1e6 / 1e9


def alu_achieved_gops(iterations: int, samples: int, trace_ms: float) -> float:
    """Algorithmic ALU-pipe operations of one trace launch per second (Gop/s)."""
    return (ALU_OPS_PER_ITER * iterations + ALU_OPS_PER_SAMPLE * samples) / (trace_ms / 1e3) / 1e9


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


class BusySampler:
    """nvidia-smi's utilization.gpu (share of each sample period in which a kernel was running)
    and SM clock sampled every 100 ms while a phase runs; stop() returns the mean busy share and
    keeps the median SM clock in `sm_mhz`."""

    def __init__(self, device_index: int):
        self.idx, self.proc, self.sm_mhz = device_index, None, None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=utilization.gpu,clocks.sm",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
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
        vals, mhz = [], []
        with open(self.path) as f:
            for ln in f:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) == 2 and all(x.replace(".", "").isdigit() for x in parts):
                    vals.append(float(parts[0]))
                    mhz.append(float(parts[1]))
        os.unlink(self.path)
        self.sm_mhz = statistics.median(mhz) if mhz else None
        return statistics.mean(vals) / 100.0 if vals else None


# ----------------------------------------------------------------------------------------------
# peaks and profile summaries
# ----------------------------------------------------------------------------------------------
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


TRACE_SOURCES = ("k_trace.cu", "ssgi_ops.cuh", "ssgi_device.cuh", "ssgi_internal.h")
TRACE_PROFILE = os.path.join(ROOT, "profiles", "k_trace_1600x900x16spp.txt")


def kernel_source_hash(files=TRACE_SOURCES) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2504_01358_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_summary(path=TRACE_PROFILE, files=TRACE_SOURCES):
    """`key: value` lines of a committed ncu summary, or None if it was taken on other source."""
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith((" ", "#")):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
                elif line.startswith("    ") and len(line.split()) == 2:  # "    metric   value"
                    k, v = line.split()
                    kv.setdefault(k, v)
        return kv if kv.get("kernel_source_sha256_16") == kernel_source_hash(files) else None
    except OSError:
        return None


def profiled(kv, key):
    try:
        return float(kv[key]) if kv else None
    except (KeyError, ValueError):
        return None


def probe_bandwidth():
    """L2 and HBM read ceilings from the library's own probe (ssgi_read_bandwidth_probe)."""
    import torch
    import paper_2504_01358_gb300 as S
    out = {}
    for name, nbytes, reps in (("l2", 32 << 20, 64), ("hbm", 4 << 30, 1)):
        buf = torch.empty(nbytes // 4, device="cuda", dtype=torch.float32).fill_(1.0)
        sink = torch.zeros(1, device="cuda", dtype=torch.int32)
        for _ in range(3):
            S.ssgi_read_bandwidth_probe(buf, reps, sink)
        torch.cuda.synchronize()
        ts = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            S.ssgi_read_bandwidth_probe(buf, reps, sink)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        out[name + "_read_gbs"] = nbytes * reps / (min(ts) / 1e3) / 1e9
        del buf
    out["method"] = ("ssgi_read_bandwidth_probe: 16-byte ld.global.cg from 8 blocks x 256 threads per SM; "
                     "l2 = a 32 MiB buffer read 64 times per launch, hbm = a 4 GiB buffer read once; best of 5")
    return out


def run_config1(flush):
    """Forward only (env mips, Hi-Z, direct shading, trace) of the 256x256, 4 spp, 32-step
    single view with a 64x128 map: 12 timed frames after 3 warm-up ones, L2 flushed before each."""
    import torch
    import ssgi_inputs as si
    import paper_2504_01358_gb300 as S
    wl = si.config1()
    V, H, W = wl.depth.shape
    p = S.params_of(wl.params)
    pipe = S.FramePipeline((V, H, W), wl.env.shape[:2], p, wl.cams)
    pipe.load(wl)
    stream = torch.cuda.current_stream()
    ts, tr = [], []
    for k in range(15):
        flush.fill_(float(k))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        pipe.env_mips()
        pipe.hiz_build()
        pipe.shade()
        ev[1].record(stream)
        pipe.trace()
        ev[2].record(stream)
        ev[2].synchronize()
        if k >= 3:
            ts.append(ev[0].elapsed_time(ev[2]))
            tr.append(ev[1].elapsed_time(ev[2]))
    ms, trace_ms = statistics.mean(ts), statistics.mean(tr)
    rays = V * H * W * p.spp
    return {"workload": f"{W}x{H} {p.spp}spp {p.max_steps} steps forward only, ground + 3 boxes, env "
                        f"{wl.env.shape[0]}x{wl.env.shape[1]} log-normal",
            "forward_ms": ms, "rays_per_s": rays / (ms / 1e3), "trace_ms": trace_ms,
            "trace_rays_per_s": rays / (trace_ms / 1e3), "launches_per_frame": pipe.kernels_per_step() - 4,
            "frames": len(ts), "l2": "flushed before each frame"}


def run_fused(steps: int, warmup: int):
    """The multi-view step (8 views at 1245x825, 32 spp, one 512x1024 env) as one
    launch (ssgi_step_fused) and, for comparison, as the per-stage calls."""
    import torch
    import ssgi_inputs as si
    import paper_2504_01358_gb300 as S
    wl = si.config4()
    V, H, W = wl.depth.shape
    p = S.params_of(wl.params)
    g, env, cams, tgt = S.to_device_workload(wl)
    lut = S.ssgi_build_brdf_lut()
    out = S.ssgi_step_fused(g, cams, env, lut, tgt, p)
    ws = out["_workspace"]

    def fused():
        S.ssgi_step_fused(g, cams, env, lut, tgt, p, out=out, workspace=ws)

    pipe = S.FramePipeline((V, H, W), wl.env.shape[:2], p, wl.cams, lut=lut)
    pipe.load(wl)

    def timed(fn):
        for _ in range(max(warmup, 3)):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.mean(ts)

    f_ms = timed(fused)
    if S.ssgi_step_fused_check(ws):
        raise RuntimeError("a block of the fused step gave up waiting for the previous phase")
    phases = {k: v / 1e6 for k, v in S.ssgi_step_fused_phase_ns(ws).items()}
    s_ms = timed(pipe.step)
    rays = V * H * W * p.spp
    return {"workload": f"{V} views x {W}x{H}, {p.spp} spp, 60-box scene on a ring of cameras, env "
                        f"{wl.env.shape[1]}x{wl.env.shape[0]}, forward + L2 loss + backward",
            "fused_ms": f_ms, "fused_rays_per_s": rays / (f_ms / 1e3), "fused_launches_per_step": 1,
            "fused_phase_ms": phases, "per_stage_ms": s_ms, "per_stage_rays_per_s": rays / (s_ms / 1e3),
            "per_stage_launches_per_step": pipe.kernels_per_step(), "steps": steps,
            "inputs": "G-buffer 296 MB + hit indices 1.05 GB per step: larger than L2, no flush needed"}


# ----------------------------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ----------------------------------------------------------------------------------------------
def oracle_step(wl, lut):
    import oracle as O
    r = O.forward(wl, lut=lut)
    g_final = 2.0 * (r["final"] - wl.target) / r["final"].size
    He, We = wl.env.shape[:2]
    r["grads"] = O.backward(wl.depth, wl.normal, wl.albedo, wl.rough, wl.metal, wl.cams, r["mips"], He, We, lut,
                            r["c1"], r["hit_idx"], g_final, wl.params.spp, wl.params.seed, wl.params.flags)
    return r


def parity_record(gpu, r):
    """The timed GPU step's outputs against the oracle's whole step on the same inputs, under the
    parity tests' rules: hit indices bit for bit per sample; pixels whose samples hit alike on
    both sides (and that no differing sample hits) compared per pixel, RGB |gpu - oracle|_inf /
    max(|oracle|_inf, 1e-3); their gradients against each buffer's scale (the environment's as a
    norm over all texels).  The pixels over 1e-4 are the rounding cases the parity tests replay at
    the GPU's own lookup coordinates."""
    import numpy as np
    hg, ho = gpu["hit_idx"], r["hit_idx"]
    bad = hg != ho
    aff = bad.any(axis=-1)
    W = hg.shape[2]
    for hh in (hg, ho):
        vv, yy, xx, ss = np.nonzero(bad & (hh >= 0))
        q = hh[vv, yy, xx, ss]
        aff[vv, q // W, q % W] = True
    ok = ~aff
    fin = gpu["final"].astype(np.float64)
    err = np.abs(fin - r["final"]).max(axis=-1) / np.maximum(np.abs(r["final"]).max(axis=-1), 1e-3)
    e = err[ok]
    grads = {}
    for k, g in gpu["grads"].items():
        o = r["grads"][k]
        d = np.abs(g.astype(np.float64) - o)
        if k == "env":
            grads[k] = float(np.linalg.norm(d) / max(float(np.linalg.norm(o)), 1e-30))
        else:
            m = ok if d.ndim == ok.ndim else ok[..., None]
            grads[k] = float(np.where(m, d, 0.0).max() / max(float(np.abs(np.where(m, o, 0.0)).max()), 1e-30))
    return {"hit_index_match": float((~bad).mean()), "pixels_with_a_differing_hit": int(aff.sum()),
            "pixels_compared": int(ok.sum()), "pixels_within_1e-4": float((e <= 1e-4).mean()),
            "pixels_over_1e-4": int((e > 1e-4).sum()), "max_pixel_rel_err": float(e.max()),
            "grad_max_err_over_scale": grads,
            "reference": "the oracle's last whole step above (FP64) against the timed step's final image, hit "
                         "indices and gradients (each side's own dL/dfinal)"}


def cpu_baseline(wl, gpu_out=None):
    """The oracle on the host cores: five whole steps at all cores, then the trace stage of a
    seeded 65,536-pixel sample at one thread (the same binary, FP64); with the timed GPU step's
    outputs, also their parity against the last of those steps."""
    import numpy as np
    import oracle as O
    lut = O.build_lut()
    cores = O.max_threads()
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        r = oracle_step(wl, lut)
    dt = (time.perf_counter() - t0) / reps
    V, H, W = wl.depth.shape
    p = wl.params
    rays = V * H * W * p.spp
    pl = np.sort(np.random.default_rng(7).choice(V * H * W, size=65536, replace=False))
    He, We = wl.env.shape[:2]
    O.set_threads(1)
    try:
        t1 = time.perf_counter()
        O.trace(wl.depth, wl.normal, wl.albedo, wl.rough, wl.metal, wl.cams, r["mips"], He, We, r["hiz"], r["c1"],
                r["cd"], p.spp, p.max_steps, p.hiz_levels, p.thickness, p.max_distance, p.seed, p.flags, pix_list=pl)
        dt1 = time.perf_counter() - t1
    finally:
        O.set_threads(cores)
    par = None if gpu_out is None else parity_record(gpu_out, r)
    return {"value": rays / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "parity": par,
            "sample": f"{reps} whole steps of the same workload ({rays} rays each: FP64 direct shading, Hi-Z, "
                      f"trace, Monte-Carlo sum and adjoint, OpenMP over pixels), {dt:.2f} s wall per step",
            "single_thread": {"value": len(pl) * p.spp / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"trace stage only (march + Monte-Carlo sum) of 65536 seeded random pixels "
                                        f"x {p.spp} spp at one thread, {dt1:.2f} s wall"}}


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
# serving (Poisson request stream, mixed resolutions and sample counts)
# ----------------------------------------------------------------------------------------------
SERVE_RES = [(360, 640), (720, 1280), (900, 1600), (1080, 1920)]
SERVE_SPP = [4, 8, 16, 32]


def serving_workload(n_requests: int, rate: float, seed: int = 5):
    """Request list of the serving configuration: Poisson arrivals at `rate`/s, resolution and
    spp uniform over the four choices, seeded scenes (config-2 generator) and 128x256
    log-normal environments drawn from pools of 4 scenes per resolution and 32 maps."""
    import numpy as np
    import ssgi_inputs as si
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    res = rng.integers(0, len(SERVE_RES), size=n_requests)
    spp = rng.choice(SERVE_SPP, size=n_requests)
    scenes = {}
    for r, (H, W) in enumerate(SERVE_RES):
        for k in range(4):
            scenes[(r, k)] = si.single_view(f"serve-{W}x{H}-{k}", 100 + 10 * r + k, H, W, 40, 8.0, 2, (128, 256),
                                            si.TraceParams(spp=4, max_steps=64))
    envs = [si.lognormal_env(5000 + j, 128, 256) for j in range(32)]
    reqs = [dict(arrival=float(arrivals[i]), scene=scenes[(int(res[i]), i % 4)], env=envs[i % 32], spp=int(spp[i]),
                 seed=i, res=int(res[i])) for i in range(n_requests)]
    return reqs


def run_serving(n_requests: int, rate: float, slots: int, budget_gb: float, with_resident: bool = False):
    import numpy as np
    import torch

    import paper_2504_01358_gb300 as S
    from paper_2504_01358_gb300 import _native as N
    from paper_2504_01358_gb300.serve import Server

    reqs = serving_workload(n_requests, rate)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    host = {}
    for rq in reqs:
        wl = rq["scene"]
        if id(wl) not in host:
            host[id(wl)] = {k: pin(getattr(wl, k)) for k in ("depth", "normal", "albedo", "rough", "metal")}
    envs = {}
    for rq in reqs:
        if id(rq["env"]) not in envs:
            envs[id(rq["env"])] = pin(rq["env"])
    ring = 64
    outs = {r: [torch.empty((1, H, W, 3)).pin_memory() for _ in range(ring)] for r, (H, W) in enumerate(SERVE_RES)}

    def params(rq):
        return S.TraceParams(spp=rq["spp"], max_steps=64, hiz_levels=8, thickness=0.05, max_distance=100.0,
                             seed=rq["seed"], flags=0)

    rays = sum(rq["spp"] * rq["scene"].depth.size for rq in reqs)

    # ---- served: continuous batching --------------------------------------------------------
    def serve_stream(resident: bool):
        """The request stream through one server: each request ships its G-buffer (resident=False)
        or names one of the pool's scenes registered before the stream (resident=True: G-buffer and
        Hi-Z stay on the device).  Returns (latencies in s, span, busy share, SM MHz, stats)."""
        srv = Server(int(budget_gb * (1 << 30)), max_slots=slots, queue_capacity=n_requests + 16)
        sid = {}
        if resident:
            for rq in reqs:
                wl = rq["scene"]
                if id(wl) not in sid:
                    h = host[id(wl)]
                    sid[id(wl)] = srv.scene_add(h["depth"], h["normal"], h["albedo"], h["rough"], h["metal"], wl.cams, 8)

        def submit(rq, out):
            if resident:
                return srv.submit(out, envs[id(rq["env"])], params(rq), scene=sid[id(rq["scene"])])
            h = host[id(rq["scene"])]
            return srv.submit(out, envs[id(rq["env"])], params(rq), depth=h["depth"], normal=h["normal"],
                              albedo=h["albedo"], rough=h["rough"], metal=h["metal"], cams=rq["scene"].cams)

        # warm up every resolution once
        for r in range(len(SERVE_RES)):
            rc, t = submit(next(q for q in reqs if q["res"] == r), outs[r][0])
            srv.wait(t, 60000)
        tickets = []
        busy = BusySampler(torch.cuda.current_device())
        busy.start()
        t0 = time.perf_counter()
        for i, rq in enumerate(reqs):
            while time.perf_counter() - t0 < rq["arrival"]:
                pass
            t_sub = time.perf_counter() - t0
            rc, t = submit(rq, outs[rq["res"]][i % ring])
            if rc != N.OK:
                raise RuntimeError(f"submit failed: {N.STATUS.get(rc, rc)}")
            tickets.append((t, t_sub))
        lat = []
        for (t, t_sub), rq in zip(tickets, reqs):
            rc, ms = srv.wait(t, 600000)
            if rc != N.OK:
                raise RuntimeError(f"request failed: {N.STATUS.get(rc, rc)}")
            lat.append(t_sub - rq["arrival"] + ms / 1e3)
        span = max(rq["arrival"] + l for rq, l in zip(reqs, lat)) - reqs[0]["arrival"]
        share = busy.stop()
        st = srv.stats()
        srv.close()
        return lat, span, share, busy.sm_mhz, st

    lat, served_span, served_busy, served_mhz, st = serve_stream(False)
    res_run = serve_stream(True) if with_resident else None

    # ---- plain: one request at a time, synchronous, preallocated buffers --------------------
    Hm, Wm = max(SERVE_RES)
    f = lambda *sh: torch.empty(sh, device="cuda")  # noqa: E731
    g = S.GBuffer(f(1, Hm, Wm), f(1, Hm, Wm, 3), f(1, Hm, Wm, 3), f(1, Hm, Wm), f(1, Hm, Wm))
    env_d = f(128, 256, 3)
    em = S.EnvMap(f(S.ssgi_env_mip_floats(128, 256)), 128, 256)
    hiz = f(S.ssgi_hiz_floats((1, Hm, Wm), 8))
    c_d, c1, fin = f(1, Hm, Wm, 3), f(1, Hm, Wm, 3), f(1, Hm, Wm, 3)
    lut = S.ssgi_build_brdf_lut()
    stream = torch.cuda.current_stream()

    def plain_one(rq, out):
        wl = rq["scene"]
        H, W = wl.depth.shape[1:]
        n = H * W
        h = host[id(wl)]
        gv = S.GBuffer(g.depth.view(-1)[:n].view(1, H, W), g.normal.view(-1)[:3 * n].view(1, H, W, 3),
                       g.albedo.view(-1)[:3 * n].view(1, H, W, 3), g.rough.view(-1)[:n].view(1, H, W),
                       g.metal.view(-1)[:n].view(1, H, W))
        for k in ("depth", "normal", "albedo", "rough", "metal"):
            getattr(gv, k).copy_(h[k], non_blocking=True)
        env_d.copy_(envs[id(rq["env"])], non_blocking=True)
        S.ssgi_build_env_mips(env_d, out=em.mips)
        hz = hiz[: S.ssgi_hiz_floats((1, H, W), 8)]
        S.ssgi_build_hiz(gv.depth, 8, out=hz)
        cd = c_d.view(-1)[:3 * n].view(1, H, W, 3)
        cc = c1.view(-1)[:3 * n].view(1, H, W, 3)
        ff = fin.view(-1)[:3 * n].view(1, H, W, 3)
        S.ssgi_shade_direct(gv, wl.cams, em, lut, c_d=cd, c1=cc)
        S.ssgi_trace_indirect(gv, wl.cams, hz, cc, cd, em, params(rq), final=ff)
        out.copy_(ff, non_blocking=True)
        stream.synchronize()

    for r in range(len(SERVE_RES)):
        rq = next(q for q in reqs if q["res"] == r)
        plain_one(rq, outs[r][0])
    plat = []
    busy = BusySampler(torch.cuda.current_device())
    busy.start()
    t0 = time.perf_counter()
    for i, rq in enumerate(reqs):
        while time.perf_counter() - t0 < rq["arrival"]:
            pass
        plain_one(rq, outs[rq["res"]][i % ring])
        plat.append(time.perf_counter() - t0 - rq["arrival"])
    plain_span = max(rq["arrival"] + l for rq, l in zip(reqs, plat)) - reqs[0]["arrival"]
    plain_busy = busy.stop()
    plain_mhz = busy.sm_mhz

    def pct(a, q):
        import numpy as np
        return float(np.percentile(np.asarray(a) * 1e3, q))

    return {"requests": n_requests, "arrival_rate_per_s": rate, "slots": slots, "hbm_budget_gb": budget_gb,
            "offered_rays_per_s": rays / reqs[-1]["arrival"],
            "served": {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "mean_ms": 1e3 * sum(lat) / len(lat),
                       "throughput_req_per_s": n_requests / served_span, "rays_per_s": rays / served_span,
                       "arena_peak_gb": st["arena_bytes_peak"] / 2 ** 30, "gpu_busy_share": served_busy,
                       "sm_mhz_median": served_mhz},
            "plain": {"p50_ms": pct(plat, 50), "p99_ms": pct(plat, 99), "mean_ms": 1e3 * sum(plat) / len(plat),
                      "throughput_req_per_s": n_requests / plain_span, "rays_per_s": rays / plain_span,
                      "gpu_busy_share": plain_busy, "sm_mhz_median": plain_mhz},
            "p99_plain_over_served": pct(plat, 99) / max(pct(lat, 99), 1e-9),
            "served_resident": None if res_run is None else {
                "p50_ms": pct(res_run[0], 50), "p99_ms": pct(res_run[0], 99),
                "mean_ms": 1e3 * sum(res_run[0]) / len(res_run[0]), "throughput_req_per_s": n_requests / res_run[1],
                "gpu_busy_share": res_run[2], "sm_mhz_median": res_run[3],
                "p99_plain_over_served": pct(plat, 99) / max(pct(res_run[0], 99), 1e-9),
                "scenes": "the pool's 16 scenes registered once before the stream (ssgi_serve_scene_add: "
                          "G-buffer and Hi-Z resident); each request ships only its map and names its scene"},
            "workload": "Poisson arrivals, resolution uniform over 640x360/1280x720/1600x900/1920x1080, spp uniform "
                        "over 4/8/16/32, scenes from the config-2 generator (pool of 4 per resolution), 128x256 "
                        "log-normal env maps (pool of 32), 64 steps, 8 levels; latency = arrival to result on host"}


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
    p.seed = rank_seed(p.seed, rank)
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
    ms = max_over_ranks(ms, world)
    value = whole_job_rate(rays, world, ms)
    trace_ms = stage_ms["trace"]
    launches = pipe.kernels_per_step() * args.steps
    # the timed step's outputs, for the oracle's parity record (rank 0 at one GPU only)
    gpu_out = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        gpu_out = {"final": pipe.final.cpu().numpy(), "hit_idx": pipe.hit_idx.cpu().numpy(),
                   "grads": {k: v.cpu().numpy() for k, v in pipe.grads.items()}}

    # the pathwise adjoint (SSGI_PATHWISE) of the same frame next to the replay one (untimed in the step)
    from paper_2504_01358_gb300._native import PATHWISE as N_PATHWISE
    def adjoint_ms(flags):
        saved = pipe.params.flags
        pipe.params.flags = flags
        try:
            for _ in range(3):
                pipe.adjoint()
            ts = []
            for k in range(10):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                pipe.adjoint()
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            return statistics.mean(ts)
        finally:
            pipe.params.flags = saved

    adjoints = {"replay_ms": adjoint_ms(p.flags), "pathwise_ms": adjoint_ms(p.flags | N_PATHWISE),
                "note": "ssgi_backward on the same frame and hit indices, 10 calls each, L2 flushed before each"}

    # depth normals of the same frame (Sec. 3.1; 4 B read + 12 B written per pixel, HBM-bound)
    nrm = torch.empty_like(pipe.g.normal)
    ts = []
    for k in range(13):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        S.ssgi_depth_normals(pipe.g.depth, pipe.cam, out=nrm)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    dn_ms = statistics.mean(ts[3:])

    def timed_ms(fn, n=13, skip=3):
        out = []
        for k in range(n):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return statistics.mean(out[skip:])

    # the normals fused into the pyramid's pass over depth, against the two passes
    sep_ms = timed_ms(lambda: (S.ssgi_build_hiz(pipe.g.depth, p.hiz_levels, out=pipe.hiz),
                               S.ssgi_depth_normals(pipe.g.depth, pipe.cam, out=nrm)))
    fus_ms = timed_ms(lambda: S.ssgi_build_hiz_normals(pipe.g.depth, pipe.cam, p.hiz_levels, hiz=pipe.hiz,
                                                        normals=nrm))
    depth_normals = {"ms": dn_ms, "algorithmic_bytes": 16 * V * H * W,
                     "achieved_gbs": 16 * V * H * W / (dn_ms / 1e3) / 1e9, "launches": 1,
                     "note": "ssgi_depth_normals at the step's frame, L2 flushed before each of 10 timed calls",
                     "with_pyramid": {"separate_ms": sep_ms, "separate_launches": 3, "fused_ms": fus_ms,
                                      "fused_launches": 2,
                                      "note": "ssgi_build_hiz + ssgi_depth_normals vs ssgi_build_hiz_normals "
                                              "(one read of depth), same outputs bit for bit"}}
    del nrm

    # object insertion into the same frame (Sec. 4): a floating box rendered on its own and merged
    # by depth into a separate G-buffer (76 B per pixel: both depths, the winning side's other
    # 32 B, 36 B written; HBM-bound)
    import ssgi_inputs as si
    box = si.Box(np.array([-1.5, 0.3, -1.0]), np.array([1.5, 2.0, 1.0]), si.Material((0.8, 0.3, 0.2), 0.4, 0.0))
    og = si.raycast_gbuffer(si.Scene(None, 40.0, [box], []), wl.cams[0], H, W)
    obj = S.GBuffer(*(torch.from_numpy(np.ascontiguousarray(og[k][None], np.float32)).cuda()
                      for k in ("depth", "normal", "albedo", "rough", "metal")))
    cout = S.GBuffer(*(torch.empty_like(getattr(pipe.g, k)) for k in ("depth", "normal", "albedo", "rough", "metal")))
    ts = []
    for k in range(13):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        S.ssgi_composite_gbuffer(pipe.g, obj, out=cout)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    cm_ms = statistics.mean(ts[3:])
    composite = {"ms": cm_ms, "object_pixel_share": float(np.isfinite(og["depth"]).mean()),
                 "algorithmic_bytes": 76 * V * H * W, "achieved_gbs": 76 * V * H * W / (cm_ms / 1e3) / 1e9,
                 "launches": 1, "note": "ssgi_composite_gbuffer into separate planes at the step's frame, "
                                        "L2 flushed before each of 10 timed calls"}
    del obj, cout

    # output transform of the same frame (Sec. 3.3): sRGB tone map (12 B in + 12 B out per pixel)
    # and the sRGB L2 loss with its gradient (24 B in + 12 B out per pixel)
    def epilogue_ms(fn):
        ts = []
        for k in range(13):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.mean(ts[3:])

    srgb = torch.empty_like(pipe.final)
    gfs = torch.empty_like(pipe.final)
    tm_ms = epilogue_ms(lambda: S.ssgi_tonemap_srgb(pipe.final, out=srgb))
    ls_ms = epilogue_ms(lambda: S.ssgi_l2_loss_srgb(pipe.final, pipe.target, g_final=gfs, loss=pipe.loss))
    # the transform as the trace's epilogue (SSGI_SRGB_FINAL) against trace + separate pass
    from paper_2504_01358_gb300._native import SRGB_FINAL as N_SRGB_FINAL
    p_srgb = S.TraceParams(p.spp, p.max_steps, p.hiz_levels, p.thickness, p.max_distance, p.seed,
                           p.flags | N_SRGB_FINAL)
    two_ms = epilogue_ms(lambda: (pipe.trace(), S.ssgi_tonemap_srgb(pipe.final, out=srgb)))
    one_ms = epilogue_ms(lambda: S.ssgi_trace_indirect(pipe.g, pipe.cam, pipe.hiz, pipe.c1, pipe.c_d, pipe.em, p_srgb,
                                                       final=srgb, hit_idx=pipe.hit_idx))
    output_transform = {"tonemap_ms": tm_ms, "tonemap_gbs": 24 * V * H * W / (tm_ms / 1e3) / 1e9,
                        "srgb_loss_ms": ls_ms, "srgb_loss_gbs": 36 * V * H * W / (ls_ms / 1e3) / 1e9,
                        "trace_then_tonemap_ms": two_ms, "trace_with_srgb_epilogue_ms": one_ms,
                        "note": "ssgi_tonemap_srgb and ssgi_l2_loss_srgb at the step's frame, L2 flushed; the "
                                "trace with SSGI_SRGB_FINAL writes the display image itself (same bits)"}
    del srgb, gfs

    # the small single-view workload (256x256, 4 spp, 32 steps, 64x128 map): forward only
    cfg1 = run_config1(flush)

    # march iterations of one trace launch (counted by the kernel itself, untimed)
    counter = torch.zeros(1, device="cuda", dtype=torch.int64)
    pipe.trace(step_count=counter)
    torch.cuda.synchronize()
    iters = int(counter.item())
    hit = pipe.hit_idx
    valid = int((hit >= -1).sum().item())
    # rays the step budget stopped: with one more step allowed every ray repeats its iterations
    # and exactly those rays take one more, so the difference of the two totals counts them
    counter1 = torch.zeros(1, device="cuda", dtype=torch.int64)
    S.ssgi_trace_indirect(pipe.g, pipe.cam, pipe.hiz, pipe.c1, pipe.c_d, pipe.em,
                          S.params_of(dataclasses.replace(wl.params, max_steps=wl.params.max_steps + 1)),
                          step_count=counter1)
    torch.cuda.synchronize()
    exhausted = int(counter1.item()) - iters

    # end to end through the C ABI from pinned host buffers: every step's inputs go up and its
    # final image and loss come back inside the timed region
    e2e = None
    if not args.no_e2e:
        keys = ("depth", "normal", "albedo", "rough", "metal", "env", "target")
        host = {n: torch.from_numpy(np.ascontiguousarray(getattr(wl, n))).pin_memory() for n in keys}
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        d2h = pipe.final.numel() * 4 + 4

        def buffers(pp):
            return {"depth": pp.g.depth, "normal": pp.g.normal, "albedo": pp.g.albedo, "rough": pp.g.rough,
                    "metal": pp.g.metal, "env": pp.env, "target": pp.target}

        # (1) one step at a time: upload, step, read back, wait
        out_final = torch.empty_like(pipe.final, device="cpu").pin_memory()
        out_loss = torch.empty(1).pin_memory()
        dst = buffers(pipe)
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
        serial_ms = max_over_ranks(statistics.mean(e_ms), world)

        # (2) streamed frames: two buffer sets; the inputs of step k+1 go up on a copy stream while
        # step k computes, and step k's results come back as soon as it is done.  The copy stream
        # is in order, so a buffer set is uploaded again only after its last results were read.
        pipes = [pipe, S.FramePipeline((V, H, W), wl.env.shape[:2], p, wl.cams, lut=pipe.lut)]
        dsts = [buffers(pp) for pp in pipes]
        outs = [(torch.empty_like(pipe.final, device="cpu").pin_memory(), torch.empty(1).pin_memory())
                for _ in range(2)]
        copy = torch.cuda.Stream()
        up = [torch.cuda.Event(), torch.cuda.Event()]
        done = [torch.cuda.Event(), torch.cuda.Event()]

        def upload(b):
            with torch.cuda.stream(copy):
                for n, t in host.items():
                    dsts[b][n].copy_(t, non_blocking=True)
            up[b].record(copy)

        def run(nsteps):
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            copy.wait_stream(stream)
            upload(0)
            for k in range(nsteps):
                b = k & 1
                stream.wait_event(up[b])
                pipes[b].step(stream=stream)
                done[b].record(stream)
                if k + 1 < nsteps:
                    upload(1 - b)
                copy.wait_event(done[b])
                with torch.cuda.stream(copy):
                    outs[b][0].copy_(pipes[b].final, non_blocking=True)
                    outs[b][1].copy_(pipes[b].loss, non_blocking=True)
            stream.wait_stream(copy)
            t1.record(stream)
            t1.synchronize()
            return t0.elapsed_time(t1) / nsteps

        run(max(args.warmup, 3))
        # the median of three runs: the copies share the host's memory and link with other work on
        # the machine, which once stretched one run by a quarter
        em = max_over_ranks(statistics.median(run(args.steps) for _ in range(3)), world)
        e2e = {"value": whole_job_rate(rays, world, em), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": em,
               "mode": "streamed frames: pinned host inputs of step k+1 uploaded on a copy stream while step k "
                       "computes, each step's final image and loss read back when it is done (two buffer sets); "
                       "no L2 flush: every step's inputs arrive by a fresh host-to-device copy; the median of "
                       "three runs of the timed step count",
               "serial": {"value": whole_job_rate(rays, world, serial_ms), "ms_per_step": serial_ms,
                          "mode": "upload, step, read back, wait; L2 flushed before each step"}}
        del pipes, dsts, outs

    peaks, peak_src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = alu_peak_gops(sm_max)
    achieved = alu_achieved_gops(iters, valid, trace_ms)
    prof = profile_summary()
    traffic = profiled(prof, "dram_bytes_per_launch")
    bw = probe_bandwidth()
    l2_bytes = profiled(prof, "lts_bytes_per_launch")
    roofline = {"kernel": "k_trace (ssgi_trace_indirect)", "bound": "alu", "achieved": achieved, "peak": alu_peak,
                "unit": "Gop/s", "frac": achieved / alu_peak, "traffic": traffic,
                "peak_source": f"derived: {SM_COUNT} SMs x {ALU_LANES_PER_SM} integer/logic ALU-pipe lanes x "
                               f"{sm_max:.0f} MHz ({peak_src} max SM clock)",
                "work": {"alu_ops_per_march_iteration": ALU_OPS_PER_ITER, "alu_ops_per_traced_sample": ALU_OPS_PER_SAMPLE,
                         "march_iterations": iters, "traced_samples": valid,
                         "achieved = (ops_per_iteration x iterations + ops_per_sample x samples) / trace_ms": True},
                "trace_ms": trace_ms, "march_iterations": iters, "traced_samples": valid,
                "budget_exhausted_rays": exhausted, "budget_exhausted_share": exhausted / max(valid, 1),
                "hbm_algorithmic_gbs": (V * H * W * (36 + 12 + 12) + 4 * V * H * W * p.spp) / (trace_ms / 1e3) / 1e9,
                "hbm_peak_gbs": float(peaks.get("hbm_gbs", 6800.0)),
                "l2_achieved_gbs": None if l2_bytes is None else l2_bytes / (trace_ms / 1e3) / 1e9,
                "l2_peak_gbs": bw["l2_read_gbs"],
                "warp_execution_efficiency": profiled(prof, "warp_execution_efficiency"),
                # the pipe that bounds the march (integer/logic ALU) and issue, as ncu measured them
                "alu_pipe_busy_pct": profiled(prof, "alu_pipe_pct"),
                "issue_active_pct": profiled(prof, "issue_active_pct"),
                "profile": None if prof is None else os.path.relpath(TRACE_PROFILE, ROOT)}

    fused = None
    if rank == 0 and world == 1 and not args.no_fused:
        del pipe
        torch.cuda.empty_cache()
        fused = run_fused(10, 3)
        torch.cuda.empty_cache()
        pipe = None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, gpu_out)
    serving = serving_sustained = None
    if rank == 0 and not args.no_serving:
        pipe = None
        torch.cuda.empty_cache()
        serving = run_serving(args.serve_requests, args.serve_rate, args.serve_slots, 100.0)
        # a load the plain path also sustains, so that its latency is not a growing queue
        serving_sustained = run_serving(SERVE_SUSTAINED_REQUESTS, SERVE_SUSTAINED_RATE, args.serve_slots, 100.0,
                                        with_resident=True)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(wl, {"parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}),
                "fwd_bwd_ms": ms, "trace_rays_per_s": rays / (trace_ms / 1e3),
                "stage_ms": stage_ms, "wall_s": t_wall,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks, "bandwidth_probe": bw, "adjoint_modes": adjoints,
                "config1_forward": cfg1,
                "depth_normals": depth_normals, "object_insertion": composite,
                "output_transform": output_transform,
                "fused_step": fused,
                "serving": serving, "serving_sustained": serving_sustained}
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
