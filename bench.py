#!/usr/bin/env python3
"""Benchmark of the bricked multi-resolution raycaster on GB300.

Default workload (one step = one frame of the whole hot path):
  1024^3 uint16 fractal value noise (5 octaves) + 200 spheres (r 4..60), 64^3 bricks with apron,
  5 LOD levels built on the GPU, footprint LOD, 1920x1080 orbit view at a seeded angle, 45 deg FOV,
  step 0.5 voxel, 256-entry RGBA TF with 3 seeded opacity peaks, early termination at 0.99.
The metric is composited ray samples per second (and ms per frame).  The primary line renders
from uint16 bricks; the binary16 store of the same volume and a float32 store ("plain FP32 path")
are timed beside it, and the differentiable workload (forward + adjoint) adds a fwd+bwd figure.

--impl reference times the FP64 CPU oracle on a bounded seeded pixel sample of the same frame.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

L2_FLUSH_BYTES = 256 << 20


# ------------------------------------------------------------------ workloads

from synth import workloads  # noqa: E402


# ------------------------------------------------------------------ helpers

class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1])); mx.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        finally:
            os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def render_kernel_digest():
    h = hashlib.sha256()
    for f in ("kernels_render.cu", "render_common.cuh", "internal.cuh"):
        with open(os.path.join(ROOT, "paper_2509_26213_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_counter(workload_key, what):
    """A per-launch figure from the committed ncu summary (`what` is the line's label: "dram bytes"
    or "warp instructions"), if the summary was taken on this kernel source."""
    path = os.path.join(ROOT, "profiles", f"raycast_fwd_{workload_key}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_src = re.search(r"kernel source digest:\s*([0-9a-f]+)", text)
    m_b = re.search(what + r" per launch \(scaled to the bench frame\):\s*([0-9.eE+]+)", text)
    if m_src and m_b and m_src.group(1) == render_kernel_digest():
        return float(m_b.group(1))
    return None


def recorded_traffic(workload_key):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this kernel source."""
    return recorded_counter(workload_key, "dram bytes")


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        return dist, rank, ws, local
    return None, rank, ws, local


def barrier(dist):
    if dist:
        dist.barrier()


def max_over_ranks(dist, x):
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, x):
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ workload helpers

def load_workload(key, rank=0, ws=1):
    wl = getattr(workloads, key)()
    if ws > 1:
        # weak scaling: every rank renders its own frame (views rotated per rank); no collective
        wl["cams"] = [synth.seeded_orbit(wl["D"], c["w"], c["h"], 11 + rank, view=i) for i, c in enumerate(wl["cams"])]
    return wl


def oracle_volume(wl, raw):
    import oracle
    oracle.build()
    store = wl["store"]
    if (wl["src"], store) == ("u16", "f16"):
        raw = oracle.u16_to_f16(raw)
    return oracle.Volume(oracle.pyramid(raw, wl["levels"], store), store, wl["brick"])


def frame_pixels(wl, frac, seed):
    """A seeded sample of every view's pixels: [(view, pixels[n,2])]."""
    out = []
    for v, cam in enumerate(wl["cams"]):
        n = max(1, int(cam["w"] * cam["h"] * frac))
        out.append((v, synth.pixel_subset(cam["w"], cam["h"], n, seed * 1000 + v)))
    return out


def oracle_samples(ovol, wl, parts):
    import oracle
    tot = 0
    for v, pix in parts:
        tot += int(oracle.render(ovol, wl["cams"][v], wl["tf"], wl["params"], pixels=pix)["n"].sum())
    return tot


# ------------------------------------------------------------------ reference arm (the oracle)

def run_reference(args, dist, rank, ws):
    if rank != 0:
        return
    import oracle
    wl = load_workload(args.workload)
    t0 = time.time()
    ovol = oracle_volume(wl, wl["make"]())
    prep = time.time() - t0
    threads = oracle.threads()
    frac = args.ref_frac
    for i in range(args.warmup):
        oracle_samples(ovol, wl, frame_pixels(wl, frac / 16, 500 + i))
    times, samples = [], 0
    for i in range(args.steps):
        parts = frame_pixels(wl, frac, 2000 + i)
        t = time.perf_counter()
        samples += oracle_samples(ovol, wl, parts)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = samples / total
    sample = f"{frac:g} of every view's pixels per step (seeded, new each step), {args.steps} steps"
    line = {
        "impl": "reference", "metric": "ray samples/s", "value": value, "unit": "samples/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl["name"], "store": wl["store"], "sample": sample},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "prep_s": prep,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def build_volume(P, wl, store, raw):
    vol = P.Volume(wl["D"], store, wl["brick"], wl["levels"])
    vol.upload_level(0, raw, wl["src"])
    if wl["levels"] > 1:
        vol.build_lod(0)
    return vol


def time_frames(torch, vol, cams, tf, params, steps, warmup, flush, grad=False, drgba=None, dtf=None, dvox=None):
    """Per-step CUDA-event times (ms) of one frame; L2 flushed before every step (not timed)."""
    for _ in range(warmup):
        vol.render(cams, tf, params, grad=grad)
        if grad:
            vol.render_backward(drgba, dtf, dvox)
    torch.cuda.synchronize()
    evs = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        vol.render(cams, tf, params, grad=grad)
        if grad:
            vol.render_backward(drgba, dtf, dvox)
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def bytes_per_voxel(store):
    return {"u8": 1, "u16": 2, "f16": 2, "f32": 4}[store]


def run_ours(args, dist, rank, ws, local):
    import torch
    import paper_2509_26213_gb300 as pkg
    pkg.build()
    import paper_2509_26213_gb300.volume as P

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = load_workload(args.workload, rank, ws)
    raw = wl["make"]()
    cams, params = wl["cams"], dict(wl["params"])
    tf = torch.from_numpy(wl["tf"]).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    store = wl["store"]
    bpv = bytes_per_voxel(store)

    tuned = None
    if args.workload == "c3" or args.autotune:
        # ray-tile shape, refill threshold and brick size chosen by the autotuner (untimed)
        from paper_2509_26213_gb300.tune import autotune
        cache = os.environ.get("VOLRC_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "volrc_autotune.json"))
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tuned = autotune(lambda b: build_volume(P, dict(wl, brick=b), store, raw), cams, tf, params,
                         key=f"{wl['key']}|{wl['name']}", cache_path=cache)
        wl["brick"] = tuned["brick"]
        params.update(tile_w=tuned["tile_w"], tile_h=tuned["tile_h"], refill=tuned["refill"])
    vol = (tuned or {}).pop("volume", None) or build_volume(P, wl, store, raw)
    out, ns = vol.render(cams, tf, params, nsamples=True)
    torch.cuda.synchronize()
    samples = int(ns.sum().item())
    touched = vol.stats()["touched"]
    npx = sum(c["w"] * c["h"] for c in cams)

    barrier(dist)
    with Clocks(local) as clk:
        wall0 = time.perf_counter()
        ms = time_frames(torch, vol, cams, tf, params, args.steps, args.warmup, flush)
        wall = time.perf_counter() - wall0
    launches_per_frame = vol.stats()["launches"]  # library kernels of one render (the last timed one)
    clocks = clk.summary()
    t_mean = statistics.mean(ms)
    t_step = max_over_ranks(dist, t_mean)
    total_samples = sum_over_ranks(dist, samples)
    value = total_samples / (t_step * 1e-3)

    # end to end through the public API with host buffers: TF up, image down, every step.  The
    # image goes to page-locked host memory that the render kernel writes directly (through the
    # host link), so no separate copy follows the render.
    tf_host = torch.from_numpy(wl["tf"]).pin_memory()
    img_host = torch.empty((npx, 4), dtype=torch.float32).pin_memory()
    tf_dev = torch.empty_like(tf)
    for _ in range(args.warmup):
        tf_dev.copy_(tf_host, non_blocking=True)
        vol.render(cams, tf_dev, params, out=img_host)
    torch.cuda.synchronize()
    barrier(dist)
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        tf_dev.copy_(tf_host, non_blocking=True)
        vol.render(cams, tf_dev, params, out=img_host)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t))
    e2e_step = max_over_ranks(dist, statistics.mean(e2e_ms))
    e2e_value = total_samples / (e2e_step * 1e-3)

    # roofline of the render kernel: algorithmic bytes = bricks touched + image + TF + page-table words
    b_unique = touched * (wl["brick"] + 1) ** 3 * bpv + npx * 16 + 4096 + touched * 4
    b_sample = samples * (8 * bpv + 4)
    peak, peak_kind = measured_peaks()
    achieved = b_unique / (t_mean * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": recorded_traffic(wl["key"]), "peak_kind": f"{peak_kind} hbm_gbs (copy, burst)",
                "kernel": "k_render",
                "bytes_accounting": "bricks touched x (B+1)^3 x bytes/voxel + image 16 B/px + TF 4 KiB + 4 B/brick page-table word",
                "bytes_per_frame": b_unique,
                "per_sample_gather_GBps": b_sample / (t_mean * 1e-3) / 1e9}
    # the bound the kernel actually meets: instruction issue (one warp instruction per scheduler
    # and clock: 152 SMs x 4 schedulers at the sampled SM clock), from the recorded warp
    # instructions of one launch
    winst = recorded_counter(wl["key"], "warp instructions")
    if winst and clocks.get("sm_mhz"):
        issue_peak = 152 * 4 * clocks["sm_mhz"] * 1e6
        roofline["issue"] = {"achieved_warp_inst_per_s": winst / (t_mean * 1e-3), "peak_warp_inst_per_s": issue_peak,
                             "frac": winst / (t_mean * 1e-3) / issue_peak, "warp_inst_per_frame": winst,
                             "peak_kind": "152 SMs x 4 schedulers x sampled SM clock"}

    variants = {}
    # empty-space skipping (the paper's ES column): same image and sample counts, less work
    ms_es = time_frames(torch, vol, cams, tf, dict(params, flags=2), max(5, args.steps // 4), args.warmup, flush)
    variants["skip_empty"] = {"ms_per_frame": statistics.mean(ms_es),
                              "samples_per_s": samples / (statistics.mean(ms_es) * 1e-3)}
    if params.get("lod_mode"):
        # level-scaled sampling: coarse levels take steps of dt 2^l with corrected opacity (a
        # different, cheaper image of the same volume; reported beside the default line)
        pl = dict(params, flags=16)
        _, nsl = vol.render(cams, tf, pl, nsamples=True)
        torch.cuda.synchronize()
        sl = int(nsl.sum().item())
        msl = statistics.mean(time_frames(torch, vol, cams, tf, pl, max(3, args.steps // 4), args.warmup, flush))
        variants["level_step"] = {"ms_per_frame": msl, "samples_per_frame": sl, "samples_per_s": sl / (msl * 1e-3)}
    if not args.quick and args.workload in ("c2", "c3"):
        # maximum-opacity projection (the compositing of the paper's Kidney renderings) and
        # maximum-intensity projection: every ray runs to its exit unless it reaches the
        # largest TF opacity (MOP) or coordinate (MIP); with and without empty-space skipping
        for mode in ("mop", "mip"):
            pm = dict(params, composite=mode)
            _, nsm = vol.render(cams, tf, pm, nsamples=True)
            torch.cuda.synchronize()
            sm = int(nsm.sum().item())
            nrep = max(3, args.steps // 4)
            msm = statistics.mean(time_frames(torch, vol, cams, tf, pm, nrep, args.warmup, flush))
            msk = statistics.mean(time_frames(torch, vol, cams, tf, dict(pm, flags=2), nrep, args.warmup, flush))
            variants[mode] = {"ms_per_frame": msm, "samples_per_frame": sm, "samples_per_s": sm / (msm * 1e-3),
                              "ms_per_frame_skip_empty": msk}
    if not args.quick and args.workload == "c3":
        # the plain form at matched rays: the same views rendered one launch each from a float32
        # store of the same volume (converted on the GPU; compact slots keep it to ~41 GB)
        vol.close()
        torch.cuda.empty_cache()
        v32 = P.Volume(wl["D"], "f32", wl["brick"], wl["levels"], layout="compact")
        v32.upload_level(0, raw, wl["src"])
        v32.build_lod(0)
        s32 = 0
        for cam in cams:
            _, nsv = v32.render(cam, tf, params, nsamples=True)
            s32 += int(nsv.sum().item())
        torch.cuda.synchronize()
        per_view = []
        for _ in range(max(2, args.steps // 4)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for cam in cams:
                v32.render(cam, tf, params)
            b.record()
            torch.cuda.synchronize()
            per_view.append(a.elapsed_time(b))
        ms32 = statistics.mean(per_view)
        variants["single_view_f32"] = {"ms_per_frame": ms32, "samples_per_frame": s32,
                                       "samples_per_s": s32 / (ms32 * 1e-3), "launches": len(cams),
                                       "store": "f32 compact"}
        v32.close()
        torch.cuda.empty_cache()
    if not args.quick and args.workload == "c2":
        for st2 in ("f16", "f32"):
            v2 = build_volume(P, wl, st2, raw)
            _, ns2 = v2.render(cams, tf, params, nsamples=True)
            torch.cuda.synchronize()
            s2 = int(ns2.sum().item())
            ms2 = time_frames(torch, v2, cams, tf, params, max(5, args.steps // 4), args.warmup, flush)
            variants[st2] = {"samples_per_s": s2 / (statistics.mean(ms2) * 1e-3),
                             "ms_per_frame": statistics.mean(ms2), "samples_per_frame": s2}
            v2.close()
            torch.cuda.empty_cache()
    if not args.quick and args.workload in ("c2", "c4"):
        # differentiable workload: forward in gradient mode + adjoint
        w4 = workloads.c4()
        raw4 = w4["make"]() if args.workload != "c4" else raw
        v4 = build_volume(P, w4, "f32", raw4)
        tf4 = torch.from_numpy(w4["tf"]).to(dev)
        o4, ns4 = v4.render(w4["cams"], tf4, w4["params"], nsamples=True, grad=True)
        torch.cuda.synchronize()
        s4 = int(ns4.sum().item())
        drgba = torch.randn_like(o4) * 0.01
        dtf = torch.zeros((256, 4), dtype=torch.float32, device=dev)
        dvox = torch.zeros((256, 256, 256), dtype=torch.float32, device=dev)
        n4 = max(5, args.steps // 4)
        ms_f = time_frames(torch, v4, w4["cams"], tf4, w4["params"], n4, args.warmup, flush)
        ms_fb = time_frames(torch, v4, w4["cams"], tf4, w4["params"], n4, args.warmup, flush,
                            grad=True, drgba=drgba, dtf=dtf, dvox=dvox)
        variants["fwd_bwd"] = {"workload": w4["name"], "samples_per_frame": s4,
                               "fwd_ms": statistics.mean(ms_f), "fwd_bwd_ms": statistics.mean(ms_fb),
                               "fwd_samples_per_s": s4 / (statistics.mean(ms_f) * 1e-3),
                               "fwd_bwd_samples_per_s": s4 / (statistics.mean(ms_fb) * 1e-3)}
        v4.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(wl, raw, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": "ray samples/s", "value": value, "unit": "samples/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["name"], "store": store, "brick": wl["brick"], "levels": wl["levels"],
                       "views": len(cams), "pixels": npx, "lod": "footprint" if params.get("lod_mode") else "level 0",
                       "step": params["step"], "et": params["et"], "samples_per_frame": samples,
                       "bricks_touched": touched,
                       "l2": f"flushed before every step ({L2_FLUSH_BYTES >> 20} MiB write, untimed)",
                       "parallelism": f"replicas x{ws}",
                       "tile": [params.get("tile_w", 0), params.get("tile_h", 0)], "refill": params.get("refill", 0),
                       "autotuned": None if tuned is None else {k: tuned[k] for k in ("brick", "tile_w", "tile_h", "refill", "ms", "cached")}},
            "ms_per_frame": t_mean,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "samples/s", "h2d_bytes_per_step": 4096,
                    "d2h_bytes_per_step": npx * 16, "ms_per_step": e2e_step,
                    "image": "written by the render kernel into page-locked host memory"},
            # per step: the render kernel and the two tile-order scheduling kernels
            "gpu_launches": launches_per_frame * args.steps,
            "clocks": clocks,
            "wall_s_timed": wall,
            "variants": variants,
        }
        print(json.dumps(line), flush=True)
    vol.close()


def run_outofcore(args, dist, rank, ws, local):
    """Out-of-core fly-through: 4096^3 u8 volume whose bricks (every level) are generated on
    demand on the host cores into pinned memory, 64^3 bricks, 7 levels, a 16 GiB brick cache with
    LRU eviction, 30 frames at 1920x1080.  Steady state = frames 10-29.  Frame times are wall
    times of the render call: it waits for the request/load/resume passes."""
    import torch
    import paper_2509_26213_gb300 as pkg
    pkg.build()
    import paper_2509_26213_gb300.volume as P

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = workloads.c5()
    g = wl["noise"]
    vol = P.Volume(wl["D"], "u8", wl["brick"], wl["levels"], cache_bytes=wl["cache_bytes"], layout="compact")
    src = synth.brick_source(wl["D"], wl["brick"], wl["levels"], 5, dtype="u8", **g)
    vol.set_provider_batch(synth.brick_provider_address(), src, "u8")
    tf = torch.from_numpy(wl["tf"]).to(dev)
    params = dict(wl["params"], max_passes=100000)
    cams = wl["cams"]
    if ws > 1:
        cams = cams[rank::ws] * ws
    def flythrough(v, p):
        fr = []
        for cam in cams:
            torch.cuda.synchronize()
            t = time.perf_counter()
            out, ns = v.render(cam, tf, p, nsamples=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            st = v.stats()
            fr.append({"ms": 1e3 * dt, "samples": int(ns.sum().item()), "passes": st["passes"],
                       "bricks_loaded": st["bricks_loaded"], "bytes_loaded": st["bytes_loaded"],
                       "evicted": st["evicted"], "resident": st["resident"], "touched": st["touched"],
                       "load_wait_ms": st["load_wait_us"] * 1e-3, "launches": st["launches"],
                       "preview_samples": st["preview_samples"]})
        return fr

    barrier(dist)
    with Clocks(local) as clk:
        frames = flythrough(vol, params)
    clocks = clk.summary()
    vol.close()
    steady = frames[10:] if len(frames) > 10 else frames
    variants = {}
    if not args.quick:
        # the same fly-through, cold cache: loading between passes only (no overlap), and with
        # empty-space skipping
        for name, flags in (("serial_loads", 4), ("skip_empty", 2), ("preview", 8), ("level_step", 16),
                            ("sparse_pt", 0)):
            # sparse_pt: the same volume addressed through the three-level sparse page table
            v2 = P.Volume(wl["D"], "u8", wl["brick"], wl["levels"], cache_bytes=wl["cache_bytes"], layout="compact",
                          sparse_pt=name == "sparse_pt")
            v2.set_provider_batch(synth.brick_provider_address(), src, "u8")
            fr2 = flythrough(v2, dict(params, flags=flags))
            v2.close()
            st2 = fr2[10:] if len(fr2) > 10 else fr2
            variants[name] = {"ms_per_frame": statistics.mean(f["ms"] for f in st2), "first_frame_ms": fr2[0]["ms"],
                              "load_wait_ms_per_frame": statistics.mean(f["load_wait_ms"] for f in st2),
                              "passes_per_frame": statistics.mean(f["passes"] for f in st2)}
            if flags == 8:  # one pass per frame: samples on a coarser level than their own, or left out
                variants[name]["preview_sample_fraction"] = statistics.mean(
                    f["preview_samples"] / max(1, f["samples"]) for f in st2)
    ms = statistics.mean(f["ms"] for f in steady)
    samples = statistics.mean(f["samples"] for f in steady)
    t_step = max_over_ranks(dist, ms)
    value = sum_over_ranks(dist, samples) / (t_step * 1e-3)
    if rank == 0:
        line = {
            "metric": "ray samples/s", "value": value, "unit": "samples/s", "n_gpus": ws, "steps": len(steady),
            "warmup": len(frames) - len(steady), "ms_per_step": t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["name"], "store": "u8", "brick": wl["brick"], "levels": wl["levels"],
                       "layout": "compact", "cache_bytes": wl["cache_bytes"], "provider": "host cores, pinned memory",
                       "parallelism": f"replicas x{ws}"},
            "steady_state": {"ms_per_frame": ms,
                             "miss_bytes_per_frame": statistics.mean(f["bytes_loaded"] for f in steady),
                             "bricks_loaded_per_frame": statistics.mean(f["bricks_loaded"] for f in steady),
                             "passes_per_frame": statistics.mean(f["passes"] for f in steady),
                             "load_wait_ms_per_frame": statistics.mean(f["load_wait_ms"] for f in steady),
                             "first_frame_ms": frames[0]["ms"]},
            "variants": variants,
            "frames": frames,
            "clocks": clocks,
            "gpu_launches": sum(f["launches"] for f in steady),
        }
        print(json.dumps(line), flush=True)


def cpu_baseline(wl, raw, seconds):
    """The oracle as it stands on the host cores: seeded 1/64 samples of every view's pixels
    (a new sample each round) until `seconds` have passed."""
    import oracle
    ovol = oracle_volume(wl, raw)
    samples, rounds = 0, 0
    t = time.perf_counter()
    while True:
        samples += oracle_samples(ovol, wl, frame_pixels(wl, 1.0 / 64, 7000 + rounds))
        rounds += 1
        dt = time.perf_counter() - t
        if dt >= seconds:
            break
    return {"value": samples / dt, "unit": "samples/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{rounds} x (1/64 of every view's pixels, seeded), {samples} samples in {dt:.1f} s"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="primary line only (no storage variants, no fwd+bwd)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--autotune", action="store_true", help="autotune tile, refill and brick size first")
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c2s", "c3", "c4", "c5"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-frac", type=float, default=0.25, help="reference arm: fraction of pixels per step")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    dist, rank, ws, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, dist, rank, ws)
    else:
        if args.workload == "c5":
            run_outofcore(args, dist, rank, ws, local)
        else:
            run_ours(args, dist, rank, ws, local)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
