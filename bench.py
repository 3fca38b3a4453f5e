#!/usr/bin/env python3
"""Benchmark of the bricked multi-resolution raycaster on GB300.

Primary line (one step = one frame of the whole hot path):
  1024^3 uint16 fractal value noise (5 octaves) + 200 spheres (r 4..60), 64^3 bricks with apron,
  5 LOD levels built on the GPU, footprint LOD, 1920x1080 orbit view at a seeded angle, 45 deg FOV,
  step 0.5 voxel, 256-entry RGBA TF with 3 seeded opacity peaks, early termination at 0.99.
The metric is composited ray samples per second (and ms per frame).

Beside it, in the same JSON line (single GPU, unless --quick):
  variants   the same frame from binary16 and float32 bricks (with the binary16 quantisation error
             against the uint16 source), with empty-space skipping, level-scaled sampling, and as
             maximum-opacity / maximum-intensity projections;
  fwd_bwd    the differentiable workload: 256^3 float32 blobs, 16 views at 512^2, forward in
             gradient mode + adjoint of the L2 loss against images rendered with a seeded
             perturbed transfer function, with its own roofline;
  workloads  the plain single view (128^3 uint8, 256^2), the batched form (64 views of
             {256..1024}^2 over a 2048^3 uint8 volume, autotuned tile and brick, against the plain
             float32 one-view-per-launch form at matched rays), and the out-of-core fly-through
             (4096^3 procedural bricks generated on demand into a 16 GiB cache, steady-state
             ms/frame and miss bytes/frame).
Every image's max-abs per-channel error against the FP64 oracle is stated on a seeded pixel
subset (error_vs_fp64 and per workload).

--impl reference times the FP64 CPU oracle on a bounded seeded pixel sample of the same frame.
"""
from __future__ import annotations

import argparse
import hashlib
import json
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
from synth import workloads  # noqa: E402

L2_FLUSH_BYTES = 256 << 20
AMB = 1e-5  # early-termination margin within which float32 and float64 may decide differently
TOL = {"u8": 1e-4, "f32": 1e-4, "u16": 2e-3, "f16": 2e-3}  # FP32 path / reduced-precision storage


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


def kernel_digest(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2509_26213_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


RENDER_SOURCES = ("kernels_render.cu", "render_common.cuh", "internal.cuh")


def recorded_counter(profile, what):
    """A per-launch figure from a committed ncu summary (`what` is the line's label, e.g. "dram
    bytes" or "warp instructions"), if the summary was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", profile)
    try:
        text = open(path).read()
    except OSError:
        return None
    m_src = re.search(r"kernel source digest:\s*([0-9a-f]+)", text)
    m_b = re.search(what + r" per launch \(scaled to the bench frame\):\s*([0-9.eE+]+)", text)
    if m_src and m_b and m_src.group(1) == kernel_digest(RENDER_SOURCES):
        return float(m_b.group(1))
    return None


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


def mean(xs):
    return statistics.mean(xs)


def bytes_per_voxel(store):
    return {"u8": 1, "u16": 2, "f16": 2, "f32": 4}[store]


# ------------------------------------------------------------------ workload helpers

def load_workload(key, rank=0, ws=1):
    wl = getattr(workloads, key)()
    if ws > 1:
        # weak scaling: every rank renders its own frame (views rotated per rank); no collective
        wl["cams"] = [synth.seeded_orbit(wl["D"], c["w"], c["h"], 11 + rank, view=i) for i, c in enumerate(wl["cams"])]
    return wl


def workload_config(wl, ws):
    """The keys that define the workload (printed identically by both arms)."""
    p = wl["params"]
    return {"workload": wl["name"], "store": wl["store"], "brick": wl["brick"], "levels": wl["levels"],
            "layout": wl.get("layout", "quad"),
            "views": len(wl["cams"]), "pixels": sum(c["w"] * c["h"] for c in wl["cams"]),
            "lod": "footprint" if p.get("lod_mode") else "level 0", "step": p["step"], "et": p["et"],
            "l2": f"flushed before every step ({L2_FLUSH_BYTES >> 20} MiB write, untimed)",
            "parallelism": f"replicas x{ws}"}


def oracle_volume(wl, raw, store=None):
    import oracle
    oracle.build()
    store = store or wl["store"]
    if (wl["src"], store) == ("u16", "f16"):
        raw = oracle.u16_to_f16(raw)
    elif (wl["src"], store) == ("u16", "f32"):
        raw = oracle.u16_to_f32(raw)
    elif (wl["src"], store) == ("u8", "f32"):
        raw = oracle.u8_to_f32(raw)
    return oracle.Volume(oracle.pyramid(raw, wl["levels"], store), store, wl["brick"])


def frame_pixels(wl, frac, seed):
    """A seeded sample of every view's pixels: [(view, pixels[n,2])]."""
    out = []
    for v, cam in enumerate(wl["cams"]):
        n = max(1, int(cam["w"] * cam["h"] * frac))
        out.append((v, synth.pixel_subset(cam["w"], cam["h"], n, seed * 1000 + v)))
    return out


def oracle_render_parts(ovol, wl, parts, params=None):
    import oracle
    return [oracle.render(ovol, wl["cams"][v], wl["tf"], params or wl["params"], pixels=pix, amb=AMB)
            for v, pix in parts]


def error_vs_oracle(wl, img, parts, refs, tol):
    """Max-abs per-channel error of the GPU image (packed views, host array [n,4]) against the FP64
    oracle on the pixels of `parts`; where the oracle's early-termination decision lies within
    rounding of the threshold, its alternate result counts for that pixel (both are correct)."""
    offs = np.cumsum([0] + [c["w"] * c["h"] for c in wl["cams"]])
    emax, npx, nalt, nbad = 0.0, 0, 0, 0
    for (v, pix), ref in zip(parts, refs):
        g = img[offs[v] + pix[:, 1].astype(np.int64) * wl["cams"][v]["w"] + pix[:, 0]].astype(np.float64)
        ep = np.abs(g - ref["rgba"]).max(1)
        ea = np.abs(g - ref["alt_rgba"]).max(1)
        alt = ref["amb"] & (ep > tol) & (ea <= tol)
        err = np.where(alt, ea, ep)
        emax = max(emax, float(err.max(initial=0.0)))
        npx += len(pix)
        nalt += int(alt.sum())
        nbad += int((err > tol).sum())
    return {"max_abs": emax, "tolerance": tol, "within": nbad == 0, "pixels": npx, "alternate_et": nalt}


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
        oracle_render_parts(ovol, wl, frame_pixels(wl, frac / 16, 500 + i))
    times, samples = [], 0
    for i in range(args.steps):
        parts = frame_pixels(wl, frac, 2000 + i)
        t = time.perf_counter()
        samples += sum(int(r["n"].sum()) for r in oracle_render_parts(ovol, wl, parts))
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = samples / total
    sample = f"{frac:g} of every view's pixels per step (seeded, new each step), {args.steps} steps"
    line = {
        "impl": "reference", "metric": "ray samples/s", "value": value, "unit": "samples/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(wl, ws),
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "prep_s": prep,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def build_volume(P, wl, store, raw, layout=None):
    vol = P.Volume(wl["D"], store, wl["brick"], wl["levels"], layout=layout or wl.get("layout", "quad"))
    vol.upload_level(0, raw, wl["src"])
    if wl["levels"] > 1:
        vol.build_lod(0)
    return vol


def time_frames(torch, vol, cams, tf, params, steps, warmup, flush, grad=False, drgba=None, dtf=None, dvox=None):
    """Per-step CUDA-event times (ms) of one frame; L2 flushed before every step (not timed).
    grad: the forward in gradient mode, followed by the adjoint when drgba is given."""
    back = grad and drgba is not None
    for _ in range(warmup):
        vol.render(cams, tf, params, grad=grad)
        if back:
            vol.render_backward(drgba, dtf, dvox)
    torch.cuda.synchronize()
    evs = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        vol.render(cams, tf, params, grad=grad)
        if back:
            vol.render_backward(drgba, dtf, dvox)
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def frame_stats(torch, vol, cams, tf, params):
    """One untimed render: its image (host), composited samples, bricks touched, samples skipped."""
    out, ns = vol.render(cams, tf, params, nsamples=True)
    torch.cuda.synchronize()
    st = vol.stats()
    return out, int(ns.sum().item()), st


def hbm_roofline(bytes_per_frame, ms, what, kernel):
    peak, kind = measured_peaks()
    achieved = bytes_per_frame / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": f"{kind} hbm_gbs (copy, burst)", "kernel": kernel, "bytes_accounting": what,
            "bytes_per_frame": bytes_per_frame}


FWD_BYTES = "bricks touched x (B+1)^3 x bytes/voxel + image 16 B/px + TF 4 KiB + 4 B/brick page-table word"


def forward_bytes(touched, brick, bpv, npx):
    return touched * (brick + 1) ** 3 * bpv + npx * 16 + 4096 + touched * 4


def measure_variants(torch, P, vol, wl, raw, cams, tf, params, samples, args, flush):
    """The primary frame from other storage types, with empty-space skipping, level-scaled
    sampling and as projections."""
    variants = {}
    nrep = max(5, args.steps // 4)
    pe = dict(params, flags=P.C.VOL_RENDER_SKIP_EMPTY)
    _, _, st = frame_stats(torch, vol, cams, tf, pe)
    ms_es = mean(time_frames(torch, vol, cams, tf, pe, nrep, args.warmup, flush))
    comp = samples - st["skipped_samples"]
    variants["skip_empty"] = {"ms_per_frame": ms_es, "samples_composited": comp, "samples_skipped": st["skipped_samples"],
                              "samples_per_s": comp / (ms_es * 1e-3)}
    if params.get("lod_mode"):
        # level-scaled sampling: coarse levels take steps of dt 2^l with corrected opacity (a
        # different, cheaper image of the same volume; reported beside the default line)
        pl = dict(params, flags=P.C.VOL_RENDER_LEVEL_STEP)
        _, sl, _ = frame_stats(torch, vol, cams, tf, pl)
        msl = mean(time_frames(torch, vol, cams, tf, pl, nrep, args.warmup, flush))
        variants["level_step"] = {"ms_per_frame": msl, "samples_per_frame": sl, "samples_per_s": sl / (msl * 1e-3)}
    # maximum-opacity projection (the compositing of the paper's Kidney renderings) and
    # maximum-intensity projection: every ray runs to its exit unless it reaches the largest TF
    # opacity (MOP) or coordinate (MIP); with and without empty-space skipping
    for mode in ("mop", "mip"):
        pm = dict(params, composite=mode)
        _, sm, _ = frame_stats(torch, vol, cams, tf, pm)
        n3 = max(3, args.steps // 8)
        msm = mean(time_frames(torch, vol, cams, tf, pm, n3, args.warmup, flush))
        pk = dict(pm, flags=P.C.VOL_RENDER_SKIP_EMPTY)
        _, _, stk = frame_stats(torch, vol, cams, tf, pk)
        msk = mean(time_frames(torch, vol, cams, tf, pk, n3, args.warmup, flush))
        variants[mode] = {"ms_per_frame": msm, "samples_per_frame": sm, "samples_per_s": sm / (msm * 1e-3),
                          "ms_per_frame_skip_empty": msk, "samples_skipped": stk["skipped_samples"]}
    return variants


def storage_variants(torch, P, wl, raw, cams, tf, params, args, flush, img_u16):
    """The same frame from binary16 and float32 bricks of the same uint16 volume; the binary16
    store's quantisation error against the uint16 source, per voxel value and per image."""
    out = {}
    hist = np.bincount(raw.ravel(), minlength=65536) if wl["src"] == "u16" else None
    for st2 in ("f16", "f32"):
        v2 = build_volume(P, wl, st2, raw)
        img2, s2, stv = frame_stats(torch, v2, cams, tf, params)
        ms2 = mean(time_frames(torch, v2, cams, tf, params, max(5, args.steps // 4), args.warmup, flush))
        touched = stv["touched"]
        rec = {"ms_per_frame": ms2, "samples_per_frame": s2, "samples_per_s": s2 / (ms2 * 1e-3),
               "roofline_frac": hbm_roofline(forward_bytes(touched, wl["brick"], bytes_per_voxel(st2),
                                                           img2.shape[0]), ms2, FWD_BYTES, "k_render")["frac"]}
        img2h = img2.cpu().numpy()
        if st2 == "f16" and hist is not None:
            u = np.arange(65536, dtype=np.float64)
            exact = u / 65535.0
            q = np.abs((u / 65535.0).astype(np.float32).astype(np.float16).astype(np.float64) - exact)
            present = hist > 0
            rec["quantisation_vs_u16"] = {
                "voxel_value_max_abs": float(q[present].max()),
                "voxel_value_mean_abs": float((q * hist).sum() / hist.sum()),
                "image_max_abs_vs_u16_store": float(np.abs(img2h - img_u16).max()),
                "note": "value error of binary16(u / 65535) against u / 65535, and the largest per-channel "
                        "difference between the images rendered from the binary16 and the uint16 bricks"}
        out[st2] = (rec, img2h)
        v2.close()
        torch.cuda.empty_cache()
    return out


def fwd_bwd(torch, P, args, flush, dev, do_err, key="c4"):
    """Differentiable workload: forward in gradient mode + adjoint of L = 1/2 sum (I - I*)^2, I*
    rendered with the seeded perturbed TF."""
    w4 = getattr(workloads, key)()
    raw4 = w4["make"]()
    v4 = build_volume(P, w4, "f32", raw4)
    tf4 = torch.from_numpy(w4["tf"]).to(dev)
    tgt_tf = torch.from_numpy(synth.tf_perturbed(w4["tf"], 13)).to(dev)
    cams, params = w4["cams"], w4["params"]
    target = v4.render(cams, tgt_tf, params).clone()
    o4, ns4 = v4.render(cams, tf4, params, nsamples=True, grad=True)
    torch.cuda.synchronize()
    ns = ns4.cpu().numpy().astype(np.int64)
    s4 = int(ns.sum())
    st = v4.stats()
    touched = st["touched"]
    drgba = (o4 - target).contiguous()  # dL/dI of the L2 loss (the forward is deterministic)
    loss = 0.5 * float((drgba.double() ** 2).sum().item())
    dtf = torch.zeros((256, 4), dtype=torch.float32, device=dev)
    dvox = torch.zeros(tuple(w4["D"][::-1]), dtype=torch.float32, device=dev)
    v4.render_backward(drgba, dtf, dvox)
    torch.cuda.synchronize()
    dvox_touched = int(torch.count_nonzero(dvox).item())
    n4 = max(5, args.steps // 4)
    ms_f = mean(time_frames(torch, v4, cams, tf4, params, n4, args.warmup, flush))
    ms_fg = mean(time_frames(torch, v4, cams, tf4, params, n4, args.warmup, flush, grad=True))
    ms_fb = mean(time_frames(torch, v4, cams, tf4, params, n4, args.warmup, flush, grad=True,
                             drgba=drgba, dtf=dtf, dvox=dvox))
    launches = v4.stats()["launches"]
    npx = o4.shape[0]
    B1 = w4["brick"] + 1
    ckpts = int(np.maximum(ns - 1, 0).__floordiv__(32).sum())  # T before samples 32, 64, ... < n
    brick_bytes = touched * B1 ** 3 * 4
    b_fwd = brick_bytes + npx * 16 + 4096 + touched * 4 + ckpts * 4 + npx * 4
    b_bwd = brick_bytes + touched * 4 + 4096 + npx * 16 + npx * 4 + ckpts * 4 + 4096 + dvox_touched * 8
    roof = hbm_roofline(b_fwd + b_bwd, ms_fb, (
        "forward: bricks touched x 33^3 x 4 B + image 16 B/px + TF + page-table words + checkpoints 4 B each "
        "(one before every 32nd sample) + sample counts 4 B/ray; adjoint: bricks again + page-table words + TF + "
        "dL/dI 16 B/px + sample counts + checkpoints + dL/dtf 4 KiB + dL/dvoxel read-modify-write 8 B per "
        "voxel with a non-zero gradient"), "k_render<grad> + k_backward")
    roof["traffic"] = None
    roof["bytes_forward"] = b_fwd
    roof["bytes_adjoint"] = b_bwd
    roof["forward_frac"] = hbm_roofline(b_fwd, ms_fg, "", "")["frac"]
    # the adjoint kernel alone (the dominant one of the step), with its recorded DRAM traffic
    adj = hbm_roofline(b_bwd, ms_fb - ms_fg, "the adjoint's part of the accounting above", "k_backward")
    adj["traffic"] = recorded_counter(f"raycast_bwd_{key}.md", "dram bytes") if key == "c4" else None
    roof["adjoint"] = adj
    rec = {"workload": w4["name"], "samples_per_frame": s4, "fwd_ms": ms_f, "fwd_grad_ms": ms_fg, "fwd_bwd_ms": ms_fb,
           "adjoint_ms": ms_fb - ms_fg, "fwd_samples_per_s": s4 / (ms_f * 1e-3),
           "fwd_bwd_samples_per_s": s4 / (ms_fb * 1e-3), "loss": loss,
           "loss_definition": "1/2 sum over views, pixels, channels of (I - I*)^2; I* from the TF plus seeded "
                              "Gaussian noise (sigma 0.05 max), clamped at 0",
           "bricks_touched": touched, "checkpoints": ckpts, "voxels_with_gradient": dvox_touched,
           "launches_per_step": launches, "roofline": roof}
    if do_err:
        import oracle
        wl = dict(w4)
        ovol = oracle_volume(wl, raw4)
        parts = frame_pixels(wl, 1.0 / 256, 4100)
        refs = oracle_render_parts(ovol, wl, parts)
        rec["error_vs_fp64"] = error_vs_oracle(wl, o4.cpu().numpy(), parts, refs, TOL["f32"])
        # gradient of the loss restricted to 512 seeded pixels: GPU adjoint vs the FP64 oracle's
        offs = np.cumsum([0] + [c["w"] * c["h"] for c in cams])
        mask = np.zeros(npx, bool)
        mask[np.random.default_rng(4101).choice(npx, 512, replace=False)] = True
        dI = drgba.cpu().numpy()
        dI[~mask] = 0
        v4.render(cams, tf4, params, grad=True)
        g_tf = torch.zeros_like(dtf)
        g_vox = torch.zeros_like(dvox)
        v4.render_backward(torch.from_numpy(dI).to(dev), g_tf, g_vox)
        torch.cuda.synchronize()
        odtf, odvox = np.zeros((256, 4)), np.zeros(raw4.shape)
        img = o4.cpu().numpy()
        for v, cam in enumerate(cams):
            sel = np.flatnonzero(mask[offs[v]:offs[v + 1]])
            if not len(sel):
                continue
            pix = np.stack([sel % cam["w"], sel // cam["w"]], 1).astype(np.int32)
            ref = oracle.render(ovol, cam, w4["tf"], params, pixels=pix, amb=AMB)
            g = img[offs[v] + sel].astype(np.float64)
            ep, ea = np.abs(g - ref["rgba"]).max(1), np.abs(g - ref["alt_rgba"]).max(1)
            alt = ref["amb"] & (ep > TOL["f32"]) & (ea <= TOL["f32"])
            a, b = oracle.render_grad(ovol, cam, w4["tf"], params, dI[offs[v] + sel].astype(np.float64), pixels=pix,
                                      alt_select=alt.astype(np.int32), amb=AMB)
            odtf += a
            odvox += b
        gt, gv = g_tf.cpu().numpy(), g_vox.cpu().numpy()
        rec["gradient_error_vs_fp64"] = {
            "pixels": 512,
            "dtf_max_abs_rel": float(np.abs(gt - odtf).max() / np.abs(odtf).max()),
            "dvoxel_max_abs_rel": float(np.abs(gv - odvox).max() / np.abs(odvox).max()),
            "tolerance_rel": 1e-4}
    v4.close()
    torch.cuda.empty_cache()
    return rec


def single_workload(torch, P, key, args, flush, dev, do_err, autotune=False):
    """One in-memory workload (plain single view or batched), with its oracle error."""
    wl = load_workload(key)
    raw = wl["make"]()
    cams, params = wl["cams"], dict(wl["params"])
    tf = torch.from_numpy(wl["tf"]).to(dev)
    store = wl["store"]
    plain_brick, plain_params = wl["brick"], dict(wl["params"])  # the config's own, before autotuning
    tuned = None
    if autotune:
        tuned = run_autotune(P, wl, store, raw, cams, tf, params)
    vol = (tuned or {}).pop("volume", None) or build_volume(P, wl, store, raw)
    img, samples, st = frame_stats(torch, vol, cams, tf, params)
    touched = st["touched"]
    npx = img.shape[0]
    with Clocks(dev.index or 0) as clk:
        ms = mean(time_frames(torch, vol, cams, tf, params, max(5, args.steps // 2), args.warmup, flush))
    rec = {"workload": wl["name"], "config": workload_config(wl, 1), "ms_per_frame": ms, "samples_per_frame": samples,
           "samples_per_s": samples / (ms * 1e-3), "bricks_touched": touched, "launches_per_frame": st["launches"],
           "roofline": hbm_roofline(forward_bytes(touched, wl["brick"], bytes_per_voxel(store), npx), ms, FWD_BYTES,
                                    "k_render"),
           "clocks": clk.summary()}
    if tuned is not None:
        rec["autotuned"] = {k: tuned[k] for k in ("brick", "tile_w", "tile_h", "refill", "ms", "cached")}
    pe = dict(params, flags=P.C.VOL_RENDER_SKIP_EMPTY)
    _, _, ste = frame_stats(torch, vol, cams, tf, pe)
    ms_es = mean(time_frames(torch, vol, cams, tf, pe, max(3, args.steps // 4), args.warmup, flush))
    rec["skip_empty"] = {"ms_per_frame": ms_es, "samples_skipped": ste["skipped_samples"],
                         "samples_per_s": (samples - ste["skipped_samples"]) / (ms_es * 1e-3)}
    imgh = img.cpu().numpy()
    vol.close()
    del img
    torch.cuda.empty_cache()
    if key == "c1":
        # the same view from float32 bricks (u8 / 255 rounded once), the plain float32 storage path
        v32 = build_volume(P, wl, "f32", raw)
        img32, s32, st32 = frame_stats(torch, v32, cams, tf, params)
        ms32 = mean(time_frames(torch, v32, cams, tf, params, max(5, args.steps // 2), args.warmup, flush))
        rec["f32_store"] = {"ms_per_frame": ms32, "samples_per_s": s32 / (ms32 * 1e-3)}
        img32h = img32.cpu().numpy()
        v32.close()
    if key == "c3":
        # the plain form at matched rays: the same views rendered one launch each from a float32
        # store of the same volume (converted on the GPU; compact slots keep it to ~41 GB), with
        # the configuration's own brick size and the default ray tiles
        wl32 = dict(wl, brick=plain_brick)
        v32 = build_volume(P, wl32, "f32", raw, layout="compact")
        s32 = 0
        for cam in cams:
            _, nsv = v32.render(cam, tf, plain_params, nsamples=True)
            s32 += int(nsv.sum().item())
        torch.cuda.synchronize()
        per_view = []
        for _ in range(max(2, args.steps // 8)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for cam in cams:
                v32.render(cam, tf, plain_params)
            b.record()
            torch.cuda.synchronize()
            per_view.append(a.elapsed_time(b))
        ms32 = mean(per_view)
        rec["plain_f32_one_view_per_launch"] = {"ms_per_frame": ms32, "samples_per_frame": s32,
                                                "samples_per_s": s32 / (ms32 * 1e-3), "launches": len(cams),
                                                "store": "f32 compact", "brick": plain_brick,
                                                "tile": "default (4 x 8)", "speedup_of_batched": ms32 / ms}
        v32.close()
    torch.cuda.empty_cache()
    if do_err:
        frac = 1.0 if key == "c1" else 1.0 / 1024
        parts = frame_pixels(wl, frac, 4200)
        ovol = oracle_volume(wl, raw)
        refs = oracle_render_parts(ovol, wl, parts)
        rec["error_vs_fp64"] = error_vs_oracle(wl, imgh, parts, refs, TOL[store])
        if key == "c1":
            ov32 = oracle_volume(wl, raw, "f32")
            rec["f32_store"]["error_vs_fp64"] = error_vs_oracle(wl, img32h, parts,
                                                                oracle_render_parts(ov32, wl, parts), TOL["f32"])
    return rec


def run_autotune(P, wl, store, raw, cams, tf, params):
    # ray-tile shape, refill threshold and brick size chosen by the autotuner (untimed)
    from paper_2509_26213_gb300.tune import autotune
    cache = os.environ.get("VOLRC_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "volrc_autotune.json"))
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    tuned = autotune(lambda b: build_volume(P, dict(wl, brick=b), store, raw), cams, tf, params,
                     key=f"{wl['key']}|{wl['name']}", cache_path=cache)
    wl["brick"] = tuned["brick"]
    params.update(tile_w=tuned["tile_w"], tile_h=tuned["tile_h"], refill=tuned["refill"])
    return tuned


def run_ours(args, dist, rank, ws, local):
    import torch
    import paper_2509_26213_gb300 as pkg
    pkg.build()
    import paper_2509_26213_gb300.volume as P

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    wl = load_workload(args.workload, rank, ws)
    wl["layout"] = args.layout
    raw = wl["make"]()
    cams, params = wl["cams"], dict(wl["params"])
    if args.skip_empty:  # (profiling aid: the primary frame rendered by the skip variant)
        params["flags"] = params.get("flags", 0) | P.C.VOL_RENDER_SKIP_EMPTY
    tf = torch.from_numpy(wl["tf"]).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    store = wl["store"]
    bpv = bytes_per_voxel(store)
    extras = not args.quick and ws == 1

    tuned = None
    if args.workload == "c3" or args.autotune:
        tuned = run_autotune(P, wl, store, raw, cams, tf, params)
    vol = (tuned or {}).pop("volume", None) or build_volume(P, wl, store, raw)
    img, samples, st0 = frame_stats(torch, vol, cams, tf, params)
    touched = st0["touched"]
    npx = sum(c["w"] * c["h"] for c in cams)

    barrier(dist)
    with Clocks(local) as clk:
        wall0 = time.perf_counter()
        ms = time_frames(torch, vol, cams, tf, params, args.steps, args.warmup, flush)
        wall = time.perf_counter() - wall0
    launches_per_frame = vol.stats()["launches"]  # library kernels of one render (the last timed one)
    clocks = clk.summary()
    t_mean = mean(ms)
    t_step = max_over_ranks(dist, t_mean)
    total_samples = sum_over_ranks(dist, samples)
    value = total_samples / (t_step * 1e-3)

    # end to end through the public API with host buffers, every step: the TF up from pinned
    # memory, the frame rendered, its image down into pinned memory.  A frame loop renders into
    # one of two device images while a copy stream moves the previous frame's image to the host,
    # so the copy overlaps the next render; the K steps are timed as one wall-clock interval
    # (the volume's atlas is larger than L2, so no flush between steps).
    tf_host = torch.from_numpy(wl["tf"]).pin_memory()
    tf_dev = torch.empty_like(tf)
    dimg = [torch.empty((npx, 4), dtype=torch.float32, device=dev) for _ in range(2)]
    himg = [torch.empty((npx, 4), dtype=torch.float32).pin_memory() for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=dev)
    rendered = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]

    def e2e_steps(n):
        main = torch.cuda.current_stream()
        for i in range(n):
            b = i & 1
            main.wait_event(copied[b])  # the copy out of this buffer two frames ago is done
            tf_dev.copy_(tf_host, non_blocking=True)
            vol.render(cams, tf_dev, params, out=dimg[b])
            rendered[b].record(main)
            copy_stream.wait_event(rendered[b])
            with torch.cuda.stream(copy_stream):
                himg[b].copy_(dimg[b], non_blocking=True)
                copied[b].record(copy_stream)

    e2e_steps(args.warmup)
    torch.cuda.synchronize()
    barrier(dist)
    t = time.perf_counter()
    e2e_steps(args.steps)
    torch.cuda.synchronize()
    e2e_step = max_over_ranks(dist, 1e3 * (time.perf_counter() - t) / args.steps)
    e2e_value = total_samples / (e2e_step * 1e-3)
    assert torch.equal(himg[(args.steps - 1) & 1], dimg[(args.steps - 1) & 1].cpu())
    # the same through a pinned host image the kernel writes directly, one frame at a time
    direct_ms = []
    for i in range(args.warmup + max(5, args.steps // 4)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        tf_dev.copy_(tf_host, non_blocking=True)
        vol.render(cams, tf_dev, params, out=himg[0])
        torch.cuda.synchronize()
        if i >= args.warmup:
            direct_ms.append(1e3 * (time.perf_counter() - t))

    # roofline of the render kernel: algorithmic bytes = bricks touched + image + TF + page-table words
    b_unique = forward_bytes(touched, wl["brick"], bpv, npx)
    roofline = hbm_roofline(b_unique, t_mean, FWD_BYTES, "k_render")
    roofline["traffic"] = recorded_counter(f"raycast_fwd_{wl['key']}.md", "dram bytes")
    roofline["per_sample_gather_GBps"] = samples * (8 * bpv + 4) / (t_mean * 1e-3) / 1e9
    # the bound the kernel actually meets: instruction issue (one warp instruction per scheduler
    # and clock: SMs x 4 schedulers at the sampled SM clock), from the recorded warp instructions
    # of one launch
    winst = recorded_counter(f"raycast_fwd_{wl['key']}.md", "warp instructions")
    if winst and clocks.get("sm_mhz"):
        issue_peak = nsm * 4 * clocks["sm_mhz"] * 1e6
        roofline["issue"] = {"achieved_warp_inst_per_s": winst / (t_mean * 1e-3), "peak_warp_inst_per_s": issue_peak,
                             "frac": winst / (t_mean * 1e-3) / issue_peak, "warp_inst_per_frame": winst,
                             "peak_kind": f"{nsm} SMs x 4 schedulers x sampled SM clock"}

    variants, fb, others = {}, None, {}
    imgh = img.cpu().numpy() if rank == 0 else None
    del img
    if extras:
        variants = measure_variants(torch, P, vol, wl, raw, cams, tf, params, samples, args, flush)
    vol.close()
    torch.cuda.empty_cache()
    stores = {}
    if extras and args.workload == "c2":
        stores = storage_variants(torch, P, wl, raw, cams, tf, params, args, flush, imgh)
        for k, (rec, _) in stores.items():
            variants[k] = rec
    if extras and args.workload in ("c2", "c4", "c4s"):
        fb = fwd_bwd(torch, P, args, flush, dev, do_err=not args.no_cpu, key="c4s" if args.workload == "c4s" else "c4")
    if extras and args.workload == "c2" and not args.only_primary:
        others["c1"] = single_workload(torch, P, "c1", args, flush, dev, do_err=not args.no_cpu)
        others["c3"] = single_workload(torch, P, "c3", args, flush, dev, do_err=not args.no_cpu, autotune=True)
        others["c5"] = outofcore(torch, P, args, dev, variants=True)[0]

    cpu, err = None, None
    if rank == 0 and ws == 1 and not args.no_cpu:
        ovol = oracle_volume(wl, raw)
        cpu, refs, parts = cpu_baseline(ovol, wl, args.cpu_seconds)
        err = {store: error_vs_oracle(wl, imgh, parts, refs, TOL[store])}
        if "f16" in stores:
            ov16 = oracle_volume(wl, raw, "f16")
            err["f16"] = error_vs_oracle(wl, stores["f16"][1], parts, oracle_render_parts(ov16, wl, parts), TOL["f16"])
        if "f32" in stores:
            ov32 = oracle_volume(wl, raw, "f32")
            err["f32"] = error_vs_oracle(wl, stores["f32"][1], parts, oracle_render_parts(ov32, wl, parts), TOL["f32"])

    if rank == 0:
        config = workload_config(wl, ws)
        line = {
            "metric": "ray samples/s", "value": value, "unit": "samples/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config,
            "measured": {"samples_per_frame": samples, "bricks_touched": touched,
                         "tile": [params.get("tile_w", 0), params.get("tile_h", 0)], "refill": params.get("refill", 0),
                         "autotuned": None if tuned is None else {k: tuned[k] for k in ("brick", "tile_w", "tile_h",
                                                                                       "refill", "ms", "cached")}},
            "ms_per_frame": t_mean,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "error_vs_fp64": err,
            "e2e": {"value": e2e_value, "unit": "samples/s", "h2d_bytes_per_step": 4096,
                    "d2h_bytes_per_step": npx * 16, "ms_per_step": e2e_step,
                    "image": "rendered into one of two device images; a copy stream moves each frame to "
                             "page-locked host memory while the next renders; K steps timed as one interval",
                    "l2": "not flushed: the volume's atlas is larger than L2",
                    "one_frame_at_a_time_ms": mean(direct_ms),
                    "one_frame_at_a_time": "the kernel writes the image into page-locked host memory across "
                                           "the host link; synchronised after every frame"},
            # per step: the render kernel and the two tile-order scheduling kernels
            "gpu_launches": launches_per_frame * args.steps,
            "clocks": clocks,
            "wall_s_timed": wall,
            "variants": variants,
            "fwd_bwd": fb,
            "workloads": others,
        }
        print(json.dumps(line), flush=True)


def outofcore(torch, P, args, dev, variants=True, rank=0, ws=1):
    """Out-of-core fly-through: 4096^3 u8 volume whose bricks (every level) are generated on
    demand on the host cores into pinned memory, 64^3 bricks, 7 levels, a 16 GiB brick cache with
    LRU eviction, 30 frames at 1920x1080.  Steady state = frames 10-29.  Frame times are wall
    times of the render call: it waits for the request/load/resume passes."""
    wl = workloads.c5()
    g = wl["noise"]
    src = synth.brick_source(wl["D"], wl["brick"], wl["levels"], 5, dtype="u8", **g)
    tf = torch.from_numpy(wl["tf"]).to(dev)
    params = dict(wl["params"], max_passes=100000)
    cams = wl["cams"]
    if ws > 1:
        cams = cams[rank::ws] * ws

    def flythrough(flags=0, sparse=False):
        v = P.Volume(wl["D"], "u8", wl["brick"], wl["levels"], cache_bytes=wl["cache_bytes"], layout="compact",
                     sparse_pt=sparse)
        v.set_provider_batch(synth.brick_provider_address(), src, "u8")
        p = dict(params, flags=flags)
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
                       "preview_samples": st["preview_samples"], "skipped": st["skipped_samples"]})
        v.close()
        return fr

    with Clocks(dev.index or 0) as clk:
        frames = flythrough()
    steady = frames[10:] if len(frames) > 10 else frames
    rec = {"workload": wl["name"], "config": {"store": "u8", "brick": wl["brick"], "levels": wl["levels"],
                                              "layout": "compact", "cache_bytes": wl["cache_bytes"],
                                              "provider": "host cores, pinned memory", "frames": len(frames)},
           "ms_per_frame": mean(f["ms"] for f in steady),
           "samples_per_frame": mean(f["samples"] for f in steady),
           "miss_bytes_per_frame": mean(f["bytes_loaded"] for f in steady),
           "bricks_loaded_per_frame": mean(f["bricks_loaded"] for f in steady),
           "passes_per_frame": mean(f["passes"] for f in steady),
           "load_wait_ms_per_frame": mean(f["load_wait_ms"] for f in steady),
           "first_frame_ms": frames[0]["ms"], "launches_steady": sum(f["launches"] for f in steady),
           "clocks": clk.summary(),
           "error_vs_fp64": "not computed: the oracle needs dense levels, and level 0 of this volume is 64 GiB "
                            "(the out-of-core tests check the same kernels against the oracle on smaller cases)"}
    rec["samples_per_s"] = rec["samples_per_frame"] / (rec["ms_per_frame"] * 1e-3)
    if variants:
        # the same fly-through, cold cache: loading between passes only (no overlap), with
        # empty-space skipping, as a progressive preview, with level-scaled sampling, and
        # addressed through the three-level sparse page table
        var = {}
        for name, flags, sparse in (("serial_loads", 4, False), ("skip_empty", 2, False), ("preview", 8, False),
                                    ("level_step", 16, False), ("sparse_pt", 0, True)):
            fr2 = flythrough(flags, sparse)
            st2 = fr2[10:] if len(fr2) > 10 else fr2
            var[name] = {"ms_per_frame": mean(f["ms"] for f in st2), "first_frame_ms": fr2[0]["ms"],
                         "load_wait_ms_per_frame": mean(f["load_wait_ms"] for f in st2),
                         "passes_per_frame": mean(f["passes"] for f in st2)}
            if flags == 8:  # one pass per frame: samples on a coarser level than their own, or left out
                var[name]["preview_sample_fraction"] = mean(f["preview_samples"] / max(1, f["samples"]) for f in st2)
        rec["variants"] = var
    return rec, frames


def run_outofcore(args, dist, rank, ws, local):
    import torch
    import paper_2509_26213_gb300 as pkg
    pkg.build()
    import paper_2509_26213_gb300.volume as P

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    barrier(dist)
    rec, frames = outofcore(torch, P, args, dev, variants=not args.quick, rank=rank, ws=ws)
    steady = frames[10:] if len(frames) > 10 else frames
    t_step = max_over_ranks(dist, rec["ms_per_frame"])
    value = sum_over_ranks(dist, rec["samples_per_frame"]) / (t_step * 1e-3)
    if rank == 0:
        line = {
            "metric": "ray samples/s", "value": value, "unit": "samples/s", "n_gpus": ws, "steps": len(steady),
            "warmup": len(frames) - len(steady), "ms_per_step": t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(rec["config"], workload=rec["workload"], parallelism=f"replicas x{ws}"),
            "steady_state": {k: rec[k] for k in ("ms_per_frame", "miss_bytes_per_frame", "bricks_loaded_per_frame",
                                                 "passes_per_frame", "load_wait_ms_per_frame", "first_frame_ms")},
            "variants": rec.get("variants", {}),
            "frames": frames,
            "clocks": rec["clocks"],
            "gpu_launches": rec["launches_steady"],
        }
        print(json.dumps(line), flush=True)


def cpu_baseline(ovol, wl, seconds):
    """The oracle as it stands on the host cores: seeded 1/64 samples of every view's pixels
    (a new sample each round) until `seconds` have passed.  Also returns round 0's pixels and
    results (the subset on which the GPU image's error is stated)."""
    import oracle
    samples, rounds = 0, 0
    first = None
    t = time.perf_counter()
    while True:
        parts = frame_pixels(wl, 1.0 / 64, 7000 + rounds)
        refs = oracle_render_parts(ovol, wl, parts)
        if first is None:
            first = (refs, parts)
        samples += sum(int(r["n"].sum()) for r in refs)
        rounds += 1
        dt = time.perf_counter() - t
        if dt >= seconds:
            break
    cpu = {"value": samples / dt, "unit": "samples/s", "cores": oracle.threads(), "kind": "oracle",
           "sample": f"{rounds} x (1/64 of every view's pixels, seeded), {samples} samples in {dt:.1f} s"}
    return cpu, first[0], first[1]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="primary line only (no variants, no other workloads)")
    ap.add_argument("--only-primary", action="store_true",
                    help="variants and fwd+bwd, but not the plain, batched and out-of-core workloads")
    ap.add_argument("--no-cpu", action="store_true", help="no oracle: no cpu_baseline and no error statements")
    ap.add_argument("--autotune", action="store_true", help="autotune tile, refill and brick size first")
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c2s", "c3", "c4", "c4s", "c5"])
    ap.add_argument("--layout", default="quad", choices=["quad", "compact"],
                    help="atlas slot layout of the primary line's volume")
    ap.add_argument("--skip-empty", action="store_true",
                    help="render the primary frame with empty-space skipping (for profiling the skip variant)")
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
