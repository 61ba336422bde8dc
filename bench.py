"""Benchmark: scene-space denoising at 1080p over a +-30-frame window, k = 7, through libssvp.

One step = one ssvp_gather_filter call over a batch of output frames of a clip resident in HBM
(camera composition on the host, then the fused gather + filter kernel).  `value` is output
Mpix/s over all ranks; `e2e` is the same metric through the C ABI with host buffers (upload +
pack + median + gather + download every step).  `--impl reference` times the FP64 CPU oracle
on the host cores, one full output frame of the same workload per step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--colour fp32|fp16]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gathered samples/s and output Mpix/s at 1080p; PSNR vs clean render & oracle"
# workloads: name -> (W, H, frames, half window T, k, first output frame, output frames per step, mode)
WORKLOADS = {
    "fhd": (1920, 1080, 68, 30, 7, 30, 8, 0),       # 1080p denoising over +-30 frames (the headline)
    "hd": (1280, 720, 60, 15, 7, 15, 8, 0),         # 720p denoising, +-15 frames
    "aperture": (1920, 1080, 68, 30, 7, 30, 8, 1),  # 1080p virtual aperture over +-30 frames
    "aperture-hd": (1280, 720, 60, 15, 7, 15, 8, 1),  # 720p virtual aperture, +-15 frames
    "batch": (0, 0, 0, 15, 7, 0, 0, 0),              # 8 uneven clips in one plan (sizes by seed)
    "learned": (1920, 1080, 68, 30, 7, 30, 8, 2),    # learned weights, trained on generated clips
    "learned-hd": (1280, 720, 60, 15, 7, 15, 8, 2),  # same network, evaluated at 720p +-15
    "frustum": (1920, 1080, 68, 30, 7, 30, 1, 4),    # the paper's frustum gather (Eq. 1-2), 1080p +-30
    "frustum-hd": (1280, 720, 60, 15, 7, 15, 1, 4),  # frustum gather at 720p +-15
    "deblur": (1920, 1080, 68, 30, 7, 30, 8, 5),     # Eq. 5 weights, every 4th frame shaken, 1080p +-30
    "shutter": (1920, 1080, 68, 30, 7, 30, 8, 6),    # Eq. 10 long exposure (box shutter), 1080p +-30
    "superres": (640, 360, 68, 30, 7, 30, 2, 7),     # Eq. 6-7: 640x360 input -> 1920x1080 output, +-30
    "inpaint": (1920, 1080, 68, 30, 7, 30, 8, 8),    # Eq. 8-9: one box of the scene removed, 1080p +-30
    "semi": (1920, 1080, 68, 30, 7, 30, 8, 9),       # semi-transparency of the same box, 1080p +-30
}
INPAINT_OBJECT, INPAINT_SIGMA_RGB = 9, 55.0 / 255.0  # the scene's fourth box; the paper's sigma_rgb = 55
SEMI_SIGMA_RGB = 80.0 / 255.0  # the paper's sigma_rgb = 80 for semi-transparency
SR_SCALE = 3
W, H, F, T, K_WIN, O_BEGIN, N_OUT, MODE = WORKLOADS["fhd"]
APERTURE, LENS, CAP = 0.05, 16, 31
RADIUS_REL = 0.005
FRUSTUM_L, FRUSTUM_SIGMA_XYZ_REL = 3.0, 0.03  # frustum gather: l = 3 px, sigma_xyz = 3 % of the median depth
# deblurring (Sec. "Deblurring"): the paper's sigma_rgb = 200 (0-255 scale) and sigma_f = 20; image
# noise 0.01 and a 1 degree camera shake during every 4th frame's exposure
DEBLUR_SIGMA_RGB, DEBLUR_SIGMA_F, DEBLUR_SIGMA_IMG, DEBLUR_SHAKE_DEG = 200.0 / 255.0, 20.0, 0.01, 1.0
BYTES_PER_CANDIDATE = {"fp32": 16, "fp16": 12}
COLOUR_BYTES = {"fp32": 16, "fp16": 8}


def shard(rank: int, world: int):
    """Weak scaling: every rank renders and denoises its own clip (seed = rank) and batch of output
    frames; ranks exchange nothing but the barrier and the step-time maximum."""
    return {"seed": rank, "frame_begin": O_BEGIN, "frame_end": O_BEGIN + N_OUT, "world": world}


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's value (the job's time), via an all-reduce MAX when world > 1."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ncu summaries whose machine-readable block bench.py reads (per workload), and the kernel source
# each was taken on: a figure is used only while that source is unchanged
PROFILE_SUMMARIES = {"fhd": ("gather_kernel_counters_denoise_1080p.md", "ssvp_gather.cu")}
# Algorithmic FP32 operations (an FMA counts as one) of the dominant kernel: per examined
# candidate (the membership test) and per accepted sample (weight and accumulation)
ALU_OPS = {
    0: (8, 13, "window gather: per examined candidate the radius test (dz 2, X and Y 2 FMA, d^2 3, compare 1); "
               "per accepted sample the Eq. 4 weight and Eq. 3 sums (colour differences 3, |dc|^2 3, exponent 2, "
               "exp 1, sums 4)"),
    1: (17, 14, "aperture gather: per box candidate the cone test (offset to the axis 6, distance and foot depth "
                "6, cone radius 3, compare 2); per accepted sample the Eq. 14 weight and Eq. 3 sums"),
    4: (10, 13, "frustum gather: per candidate the back-projection (3 FMA pairs) and Eq. 2's L1 test (2 adds, "
                "2 compares, the product L h3); per sample the Eq. 4 weight and Eq. 3 sums"),
}


def _profile_figures(workload, colour, out_frames):
    """The committed ncu summary's figures for this launch, if they were taken on this exact kernel
    source, workload and launch size: DRAM bytes per launch and warp instructions per examined
    candidate."""
    import hashlib
    if workload not in PROFILE_SUMMARIES:
        return {}
    name, src_name = PROFILE_SUMMARIES[workload]
    try:
        kv = {}
        for line in open(os.path.join(ROOT, "profiles", name)):
            if ":" in line and line.startswith("    "):
                k, v = line.strip().split(":", 1)
                kv[k.strip()] = v.strip()
        src = os.path.join(ROOT, "paper_2102_03011_gb300", "csrc", src_name)
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if kv.get("source_sha256") != sha or kv.get("workload") != workload or kv.get("colour") != colour:
            return {}
        out = {"source": f"profiles/{name}"}
        if int(kv.get("out_frames", -1)) == out_frames and "dram_bytes_per_launch" in kv:
            out["traffic"] = int(kv["dram_bytes_per_launch"])
        if "warp_inst_per_examined" in kv:
            out["warp_inst_per_examined"] = float(kv["warp_inst_per_examined"])
        return out
    except Exception:
        return {}


def roofline_block(mode, examined, accepted, kernel_ms, sm_mhz, peaks, peak_kind, prof, touched_bytes):
    """The dominant kernel against the FP32 ALU roof it is bound by (its loads are served from L1,
    its DRAM traffic is a few percent of HBM): algorithmic FP32 operations per launch / kernel time
    against 152 SMs x 128 FP32 lanes x the SM clock sampled during the timed region.  Beside it the
    measured issue-slot use, the DRAM fraction of HBM and the touched-bytes figure (L1 hits
    included: not a roofline)."""
    t = kernel_ms / 1e3
    per_exam, per_acc, note = ALU_OPS[mode]
    ops = per_exam * examined + per_acc * accepted
    peak = 152 * 128 * sm_mhz * 1e6 / 1e12
    traffic = prof.get("traffic")
    blk = {"bound": "alu", "achieved": ops / t / 1e12, "peak": peak, "unit": "TFLOP/s", "frac": ops / t / 1e12 / peak,
           "traffic": traffic, "kernel_ms": kernel_ms,
           "accounting": f"{per_exam} FP32 operations per examined candidate + {per_acc} per accepted sample "
                         f"(FMA = 1; {note}); peak = 152 SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz (median SM clock "
                         f"sampled during the timed region), derived, not measured"}
    if traffic is not None:
        blk["hbm"] = {"achieved": traffic / t / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                      "frac": traffic / t / 1e9 / peaks["hbm_gbs"],
                      "accounting": f"DRAM bytes per launch ({prof['source']}) / kernel time, {peak_kind} peak"}
    if "warp_inst_per_examined" in prof:
        slots = 152 * 4 * sm_mhz * 1e6 * t
        blk["issue"] = {"frac": prof["warp_inst_per_examined"] * examined / slots,
                        "accounting": f"warp instructions per examined candidate ({prof['source']}) x examined "
                                      "candidates / (152 SMs x 4 schedulers x SM clock x kernel time)"}
    blk["touched_bytes"] = {"achieved": touched_bytes / t / 1e9, "unit": "GB/s",
                            "frac_of_hbm": touched_bytes / t / 1e9 / peaks["hbm_gbs"],
                            "note": "effective bytes of every candidate load, L1 hits included (not a roofline)"}
    return blk


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                self.out = ""
        else:
            self.out = ""

    def summary(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, pw, reasons = [], [], [], set()
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            try:
                pw.append(float(f[2]))
            except ValueError:
                pass
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm), "sm_mhz_min": float(min(sm)),
                "power_w_median": float(np.median(pw)) if pw else None}


def _workload_clip(seed, frames=None):
    import synth
    frames = F if frames is None else frames
    if MODE == 5:
        c = synth.make_clip("room", W, H, frames, seed=seed, sigma_img=DEBLUR_SIGMA_IMG)
        return synth.shake_blur(c, range(2, frames, 4), shake_deg=DEBLUR_SHAKE_DEG, seed=seed)
    return synth.make_clip("room", W, H, frames, seed=seed)


def _inpaint_box(clip):
    """World box around the removed object (kept off the floor and ceiling planes it may touch)."""
    import synth
    return synth.object_box(clip.meta["objects"][INPAINT_OBJECT], 0.02, (-2.2 + 0.02, 1.5 - 0.02))


def _shutter_xi():
    """The long exposure of Sec. "Computational scene-space shutters": a box over the window."""
    return np.ones(2 * T + 1, np.float32)


def _oracle_params(clip):
    """The oracle's parameters for the current workload (window gather modes)."""
    import oracle
    if MODE == 5:
        return oracle.default_params(clip.depth, mode=oracle.MODE_DEBLUR, k=K_WIN, T=T, radius_rel=RADIUS_REL,
                                     sigma_rgb=DEBLUR_SIGMA_RGB, sigma_f=DEBLUR_SIGMA_F,
                                     frame_w=oracle.frame_sharpness(oracle.ClipView.of(clip)))  # raw Eq. 5 factor
    if MODE == 6:
        return oracle.default_params(clip.depth, mode=oracle.MODE_SHUTTER, k=K_WIN, T=T, radius_rel=RADIUS_REL,
                                     slot_w=_shutter_xi().astype(np.float64))
    return oracle.default_params(clip.depth, k=K_WIN, T=T, radius_rel=RADIUS_REL)


def _config(colour):
    if MODE in (8, 9):
        weights = ("Eq. 8 mean then two Eq. 9 steps, sigma_rgb = 55/255" if MODE == 8 else
                   "Eq. 8 mean, one Eq. 9 step, then Eq. 9 plus Eq. 4 around the pixel's own sample, sigma_rgb = "
                   f"80/255, sigma_xyz = {FRUSTUM_SIGMA_XYZ_REL:g} x median depth, sigma_f = 6")
        return {"workload": f"{'inpaint' if MODE == 8 else 'semitransparency'}-{W}x{H}-pm{T}-l3-{colour}", "W": W,
                "H": H, "frames": F, "out_frames_per_step": N_OUT, "half_window": T,
                "gather": "frustum (Eq. 1-2), l = 3 px", "weights": weights,
                "mask": f"world box around object {INPAINT_OBJECT} (a box), unprojected depth inside it",
                "scene": "synthetic 6 planes + 4 boxes, hand-held path, depth noise 2%, image noise 0.05",
                "colour": colour, "l2": "no flush: packed input planes exceed the 129 MB L2"}
    if MODE == 4:
        return {"workload": f"frustum-{W}x{H}-pm{T}-l3-{colour}", "W": W, "H": H, "frames": F,
                "out_frames_per_step": N_OUT, "half_window": T, "gather": "frustum (Eq. 1-2), l = 3 px, L1 test",
                "near_far": [0.01, 1000.0], "sigma_xyz": f"{FRUSTUM_SIGMA_XYZ_REL:g} x median depth",
                "scene": "synthetic 6 planes + 4 boxes, hand-held path, depth noise 2%, image noise 0.05",
                "colour": colour, "l2": "no flush: packed input planes exceed the 129 MB L2",
                "note": "frames beyond O+T are never read"}
    if MODE == 1:
        return {"workload": f"aperture-{W}x{H}-pm{T}-{colour}", "W": W, "H": H, "frames": F,
                "out_frames_per_step": N_OUT, "half_window": T, "aperture": APERTURE, "focal_plane": "median depth",
                "lens_samples": LENS, "cap": CAP, "k": K_WIN,
                "scene": "synthetic 6 planes + 4 boxes, hand-held path, depth noise 2%, image noise 0.05",
                "colour": colour, "l2": "no flush: packed input planes exceed the 129 MB L2",
                "note": "frames beyond O+T are never read, so the clip stops at 68 frames"}
    if MODE in (5, 6):
        name = "deblur" if MODE == 5 else "shutter-box"
        extra = ({"weights": "Eq. 5: Eq. 4 x the sample frame's gradient-magnitude sum", "sigma_rgb": "200/255",
                  "sigma_f": DEBLUR_SIGMA_F, "sigma_xyz": "r", "image_noise": DEBLUR_SIGMA_IMG,
                  "blur": f"camera shake of {DEBLUR_SHAKE_DEG:g} deg during the exposure of frames 2, 6, 10, ..."}
                 if MODE == 5 else {"weights": "Eq. 10: w = xi(J - O), box over the window (long exposure)"})
        return {"workload": f"{name}-{W}x{H}-pm{T}-k{K_WIN}-{colour}", "W": W, "H": H, "frames": F,
                "out_frames_per_step": N_OUT, "half_window": T, "k": K_WIN, "radius": f"{RADIUS_REL:g} x median depth",
                "scene": "synthetic 6 planes + 4 boxes, hand-held path, depth noise 2%", "colour": colour,
                "l2": "no flush: packed input planes (~3.1 GB) exceed the 129 MB L2", **extra}
    return {"workload": f"denoise-{W}x{H}-pm{T}-k{K_WIN}-{colour}", "W": W, "H": H, "frames": F,
            "out_frames_per_step": N_OUT, "half_window": T, "k": K_WIN, "radius": f"{RADIUS_REL:g} x median depth",
            "scene": "synthetic 6 planes + 4 boxes, hand-held path, depth noise 2%, image noise 0.05",
            "colour": colour, "l2": "no flush: packed input planes (~3.1 GB) exceed the 129 MB L2"}


def cpu_oracle_sample(clip, target_s=10.0, O=None, max_frames=None):
    """Times the FP64 oracle on whole output frames O, O+1, ... until about target_s seconds
    (denoising), or on a centred crop of frame O grown until about target_s / 4 seconds (aperture,
    whose full frame takes minutes on the host)."""
    import oracle
    O = O_BEGIN if O is None else O
    max_frames = N_OUT if max_frames is None else max_frames
    v = oracle.ClipView.of(clip)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    if MODE in (8, 9):
        med = oracle.median_depth(clip.depth)
        prm = oracle.Params(mode=oracle.MODE_DENOISE, k=1, T=T, radius=RADIUS_REL * med,
                            sigma_rgb=INPAINT_SIGMA_RGB if MODE == 8 else SEMI_SIGMA_RGB,
                            sigma_xyz=FRUSTUM_SIGMA_XYZ_REL * med, gather=oracle.GATHER_FRUSTUM, frustum_l=FRUSTUM_L)
        mask = oracle.mask_from_box(v, _inpaint_box(clip))
        ys, xs = np.nonzero(mask[O])
        cy, cx = (int(np.median(ys)), int(np.median(xs))) if len(ys) else (H // 2, W // 2)
        side = 4
        while True:
            crop = (min(max(cx - side // 2, 0), W - side), min(max(cy - side // 2, 0), H - side), side, side)
            t0 = time.perf_counter()
            res = oracle.inpaint_filter(v, prm, mask, O, crop=crop, semi=MODE == 9)
            dt = time.perf_counter() - t0
            if dt > target_s / 4 or 2 * side > 64:
                break
            side *= 2
        return dict(frames=1, crop=crop, seconds=dt, mpix_s=side * side / dt / 1e6, cores=cores, results=[res],
                    examined=0, accepted=int(res.nacc.sum()),
                    sample=f"{side}x{side} crop on the removed object in output frame {O} ({dt:.1f} s)")
    if MODE == 7:
        med = oracle.median_depth(clip.depth)
        prm = oracle.Params(mode=oracle.MODE_DENOISE, k=1, T=T, radius=RADIUS_REL * med, sigma_rgb=50.0 / 255.0,
                            sigma_xyz=FRUSTUM_SIGMA_XYZ_REL * med, gather=oracle.GATHER_FRUSTUM, frustum_l=FRUSTUM_L)
        Wo, Ho, side = W * SR_SCALE, H * SR_SCALE, 4
        while True:
            crop = ((Wo - side) // 2, (Ho - side) // 2, side, side)
            t0 = time.perf_counter()
            res = oracle.superres_filter(v, prm, O, SR_SCALE, crop=crop)
            dt = time.perf_counter() - t0
            if dt > target_s / 4 or 2 * side > 64:
                break
            side *= 2
        return dict(frames=1, crop=crop, seconds=dt, mpix_s=side * side / dt / 1e6, cores=cores, results=[res],
                    examined=0, accepted=int(res.nacc.sum()),
                    sample=f"{side}x{side} centre crop of the 3x output grid of frame {O} ({dt:.1f} s)")
    if MODE == 4:
        med = oracle.median_depth(clip.depth)
        prm = oracle.Params(mode=oracle.MODE_DENOISE, k=1, T=T, radius=RADIUS_REL * med,
                            sigma_xyz=FRUSTUM_SIGMA_XYZ_REL * med, gather=oracle.GATHER_FRUSTUM, frustum_l=FRUSTUM_L)
        side = 4
        while True:
            crop = ((W - side) // 2, (H - side) // 2, side, side)
            t0 = time.perf_counter()
            res = oracle.frustum_filter(v, prm, O, crop=crop)
            dt = time.perf_counter() - t0
            if dt > target_s / 4 or 2 * side > min(W, H):
                break
            side *= 2
        return dict(frames=1, crop=crop, seconds=dt, mpix_s=side * side / dt / 1e6, cores=cores, results=[res],
                    examined=0, accepted=int(res.nacc.sum()),
                    sample=f"{side}x{side} centre crop of output frame {O}, every pixel of every window frame "
                           f"tested ({dt:.1f} s)")
    if MODE == 1:
        prm = oracle.Params(mode=oracle.MODE_APERTURE, k=K_WIN, T=T, aperture=APERTURE,
                            focal_depth=oracle.median_depth(clip.depth), lens_samples=LENS, cap=CAP)
        side = 32
        while True:
            crop = ((W - side) // 2, (H - side) // 2, side, side)
            t0 = time.perf_counter()
            res = oracle.gather_filter(v, prm, O, crop=crop)
            dt = time.perf_counter() - t0
            if dt > target_s / 4 or 2 * side > min(W, H):
                break
            side *= 2
        return dict(frames=1, crop=crop, seconds=dt, mpix_s=side * side / dt / 1e6, cores=cores, results=[res],
                    examined=int(res.nexam.sum()), accepted=int(res.nacc.sum()),
                    sample=f"{side}x{side} centre crop of output frame {O} ({dt:.1f} s)")
    prm = _oracle_params(clip)
    results, dt = [], 0.0
    while len(results) < max_frames and (not results or dt < target_s):
        t0 = time.perf_counter()
        results.append(oracle.gather_filter(v, prm, O + len(results)))
        dt += time.perf_counter() - t0
    n = len(results)
    return dict(frames=n, crop=(0, 0, W, H), seconds=dt, mpix_s=n * W * H / dt / 1e6, cores=cores,
                results=results, examined=sum(int(r.nexam.sum()) for r in results),
                accepted=sum(int(r.nacc.sum()) for r in results),
                sample=f"{n} full output frame(s) {O}..{O + n - 1} ({dt:.1f} s)")



def batch_specs():
    """The mixed-clip batch: 8 clips, seeds 0..7, W in 640..1920 (16:9), 30..150 frames."""
    specs = []
    for seed in range(8):
        rng = np.random.default_rng(30_000 + seed)
        Wc = 640 + 160 * int(rng.integers(0, 9))
        specs.append((Wc, Wc * 9 // 16, int(rng.integers(30, 151)), seed))
    return specs


def run_batch(args, ss, torch, dev, stream, world, rank):
    """All output frames of 8 uneven clips in one persistent, graph-captured plan (FP16 colour),
    against 8 sequential plain launches."""
    import synth
    specs = batch_specs()
    clips = [synth.make_clip("room", Wc, Hc, Fc, seed=sd + 100 * rank) for Wc, Hc, Fc, sd in specs]
    cfmt = ss.SSVP_COLOUR_F16
    ctx = ss.ssvp_create(int(os.environ.get("LOCAL_RANK", "0")), stream)
    for i, c in enumerate(clips):
        r, d = torch.from_numpy(c.rgb).to(dev), torch.from_numpy(c.depth).to(dev)
        ss.ssvp_load_clip(ctx, i, c.W, c.H, c.F, r, d, None, cfmt)
        ss.ssvp_set_cameras(ctx, i, c.K, 1, c.w2c)
        del r, d
    ss.ssvp_sync(ctx)
    p = ss.ssvp_params_default()
    p.k, p.half_window, p.frame_begin, p.frame_end = K_WIN, T, 0, -1
    ids = list(range(len(clips)))
    t0 = time.perf_counter()
    best = ss.ssvp_autotune(ctx, p, ids)
    tune_s = time.perf_counter() - t0
    plan = ss.ssvp_plan_create(ctx, p, ids)
    cfg, n_items, grid = ss.ssvp_plan_get_config(plan)
    total_px = sum(c.W * c.H * c.F for c in clips)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    def sequential():
        for i in ids:
            ss.ssvp_gather_filter(ctx, p, [i])

    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        plan_ms = timed(lambda: ss.ssvp_plan_launch(plan), args.steps)
    examined, accepted, sum_w = ss.ssvp_read_stats(ctx)
    seq_ms = timed(sequential, max(1, args.steps // 2))
    psnr_in, psnr_out = [], []
    for i, c in enumerate(clips):
        o = torch.empty((c.F, c.H, c.W, 3), dtype=torch.float32, device=dev)
        ss.ssvp_read_output(ctx, i, 0, c.F, o)
        ss.ssvp_sync(ctx)
        on = o.cpu().numpy()
        if i == 0:
            out0 = on[c.F // 2]  # the middle output frame of the first clip, for the oracle below
        mse = lambda a_, b_: float(np.mean((a_.astype(np.float64) - b_) ** 2))
        psnr_out.append(10 * np.log10(1 / mse(on, c.clean)))
        psnr_in.append(10 * np.log10(1 / mse(c.rgb, c.clean)))
    ss.ssvp_plan_destroy(plan)

    # the plain FP32 form on the same clips: FP32 colour planes, 8 sequential launches
    n = len(clips)
    for i, c in enumerate(clips):
        r, d = torch.from_numpy(c.rgb).to(dev), torch.from_numpy(c.depth).to(dev)
        ss.ssvp_load_clip(ctx, n + i, c.W, c.H, c.F, r, d, None, ss.SSVP_COLOUR_F32)
        ss.ssvp_set_cameras(ctx, n + i, c.K, 1, c.w2c)
        del r, d

    def sequential_fp32():
        for i in ids:
            ss.ssvp_gather_filter(ctx, p, [n + i])

    seq32_ms = timed(sequential_fp32, max(1, args.steps // 2))
    # and the batched plan over the FP32 clips (its own autotuned shape)
    ids32 = [n + i for i in ids]
    ss.ssvp_autotune(ctx, p, ids32)
    plan32 = ss.ssvp_plan_create(ctx, p, ids32)
    cfg32, _, _ = ss.ssvp_plan_get_config(plan32)
    plan32_ms = timed(lambda: ss.ssvp_plan_launch(plan32), max(1, args.steps // 2))
    ss.ssvp_plan_destroy(plan32)
    psnr32 = []
    for i, c in enumerate(clips):
        o = torch.empty((c.F, c.H, c.W, 3), dtype=torch.float32, device=dev)
        ss.ssvp_read_output(ctx, n + i, 0, c.F, o)
        ss.ssvp_sync(ctx)
        psnr32.append(10 * np.log10(1 / float(np.mean((o.cpu().numpy().astype(np.float64) - c.clean) ** 2))))
        ss.ssvp_unload_clip(ctx, n + i)

    # end to end: every step uploads all clips from pinned host memory (same shapes: the planes are
    # reused), refreshes the plan for them (ssvp_plan_update keeps its graph), launches it and reads
    # every output frame back; steps alternate between two contexts on two streams, step i + 1
    # queued before step i is read back, so the copies of one step overlap the plan of the other
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pinned = [(torch.from_numpy(c.rgb).pin_memory(), torch.from_numpy(c.depth).pin_memory()) for c in clips]
    out_h = [torch.empty((c.F, c.H, c.W, 3), dtype=torch.float32).pin_memory() for c in clips]
    stream2 = torch.cuda.Stream(dev)
    ctx2 = ss.ssvp_create(local, stream2)
    ctxs = (ctx, ctx2)
    for i, c in enumerate(clips):
        ss.ssvp_load_clip(ctx2, i, c.W, c.H, c.F, pinned[i][0], pinned[i][1], ss.SSVP_MEM_HOST, cfmt)
        ss.ssvp_set_cameras(ctx2, i, c.K, 1, c.w2c)
    plans = [ss.ssvp_plan_create(cx, p, ids, cfg) for cx in ctxs]

    def issue(i):
        cx, pl = ctxs[i % 2], plans[i % 2]
        for j, c in enumerate(clips):
            ss.ssvp_load_clip(cx, j, c.W, c.H, c.F, pinned[j][0], pinned[j][1], ss.SSVP_MEM_HOST, cfmt)
            ss.ssvp_set_cameras(cx, j, c.K, 1, c.w2c)
        ss.ssvp_plan_update(pl)
        ss.ssvp_plan_launch(pl)

    def read_back(i):  # waits for step i
        for j, c in enumerate(clips):
            ss.ssvp_read_output(ctxs[i % 2], j, 0, c.F, out_h[j], ss.SSVP_MEM_HOST)

    def e2e_run(n):
        issue(0)
        for i in range(1, n):
            issue(i)
            read_back(i - 1)
        read_back(n - 1)

    e2e_run(2)
    n_e2e = max(2, min(args.steps, 4))
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    stream2.wait_event(a0)
    e2e_run(n_e2e)
    done2 = torch.cuda.Event()
    done2.record(stream2)
    stream.wait_event(done2)
    a1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(a0.elapsed_time(a1) / n_e2e, world, dev)
    for pl in plans:
        ss.ssvp_plan_destroy(pl)
    ss.ssvp_destroy(ctx2)
    peaks, peak_kind = _peaks()
    clk_summary = clk.summary()
    roofline = roofline_block(0, examined, accepted, plan_ms, clk_summary["sm_mhz"] or 2070.0, peaks, peak_kind, {},
                              12 * examined)
    line = {
        "metric": METRIC, "value": world * total_px / 1e6 / (plan_ms / 1e3), "unit": "Mpix/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": plan_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16-colour/f32", "data": "synthetic (seeded procedural scenes)",
        "config": {"workload": "batch-8-uneven-clips-pm15-k7-fp16", "clips": [list(x) for x in specs],
                   "output_pixels": total_px, "half_window": T, "k": K_WIN,
                   "plan": {"tile_rows": cfg.tile_rows, "frame_chunk": cfg.frame_chunk, "items": n_items,
                            "grid": grid, "autotune_s": tune_s},
                   "l2": "no flush: packed planes of 8 clips (GBs) exceed the 129 MB L2"},
        "sequential_plain_launches": {"value": world * total_px / 1e6 / (seq_ms / 1e3), "unit": "Mpix/s",
                                      "ms_per_step": seq_ms, "colour": "fp16"},
        "plain_fp32_sequential": {"value": world * total_px / 1e6 / (seq32_ms / 1e3), "unit": "Mpix/s",
                                  "ms_per_step": seq32_ms, "psnr_db": float(np.mean(psnr32)),
                                  "note": "the same clips with FP32 colour, one plain launch per clip"},
        "batched_fp32": {"value": world * total_px / 1e6 / (plan32_ms / 1e3), "unit": "Mpix/s",
                         "ms_per_step": plan32_ms, "tile_rows": cfg32.tile_rows, "frame_chunk": cfg32.frame_chunk,
                         "note": "the same graph-captured plan over the FP32 clips"},
        "samples_per_s": {"examined": world * examined / (plan_ms / 1e3), "accepted": world * accepted / (plan_ms / 1e3)},
        "psnr_db": {"output_vs_clean": float(np.mean(psnr_out)), "input_vs_clean": float(np.mean(psnr_in)),
                    "reference": "clean pinhole renders, mean over clips"},
        "gpu_launches": args.steps,
        "roofline": roofline,
        "e2e": {"value": world * total_px / 1e6 / (e2e_ms / 1e3), "unit": "Mpix/s",
                "h2d_bytes_per_step": sum(c.rgb.nbytes + c.depth.nbytes for c in clips),
                "d2h_bytes_per_step": sum(c.clean.nbytes for c in clips), "ms_per_step": e2e_ms,
                "pipelining": "two contexts on two streams, each with its plan updated per step "
                              "(ssvp_plan_update); step i + 1 queued before step i is read back"},
        "clocks": clk_summary,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on a centred crop of the first clip's middle frame, grown to about 8 s: on the
        # FP16-rounded colours the plan stores (its arithmetic error) and on the FP32 colours (its
        # total error, FP16 storage included)
        import oracle
        c0, O0 = clips[0], clips[0].F // 2
        rgb16 = c0.rgb.astype(np.float16).astype(np.float32)
        c16 = synth.Clip(c0.W, c0.H, c0.F, c0.K, c0.w2c, c0.w2c_true, rgb16, c0.depth, c0.clean, c0.depth_true)
        prm = oracle.default_params(c0.depth, k=K_WIN, T=T, radius_rel=RADIUS_REL)
        side = 16
        while True:
            crop = ((c0.W - side) // 2, (c0.H - side) // 2, side, side)
            t0 = time.perf_counter()
            r16 = oracle.gather_filter(oracle.ClipView.of(c16), prm, O0, crop=crop)
            dt = time.perf_counter() - t0
            if dt > 8.0 or 2 * side > min(c0.W, c0.H):
                break
            side *= 2
        r32 = oracle.gather_filter(oracle.ClipView.of(c0), prm, O0, crop=crop)
        x0, y0, cw, ch = crop
        g = out0[y0:y0 + ch, x0:x0 + cw].astype(np.float64)
        d16, d32 = np.abs(g - r16.rgb).max(-1), np.abs(g - r32.rgb).max(-1)
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        line["cpu_baseline"] = {"value": side * side / dt / 1e6, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
                                "sample": f"{side}x{side} crop of frame {O0} of the {c0.W}x{c0.H}x{c0.F} clip, "
                                          f"FP16-rounded colours ({dt:.1f} s)"}
        line["max_abs_vs_oracle"] = {"value": float(d16.max()), "p999": float(np.quantile(d16, 0.999)),
                                     "frac_above_1e-3": float((d16 > 1e-3).mean()), "pixels": int(d16.size),
                                     "total_vs_fp32_colour_oracle": {"value": float(d32.max()),
                                                                     "p999": float(np.quantile(d32, 0.999))},
                                     "note": "the plan's output against the oracle on the FP16-rounded colours "
                                             "(arithmetic) and on the FP32 colours (total); all pixels of the crop"}
    ss.ssvp_destroy(ctx)
    return line


def run_learned(args, ss, torch, dev, stream, world, rank):
    """Train the per-sample weighting network on the GPU over generated 640x360x30 clips (seeds
    1000..), then denoise 1080p +-30 with it and with the plain filter."""
    import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    ctx = ss.ssvp_create(local, stream)
    p = ss.ssvp_params_default()
    p.k, p.half_window, p.radius = K_WIN, T, -RADIUS_REL
    # a second operating point: the same method with a shorter window (its own network and context)
    TS = args.learned_short_window
    ctx_s = ss.ssvp_create(local, stream) if TS > 0 else None
    p_s = ss.ssvp_params_default()
    p_s.k, p_s.half_window, p_s.radius = K_WIN, TS, -RADIUS_REL
    n_train, group, steps_per_group = args.train_clips, 8, args.train_steps_per_group
    losses, losses_s, t_render, t_train = [], [], 0.0, 0.0
    for g0 in range(0, n_train, group):
        t0 = time.perf_counter()
        clips = [synth.make_clip("room", 640, 360, 30, seed=1000 + i) for i in range(g0, min(g0 + group, n_train))]
        t_render += time.perf_counter() - t0
        cleans = []
        for j, c in enumerate(clips):
            r, d = torch.from_numpy(c.rgb).to(dev), torch.from_numpy(c.depth).to(dev)
            for cx in (ctx, ctx_s) if ctx_s else (ctx,):
                ss.ssvp_load_clip(cx, j, c.W, c.H, c.F, r, d)
                ss.ssvp_set_cameras(cx, j, c.K, 1, c.w2c)
            cleans.append(torch.from_numpy(c.clean).to(dev))
        cfg = ss.ssvp_train_config(steps=steps_per_group, batch_pixels=16384, lr=1e-3, bce_weight=0.1,
                                   seed=g0, init=1 if g0 == 0 else 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        losses += list(ss.ssvp_train(ctx, p, list(range(len(clips))), cleans, cfg))
        t_train += time.perf_counter() - t0
        if ctx_s:
            losses_s += list(ss.ssvp_train(ctx_s, p_s, list(range(len(clips))), cleans, cfg))
        for j in range(len(clips)):
            for cx in (ctx, ctx_s) if ctx_s else (ctx,):
                ss.ssvp_unload_clip(cx, j)
    clip = _workload_clip(seed=rank)
    r, d = torch.from_numpy(clip.rgb).to(dev), torch.from_numpy(clip.depth).to(dev)
    ss.ssvp_load_clip(ctx, 0, W, H, F, r, d)
    ss.ssvp_set_cameras(ctx, 0, clip.K, 1, clip.w2c)
    if ctx_s:
        ss.ssvp_load_clip(ctx_s, 0, W, H, F, r, d)
        ss.ssvp_set_cameras(ctx_s, 0, clip.K, 1, clip.w2c)
    del r, d
    p.frame_begin, p.frame_end = O_BEGIN, O_BEGIN + N_OUT
    p_s.frame_begin, p_s.frame_end = O_BEGIN, O_BEGIN + N_OUT

    def timed(mode, steps, cx=ctx, pp=p):
        pp.mode = mode
        for _ in range(args.warmup):
            ss.ssvp_gather_filter(cx, pp, [0])
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            ss.ssvp_gather_filter(cx, pp, [0])
        b.record(stream)
        torch.cuda.synchronize()
        out = torch.empty((N_OUT, H, W, 3), dtype=torch.float32, device=dev)
        ss.ssvp_read_output(cx, 0, O_BEGIN, O_BEGIN + N_OUT, out)
        ss.ssvp_sync(cx)
        return a.elapsed_time(b) / steps, out.cpu().numpy()

    with ClockSampler(local) as clk:
        ms_l, out_l = timed(ss.SSVP_MODE_LEARNED, args.steps)
    ms_p, out_p = timed(ss.SSVP_MODE_DENOISE, args.steps)
    # the two kernels of a learned step, timed apart: a second pass of the same steps with the
    # library's kernel trace on (CUDA events around each launch)
    p.mode = ss.SSVP_MODE_LEARNED
    ss.ssvp_trace_enable(ctx, True)
    ss.ssvp_trace_read(ctx)
    for _ in range(args.steps):
        ss.ssvp_gather_filter(ctx, p, [0])
    trace = ss.ssvp_trace_read(ctx)
    ss.ssvp_trace_enable(ctx, False)
    ex_step, acc_step, _ = ss.ssvp_read_stats(ctx)  # the last call: N_OUT output frames
    peaks, peak_kind = _peaks()
    sm_mhz = clk.summary()["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    n_ext, t_ext = trace.get("extract", (0, 0.0))
    n_inf, t_inf = trace.get("infer", (0, 0.0))
    ext_ms, inf_ms = t_ext / max(n_ext, 1), t_inf / max(n_inf, 1)
    rl_ext = roofline_block(0, ex_step / N_OUT, acc_step / N_OUT, ext_ms, sm_mhz, peaks, peak_kind, {},
                            ex_step / N_OUT * BYTES_PER_CANDIDATE["fp32"])
    rl_ext["kernel"] = "extraction gather (the window gather with the stores of the capped sample sets), one frame"
    mlp_flops = 2 * (16 * 64 + 64 * 2) * 64 * W * H  # 16 -> 64 -> 2 over 64 samples per pixel, one frame
    bf16_peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    rl_inf = {"bound": "tensor", "achieved": mlp_flops / (inf_ms / 1e3) / 1e12, "peak": bf16_peak, "unit": "TFLOP/s",
              "frac": mlp_flops / (inf_ms / 1e3) / 1e12 / bf16_peak, "traffic": None, "kernel_ms": inf_ms,
              "kernel": "tcgen05 inference, one frame",
              "accounting": "2 x (16 x 64 + 64 x 2) FLOP per sample x 64 samples per pixel x pixels of the frame "
                            f"(the network, not the padded products) / kernel time; peak = {peak_kind} BF16 "
                            "(sustained: the kernel runs inside a long step)"}
    clean = clip.clean[O_BEGIN:O_BEGIN + N_OUT]
    psnr = lambda a_: float(10 * np.log10(1.0 / np.mean((a_.astype(np.float64) - clean) ** 2)))
    mpix = N_OUT * W * H / 1e6
    short = None
    if ctx_s:
        ms_ls, out_ls = timed(ss.SSVP_MODE_LEARNED, args.steps, ctx_s, p_s)
        ms_ps, out_ps = timed(ss.SSVP_MODE_DENOISE, args.steps, ctx_s, p_s)
        short = {"half_window": TS, "learned": {"value": world * mpix / (ms_ls / 1e3), "unit": "Mpix/s",
                                                 "ms_per_step": ms_ls, "psnr_db": psnr(out_ls)},
                 "plain_same_window": {"value": world * mpix / (ms_ps / 1e3), "unit": "Mpix/s", "psnr_db": psnr(out_ps)},
                 "loss_last_40": float(np.mean(losses_s[-40:])),
                 "note": "the same method and training clips with a +-%d window and its own network, against the "
                         "plain +-%d form above (an operating point, not the workload's configuration)" % (TS, T)}
        # the learned form against the plain FP32 form of the workload: faster at equal or better PSNR?
        short["beats_plain_fp32"] = {
            "mpix_s": [short["learned"]["value"], world * mpix / (ms_p / 1e3)],
            "psnr_db": [short["learned"]["psnr_db"], psnr(out_p)],
            "holds": bool(short["learned"]["value"] > world * mpix / (ms_p / 1e3)
                          and short["learned"]["psnr_db"] >= psnr(out_p))}
        ss.ssvp_destroy(ctx_s)
    line = {
        "metric": METRIC, "value": world * mpix / (ms_l / 1e3), "unit": "Mpix/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_l, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 gather, bf16 MLP (f32 accumulate)", "data": "synthetic (seeded procedural scenes)",
        "config": {**_config("fp32"), "workload": f"learned-denoise-{W}x{H}-pm{T}-k{K_WIN}",
                   "training": {"clips": n_train, "clip": "640x360x30 room scenes, seeds 1000..",
                                "steps": len(losses), "batch_pixels": 16384, "lr": 1e-3, "bce_weight": 0.1,
                                "loss_first_40": float(np.mean(losses[:40])), "loss_last_40": float(np.mean(losses[-40:])),
                                "render_s": t_render, "train_s": t_train}},
        "psnr_db": {"learned_vs_clean": psnr(out_l), "plain_vs_clean": psnr(out_p),
                    "input_vs_clean": psnr(clip.rgb[O_BEGIN:O_BEGIN + N_OUT])},
        "plain_same_run": {"value": world * mpix / (ms_p / 1e3), "unit": "Mpix/s", "ms_per_step": ms_p},
        "learned_short_window": short,
        "gpu_launches": args.steps * N_OUT * 2,
        "roofline": rl_ext if ext_ms >= inf_ms else rl_inf,
        "roofline_other_kernel": rl_inf if ext_ms >= inf_ms else rl_ext,
        "kernel_trace": {k: {"launches": n, "ms": t} for k, (n, t) in trace.items()},
        "clocks": clk.summary(),
    }
    # end to end through the C ABI with host buffers: every step uploads the clip from pinned host
    # memory, runs the learned filter and reads the output frames back; steps alternate between two
    # contexts (the second holds the same network) on two streams, step i + 1 queued before step i
    # is read back, as in the default workload
    rgb_h = torch.from_numpy(clip.rgb).pin_memory()
    dep_h = torch.from_numpy(clip.depth).pin_memory()
    stream2 = torch.cuda.Stream(dev)
    ctx2 = ss.ssvp_create(local, stream2)
    ss.ssvp_set_mlp(ctx2, *ss.ssvp_get_mlp(ctx))
    ctxs = (ctx, ctx2)
    outs = [torch.empty((N_OUT, H, W, 3), dtype=torch.float32).pin_memory() for _ in range(2)]

    def issue(i):
        cx = ctxs[i % 2]
        ss.ssvp_load_clip(cx, 0, W, H, F, rgb_h, dep_h, ss.SSVP_MEM_HOST, 0)
        ss.ssvp_set_cameras(cx, 0, clip.K, 1, clip.w2c)
        ss.ssvp_gather_filter(cx, p, [0])

    def read_back(i):
        ss.ssvp_read_output(ctxs[i % 2], 0, O_BEGIN, O_BEGIN + N_OUT, outs[i % 2], ss.SSVP_MEM_HOST)

    def e2e_run(n):
        issue(0)
        for i in range(1, n):
            issue(i)
            read_back(i - 1)
        read_back(n - 1)

    e2e_run(2)
    n_e2e = max(2, min(2 * args.steps, 20))
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    stream2.wait_event(a)
    e2e_run(n_e2e)
    done2 = torch.cuda.Event()
    done2.record(stream2)
    stream.wait_event(done2)
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(a.elapsed_time(b) / n_e2e, world, dev)
    ss.ssvp_destroy(ctx2)
    line["e2e"] = {"value": world * mpix / (e2e_ms / 1e3), "unit": "Mpix/s", "h2d_bytes_per_step": clip.rgb.nbytes +
                   clip.depth.nbytes, "d2h_bytes_per_step": outs[0].numel() * 4, "ms_per_step": e2e_ms,
                   "pipelining": "two contexts on two streams, step i + 1 queued before step i is read back"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's learned filter (capped sets and features in C, the BF16-rounded network per
        # pixel) on a centred crop of the first output frame, grown to about 10 s
        import oracle
        W1, b1, W2, b2 = ss.ssvp_get_mlp(ctx)
        prm = oracle.default_params(clip.depth, k=K_WIN, T=T, radius_rel=RADIUS_REL)
        v = oracle.ClipView.of(clip)
        side = 16
        while True:
            crop = ((W - side) // 2, (H - side) // 2, side, side)
            t0 = time.perf_counter()
            of, oc, on, op = oracle.learned_crop(v, prm, O_BEGIN, crop=crop)
            res = np.zeros((side, side, 3))
            for y in range(side):
                for x in range(side):
                    res[y, x] = oracle.mlp_pixel(of[y, x], oc[y, x], on[y, x], W1, b1, W2, b2, round_bf16=True,
                                                 tau=p.conf_threshold, plain=op[y, x])[1]
            dt = time.perf_counter() - t0
            if dt > 10.0 or 2 * side > 512:
                break
            side *= 2
        x0, y0, cw, ch = crop
        diff = np.abs(out_l[0, y0:y0 + ch, x0:x0 + cw].astype(np.float64) - res).max(-1)
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        line["cpu_baseline"] = {"value": side * side / dt / 1e6, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
                                "sample": f"{side}x{side} crop of output frame {O_BEGIN}, learned filter with the "
                                          f"trained weights, BF16 rounding as the tensor cores ({dt:.1f} s): capped "
                                          f"sets and features on {cores} threads, the network one pixel at a time "
                                          "on one thread"}
        line["max_abs_vs_oracle"] = {"value": float(diff.max()), "p999": float(np.quantile(diff, 0.999)),
                                     "frac_above_1e-3": float((diff > 1e-3).mean()), "pixels": int(diff.size),
                                     "note": "all pixels of the crop, including radius-band, rounding-tie and "
                                             "confidence-tie pixels"}
    ss.ssvp_destroy(ctx)
    return line

def run_superres(args, ss, torch, dev, stream, world, rank):
    """Super-resolution (Sec. "Super resolution", Eq. 6-7): 640x360 input frames, +-30, onto the
    3x grid (1920x1080 output), frustum l = 3 output pixels, sigma_rgb = 50/255 (the paper's 50),
    sigma_area = one input-pixel footprint at the median depth."""
    import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    s = SR_SCALE
    Wo, Ho = W * s, H * s
    clip = _workload_clip(seed=shard(rank, world)["seed"])
    ctx = ss.ssvp_create(local, stream)
    r, d = torch.from_numpy(clip.rgb).to(dev), torch.from_numpy(clip.depth).to(dev)
    ss.ssvp_load_clip(ctx, 0, W, H, F, r, d)
    ss.ssvp_set_cameras(ctx, 0, clip.K, 1, clip.w2c)
    ss.ssvp_sync(ctx)
    del r, d
    p = ss.ssvp_params_default()
    p.half_window, p.frame_begin, p.frame_end = T, O_BEGIN, O_BEGIN + N_OUT
    p.frustum_l, p.sigma_rgb, p.radius, p.sigma_xyz = FRUSTUM_L, 50.0 / 255.0, -FRUSTUM_SIGMA_XYZ_REL, 0.0
    out = torch.empty((N_OUT, Ho, Wo, 3), dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        ss.ssvp_superres(ctx, p, 0, s, out)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            ev[i][0].record(stream)
            ss.ssvp_superres(ctx, p, 0, s, out)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(float(np.sum(step_ms)), world, dev) / args.steps
    examined, accepted, _ = ss.ssvp_read_stats(ctx)
    outn = out.cpu().numpy()
    # references: the clean render on the output grid, and bilinear upsampling of the input
    objs, _, _ = synth.scene_and_path("room", W, H, F, shard(rank, world)["seed"])
    Kh = np.repeat(synth.intrinsics(Wo, Ho)[None], N_OUT, axis=0)
    clean_hr, _, _, _ = synth.render(objs, Kh, clip.w2c_true[O_BEGIN:O_BEGIN + N_OUT], Wo, Ho)
    psnr = lambda a_, b_: float(10 * np.log10(1.0 / np.mean((a_.astype(np.float64) - b_) ** 2)))

    def upsample(img):
        t = torch.from_numpy(np.ascontiguousarray(img.transpose(0, 3, 1, 2)))
        return torch.nn.functional.interpolate(t, scale_factor=s, mode="bilinear", align_corners=False).numpy().transpose(0, 2, 3, 1)

    bil_noisy = upsample(clip.rgb[O_BEGIN:O_BEGIN + N_OUT])
    bil_clean = upsample(clip.clean[O_BEGIN:O_BEGIN + N_OUT])
    # end to end: host inputs uploaded, output read back to pinned host memory
    rgb_h = torch.from_numpy(clip.rgb).pin_memory()
    dep_h = torch.from_numpy(clip.depth).pin_memory()
    out_h = torch.empty((N_OUT, Ho, Wo, 3), dtype=torch.float32).pin_memory()

    def e2e_step():
        ss.ssvp_load_clip(ctx, 1, W, H, F, rgb_h, dep_h, ss.SSVP_MEM_HOST, ss.SSVP_COLOUR_F32)
        ss.ssvp_set_cameras(ctx, 1, clip.K, 1, clip.w2c)
        ss.ssvp_superres(ctx, p, 1, s, out)
        out_h.copy_(out, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(2, min(args.steps, 5))
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, world, dev)
    peaks, peak_kind = _peaks()
    kernel_ms = float(np.mean(step_ms))
    clk_summary = clk.summary()
    roofline = roofline_block(4, examined, accepted, kernel_ms, clk_summary["sm_mhz"] or 2070.0, peaks, peak_kind, {},
                              4 * examined + 16 * accepted)
    mpix = N_OUT * Wo * Ho / 1e6
    line = {
        "metric": METRIC, "value": world * mpix / (ms / 1e3), "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded procedural scene, rendered on the host)",
        "config": {"workload": f"superres-{W}x{H}-to-{Wo}x{Ho}-pm{T}-fp32", "W_in": W, "H_in": H, "scale": s,
                   "frames": F, "out_frames_per_step": N_OUT, "half_window": T, "frustum_l_output_px": FRUSTUM_L,
                   "sigma_rgb": "50/255", "sigma_xyz": f"{FRUSTUM_SIGMA_XYZ_REL:g} x median depth",
                   "sigma_area": "median depth / fx (one input pixel at the median depth)",
                   "scene": "synthetic 6 planes + 4 boxes, hand-held path, depth noise 2%, image noise 0.05",
                   "l2": "no flush: the step reads 61 input frames per output frame (~0.9 GB) and writes 50 MB"},
        "samples_per_s": {"examined": world * examined / (ms / 1e3), "accepted": world * accepted / (ms / 1e3)},
        "accepted_per_pixel": accepted / (N_OUT * Wo * Ho),
        "psnr_db": {"output_vs_clean_1080p": psnr(outn, clean_hr), "bilinear_of_input": psnr(bil_noisy, clean_hr),
                    "bilinear_of_clean_input": psnr(bil_clean, clean_hr),
                    "reference": "clean render on the 1920x1080 grid (true poses)"},
        "gpu_launches": args.steps,
        "roofline": roofline,
        "e2e": {"value": world * mpix / (e2e_ms / 1e3), "unit": "Mpix/s",
                "h2d_bytes_per_step": clip.rgb.nbytes + clip.depth.nbytes, "d2h_bytes_per_step": out_h.numel() * 4,
                "ms_per_step": e2e_ms},
        "clocks": clk_summary,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        v = oracle.ClipView.of(clip)
        med = oracle.median_depth(clip.depth)
        prm = oracle.Params(mode=oracle.MODE_DENOISE, k=1, T=T, radius=RADIUS_REL * med, sigma_rgb=50.0 / 255.0,
                            sigma_xyz=FRUSTUM_SIGMA_XYZ_REL * med, gather=oracle.GATHER_FRUSTUM, frustum_l=FRUSTUM_L)
        side = 4
        while True:
            crop = ((Wo - side) // 2, (Ho - side) // 2, side, side)
            t0 = time.perf_counter()
            res = oracle.superres_filter(v, prm, O_BEGIN, s, crop=crop)
            dt = time.perf_counter() - t0
            if dt > 2.5 or 2 * side > 64:
                break
            side *= 2
        x0, y0 = crop[:2]
        diff = np.abs(outn[0, y0:y0 + side, x0:x0 + side].astype(np.float64) - res.rgb).max(-1)
        line["cpu_baseline"] = {"value": side * side / dt / 1e6, "unit": "Mpix/s",
                                "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), "kind": "oracle",
                                "sample": f"{side}x{side} centre crop of output frame {O_BEGIN} ({dt:.1f} s)"}
        line["max_abs_vs_oracle"] = {"value": float(diff.max()), "pixels": int(diff.size)}
    ss.ssvp_destroy(ctx)
    return line


def run_reference(args):
    """The oracle on the host cores, on this benchmark's workload, metric and unit."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    clip = _workload_clip(0)
    times = []
    samples = []
    for i in range(args.warmup + args.steps):
        s = cpu_oracle_sample(clip, target_s=0.0 if MODE == 0 else 8.0, max_frames=1)
        if i >= args.warmup:
            times.append(s["seconds"])
            samples.append(s)
    s = samples[-1]
    px = s["crop"][2] * s["crop"][3] * s["frames"]
    value = px / float(np.mean(times)) / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(times)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(args.colour),
            "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": s["cores"], "kind": "oracle",
                             "sample": s["sample"] + " per step"},
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "samples_per_s": {"examined": s["examined"] / float(np.mean(times)),
                              "accepted": s["accepted"] / float(np.mean(times))}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--colour", default=None, choices=["fp32", "fp16"],
                    help="colour storage (default: fp16 for the virtual-aperture workloads, fp32 otherwise)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stream", action="store_true",
                    help="end to end with a full clip upload per step only (no streaming appends)")
    ap.add_argument("--workload", default="fhd", choices=sorted(WORKLOADS))
    ap.add_argument("--gather", default="window", choices=["window", "tma"],
                    help="window-gather workloads: candidate depths from the global planes (window) or from "
                         "shared-memory boxes filled by TMA tensor copies (tma, SSVP_GATHER_WINDOW_TMA)")
    ap.add_argument("--out-frames", type=int, default=None, help="output frames per step (default per workload)")
    ap.add_argument("--train-clips", type=int, default=200, help="learned workload: generated training clips")
    ap.add_argument("--train-steps-per-group", type=int, default=120,
                    help="learned workload: training steps per group of 8 clips (25 groups for 200 clips)")
    ap.add_argument("--learned-short-window", type=int, default=6,
                    help="learned workload: also train and time a network at this half window (0: off)")
    args = ap.parse_args()
    global W, H, F, T, K_WIN, O_BEGIN, N_OUT, MODE
    W, H, F, T, K_WIN, O_BEGIN, N_OUT, MODE = WORKLOADS[args.workload]
    if args.out_frames:
        N_OUT = args.out_frames
    if args.colour is None:
        # the 1080p virtual-aperture workload stores colour in FP16 (geometry and sums in FP32)
        args.colour = "fp16" if MODE == 1 else "fp32"
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import __graft_entry__ as g
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    g.build() if rank == 0 or world == 1 else None
    if world > 1:
        dist.barrier()
        g.build()
    import paper_2102_03011_gb300 as ss

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    if args.workload in ("batch", "learned", "learned-hd", "superres"):
        fn = {"batch": run_batch, "superres": run_superres}.get(args.workload, run_learned)
        line = fn(args, ss, torch, dev, stream, world, rank)
        if rank == 0:
            print(json.dumps(line))
        if world > 1:
            dist.destroy_process_group()
        return 0
    clip = _workload_clip(seed=shard(rank, world)["seed"])
    cfmt = ss.SSVP_COLOUR_F32 if args.colour == "fp32" else ss.SSVP_COLOUR_F16
    ctx = ss.ssvp_create(local, stream)
    rgb_d = torch.from_numpy(clip.rgb).to(dev)
    dep_d = torch.from_numpy(clip.depth).to(dev)
    ss.ssvp_load_clip(ctx, 0, W, H, F, rgb_d, dep_d, None, cfmt)
    ss.ssvp_set_cameras(ctx, 0, clip.K, 1, clip.w2c)
    ss.ssvp_sync(ctx)
    del rgb_d, dep_d
    p = ss.ssvp_params_default()
    p.k, p.half_window, p.frame_begin, p.frame_end = K_WIN, T, O_BEGIN, O_BEGIN + N_OUT
    p.radius = -RADIUS_REL
    if MODE == 1:
        p.mode, p.aperture, p.focal_depth, p.lens_samples, p.cap = 1, APERTURE, 0.0, LENS, CAP
    if MODE == 4:
        # the radius is no gather bound here; sigma_xyz = 0 takes it, relative to the median depth
        p.gather, p.frustum_l, p.radius, p.sigma_xyz = ss.SSVP_GATHER_FRUSTUM, FRUSTUM_L, -FRUSTUM_SIGMA_XYZ_REL, 0.0
    if MODE == 5:
        p.mode, p.sigma_rgb, p.sigma_f = ss.SSVP_MODE_DEBLUR, DEBLUR_SIGMA_RGB, DEBLUR_SIGMA_F
    if MODE == 6:
        p.mode = ss.SSVP_MODE_SHUTTER
        ss.ssvp_set_shutter(ctx, _shutter_xi(), T)
    if MODE == 8:
        p.mode, p.gather, p.frustum_l, p.sigma_rgb = ss.SSVP_MODE_INPAINT, ss.SSVP_GATHER_FRUSTUM, FRUSTUM_L, INPAINT_SIGMA_RGB
        ss.ssvp_mask_from_box(ctx, 0, _inpaint_box(clip))
    if MODE == 9:
        p.mode, p.gather, p.frustum_l, p.sigma_rgb = ss.SSVP_MODE_SEMI, ss.SSVP_GATHER_FRUSTUM, FRUSTUM_L, SEMI_SIGMA_RGB
        p.radius, p.sigma_xyz = -FRUSTUM_SIGMA_XYZ_REL, 0.0  # sigma_xyz of the Eq. 4 term: 3 % of the median depth
        ss.ssvp_mask_from_box(ctx, 0, _inpaint_box(clip))
    if args.gather == "tma":
        if MODE not in (0, 5, 6):
            raise SystemExit("--gather tma applies to the window-gather workloads (fhd, hd, deblur, shutter)")
        p.gather = ss.SSVP_GATHER_WINDOW_TMA

    def barrier():
        if world > 1:
            dist.barrier()

    # ---------------- device-resident timing
    for _ in range(args.warmup):
        ss.ssvp_gather_filter(ctx, p, [0])
    ss.ssvp_sync(ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_all0 = torch.cuda.Event(enable_timing=True)
        t_all1 = torch.cuda.Event(enable_timing=True)
        t_all0.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            ss.ssvp_gather_filter(ctx, p, [0])
            ev[i][1].record(stream)
        t_all1.record(stream)
        torch.cuda.synchronize()
    barrier()
    total_ms = t_all0.elapsed_time(t_all1)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    examined, accepted, sum_w = ss.ssvp_read_stats(ctx)
    ms_per_step = max_over_ranks(total_ms, world, dev) / args.steps
    mpix = N_OUT * W * H / 1e6
    value = world * mpix / (ms_per_step / 1e3)

    # quality: PSNR of the batch against the clean render
    out = torch.empty((N_OUT, H, W, 3), dtype=torch.float32, device=dev)
    ss.ssvp_read_output(ctx, 0, O_BEGIN, O_BEGIN + N_OUT, out)
    ss.ssvp_sync(ctx)
    outn = out.cpu().numpy()
    clean = clip.clean[O_BEGIN:O_BEGIN + N_OUT]
    noisy = clip.rgb[O_BEGIN:O_BEGIN + N_OUT]
    psnr = lambda a, b: float(10 * np.log10(1.0 / np.mean((a.astype(np.float64) - b) ** 2)))
    psnr_out, psnr_in = psnr(outn, clean), psnr(noisy, clean)
    psnr_ref = "clean pinhole render"
    if MODE == 1:
        # reference: a thin-lens render (256 lens rays per pixel) of the first output frame
        import synth
        objs, _, _ = synth.scene_and_path("room", W, H, F, rank)
        z0 = ss.ssvp_clip_median_depth(ctx, 0)
        lens = synth.render_thinlens(objs, clip.K[O_BEGIN:O_BEGIN + 1], clip.w2c_true[O_BEGIN:O_BEGIN + 1], W, H,
                                     APERTURE, z0, n_lens=256)
        psnr_out, psnr_in = psnr(outn[:1], lens), psnr(noisy[:1], lens)
        psnr_ref = "thin-lens render (256 rays/pixel) of the first output frame"

    extra_quality = {}
    if MODE in (8, 9):
        # quality on the removed object's pixels against a render of the scene without it
        import synth
        objs = list(clip.meta["objects"])
        del objs[INPAINT_OBJECT]
        bg, _, _, _ = synth.render(objs, clip.K[O_BEGIN:O_BEGIN + N_OUT], clip.w2c_true[O_BEGIN:O_BEGIN + N_OUT], W, H)
        m = ss.ssvp_read_mask(ctx, 0, F, H, W)[O_BEGIN:O_BEGIN + N_OUT].astype(bool)
        extra_quality = {"masked_fraction": float(m.mean()),
                         "output_vs_object_free_render_on_mask": psnr(outn[m], bg[m]),
                         "input_vs_object_free_render_on_mask": psnr(noisy[m], bg[m]),
                         "outside_mask_unchanged": bool(np.array_equal(outn[~m], noisy[~m]))}
        if MODE == 9:  # a see-through blend: between the object (input) and the background
            extra_quality["output_vs_input_on_mask"] = psnr(outn[m], noisy[m])
    if MODE == 5:
        # the same clip through plain Eq. 4 with the same sigmas, outside the timed region
        p.mode = ss.SSVP_MODE_DENOISE
        ss.ssvp_gather_filter(ctx, p, [0])
        plain = torch.empty_like(out)
        ss.ssvp_read_output(ctx, 0, O_BEGIN, O_BEGIN + N_OUT, plain)
        ss.ssvp_sync(ctx)
        p.mode = ss.SSVP_MODE_DEBLUR
        plainn = plain.cpu().numpy()
        blurred = [i for i in range(N_OUT) if (O_BEGIN + i) in clip.meta.get("blurred", [])]
        extra_quality = {"plain_eq4_vs_clean": psnr(plainn, clean),
                         "blurred_output_frames": [O_BEGIN + i for i in blurred]}
        if blurred:
            extra_quality.update({
                "deblur_on_blurred_frames": psnr(outn[blurred], clean[blurred]),
                "plain_eq4_on_blurred_frames": psnr(plainn[blurred], clean[blurred]),
                "input_on_blurred_frames": psnr(noisy[blurred], clean[blurred])})

    # ---------------- end to end through the C ABI with host buffers
    rgb_h = torch.from_numpy(clip.rgb).pin_memory()
    dep_h = torch.from_numpy(clip.depth).pin_memory()
    out_h = torch.empty((N_OUT, H, W, 3), dtype=torch.float32).pin_memory()
    e2e_steps = max(2, min(2 * args.steps, 20))  # the pipeline fill (one unoverlapped load) amortised over 20 steps

    # Steps alternate between two contexts on two streams (double buffering, as a streaming
    # deployment would): step i + 1's upload and gather are queued before step i's output is read
    # back to the host, so the copies of one step overlap the kernels of the other.  Every step
    # still uploads its own inputs and reads back its own result inside the timed region.
    # Inpainting and semi-transparency also compute the step's mask from the box (a reload with the
    # same shape keeps the mask's memory).
    stream2 = torch.cuda.Stream(dev)
    ctx2 = ss.ssvp_create(local, stream2)
    if MODE == 6:  # the context's own state: the Eq. 10 shutter table
        ss.ssvp_set_shutter(ctx2, _shutter_xi(), T)
    ctxs = (ctx, ctx2)
    out_hs = (out_h, torch.empty_like(out_h).pin_memory())

    def issue(i):
        cx = ctxs[i % 2]
        ss.ssvp_load_clip(cx, 1, W, H, F, rgb_h, dep_h, ss.SSVP_MEM_HOST, cfmt)
        ss.ssvp_set_cameras(cx, 1, clip.K, 1, clip.w2c)
        if MODE in (8, 9):
            ss.ssvp_mask_from_box(cx, 1, _inpaint_box(clip))
        ss.ssvp_gather_filter(cx, p, [1])

    def read_back(i):  # waits for step i on its stream
        ss.ssvp_read_output(ctxs[i % 2], 1, O_BEGIN, O_BEGIN + N_OUT, out_hs[i % 2], ss.SSVP_MEM_HOST)

    def e2e_run(n):
        issue(0)
        for i in range(1, n):
            issue(i)
            read_back(i - 1)
        read_back(n - 1)

    e2e_run(2)  # both contexts hold the clip's planes: later reloads reuse them
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk_e2e:
        e0.record(stream)
        stream2.wait_event(e0)
        e2e_run(e2e_steps)
        done2 = torch.cuda.Event()
        done2.record(stream2)
        stream.wait_event(done2)
        e1.record(stream)
        torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, world, dev)
    ss.ssvp_destroy(ctx2)
    h2d = clip.rgb.nbytes + clip.depth.nbytes
    d2h = out_h.numel() * 4
    frames_per_chunk = max(1, min(F, (4 << 30) // (W * H * 16)))
    e2e_launches = -(-F // frames_per_chunk) + 6 + 1  # packs, median passes, the gather
    e2e_launches += 1 if MODE in (4, 7, 8, 9) else 0  # frame depth ranges (frustum gathers, after each load)
    e2e_launches += 2 if MODE == 5 else 0  # Eq. 5 gradient sums (deblurring, after each load)
    e2e_launches += 1 if MODE in (8, 9) else 0  # the mask from the box
    e2e_full = {"value": world * mpix / (e2e_ms / 1e3), "unit": "Mpix/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "gpu_launches_per_step": e2e_launches,
                "pipelining": "two contexts on two streams, step i + 1 queued before step i is read back",
                "inputs": "the whole clip uploaded every step (ssvp_load_clip)", "clocks": clk_e2e.summary()}
    e2e_stream = None
    if MODE in (0, 1, 5, 6) and not args.no_stream:
        # Streaming video: a longer clip of the same scene family arrives N_OUT frames at a time.  A
        # step appends the N_OUT new frames (ssvp_append_frames: pinned host memory to the device,
        # the kept frames slid on the device into the clip's second window while the previous
        # step's gather runs), reads back the previous step's output frames and queues its gather.
        n_stream = max(2, min(args.steps, 10))
        video = _workload_clip(seed=shard(rank, world)["seed"], frames=F + N_OUT * (n_stream + 2))
        v_rgb = torch.from_numpy(video.rgb).pin_memory()
        v_dep = torch.from_numpy(video.depth).pin_memory()
        ctx3 = ss.ssvp_create(local, stream)
        if MODE == 6:
            ss.ssvp_set_shutter(ctx3, _shutter_xi(), T)
        ss.ssvp_load_clip(ctx3, 0, W, H, F, v_rgb[:F], v_dep[:F], ss.SSVP_MEM_HOST, cfmt)
        ss.ssvp_set_cameras(ctx3, 0, video.K[:F], 1, video.w2c[:F])
        outs_s = (torch.empty_like(out_h).pin_memory(), torch.empty_like(out_h).pin_memory())
        state = {"next": F}

        def s_append():
            a = state["next"]
            ss.ssvp_append_frames(ctx3, 0, N_OUT, v_rgb[a:a + N_OUT], v_dep[a:a + N_OUT], video.K[a:a + N_OUT], 1,
                                  video.w2c[a:a + N_OUT], ss.SSVP_MEM_HOST)
            state["next"] = a + N_OUT

        def s_run(n):
            s_append()
            ss.ssvp_gather_filter(ctx3, p, [0])
            for i in range(1, n):
                s_append()
                ss.ssvp_read_output(ctx3, 0, O_BEGIN, O_BEGIN + N_OUT, outs_s[(i - 1) % 2], ss.SSVP_MEM_HOST)
                ss.ssvp_gather_filter(ctx3, p, [0])
            ss.ssvp_read_output(ctx3, 0, O_BEGIN, O_BEGIN + N_OUT, outs_s[(n - 1) % 2], ss.SSVP_MEM_HOST)

        s_run(2)  # the clip's second window is allocated by the first append
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        s_run(n_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        s_ms = max_over_ranks(e0.elapsed_time(e1) / n_stream, world, dev)
        # The longer video's hand-held path is not the benchmark clip's, so its windows cost the
        # gather a different amount of work: the gather alone is timed again on the last streamed
        # window, and the difference is what streaming adds per step.
        e0.record(stream)
        for _ in range(n_stream):
            ss.ssvp_gather_filter(ctx3, p, [0])
        e1.record(stream)
        torch.cuda.synchronize()
        g_ms = max_over_ranks(e0.elapsed_time(e1) / n_stream, world, dev)
        ss.ssvp_destroy(ctx3)
        e2e_stream = {"value": world * mpix / (s_ms / 1e3), "unit": "Mpix/s",
                      "h2d_bytes_per_step": N_OUT * W * H * 16, "d2h_bytes_per_step": d2h, "ms_per_step": s_ms,
                      "gather_only_ms_same_window": g_ms, "added_ms_per_step": s_ms - g_ms,
                      "gpu_launches_per_step": 1 + 6 + 1 + (2 if MODE == 5 else 0),  # pack, median passes, gather, Eq. 5 sums
                      "inputs": f"streaming: each step appends its {N_OUT} new frames (ssvp_append_frames) to the "
                                f"{F}-frame window of a {video.F}-frame clip of the same scene family (a different "
                                f"camera path from the benchmark clip's)"}
        del video, v_rgb, v_dep

    peaks, peak_kind = _peaks()
    kernel_ms = float(np.mean(step_ms))
    if MODE in (4, 8, 9):
        cb = COLOUR_BYTES[args.colour]
        passes = 3 if MODE in (8, 9) else 1  # inpainting scans S(p) three times (Eq. 8 mean, two Eq. 9 steps)
        touched = passes * (4 * examined + cb * accepted)
        rl_mode, rl_exam, rl_acc = 4, passes * examined, passes * accepted
    else:
        touched = examined * BYTES_PER_CANDIDATE[args.colour]
        rl_mode, rl_exam, rl_acc = (1 if MODE == 1 else 0), examined, accepted
    clk_summary = clk.summary()
    sm_mhz = clk_summary["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    # the committed counters are those of the window gather reading the global planes
    prof = _profile_figures(args.workload, args.colour, N_OUT) if args.gather == "window" else {}
    roofline = roofline_block(rl_mode, rl_exam, rl_acc, kernel_ms, sm_mhz, peaks, peak_kind, prof, touched)
    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.colour == "fp32" else "f16-colour/f32",
        "data": "synthetic (seeded procedural scene, rendered on the host)",
        "config": {**_config(args.colour), **({"gather": "window, candidate depths staged by TMA tensor copies "
                                                          "(SSVP_GATHER_WINDOW_TMA)"} if args.gather == "tma" else {})},
        "samples_per_s": {"examined": world * examined / (ms_per_step / 1e3),
                          "accepted": world * accepted / (ms_per_step / 1e3)},
        "accepted_per_pixel": accepted / (N_OUT * W * H), "kept_weight_fraction": sum_w / max(accepted, 1),
        "psnr_db": {"output_vs_clean": psnr_out, "input_vs_clean": psnr_in, "reference": psnr_ref, **extra_quality},
        "gpu_launches": args.steps,
        "roofline": roofline,
        "e2e": e2e_full,
        "clocks": clk_summary,
    }
    if e2e_stream is not None:
        line["e2e_streaming"] = e2e_stream
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s = cpu_oracle_sample(clip)
        x0, y0, cw, ch = s["crop"]
        diff = np.stack([np.abs(outn[i, y0:y0 + ch, x0:x0 + cw].astype(np.float64) - r.rgb).max(-1)
                         for i, r in enumerate(s["results"])])
        line["cpu_baseline"] = {"value": s["mpix_s"], "unit": "Mpix/s", "cores": s["cores"], "kind": "oracle",
                                "sample": s["sample"]}
        line["max_abs_vs_oracle"] = {"value": float(diff.max()), "p999": float(np.quantile(diff, 0.999)),
                                     "frac_above_1e-3": float((diff > 1e-3).mean()), "pixels": int(diff.size),
                                     "note": "all pixels, including radius-band and rounding-tie pixels"}
    ss.ssvp_destroy(ctx)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
