#!/usr/bin/env python
"""Benchmark: SR projections per second for the detector-scale workload.

Workload: 4 LR frames of 2048 x 2048 float32 with half-pixel detector shifts, factor 2 ->
4096 x 4096 HR, 5x5 Gaussian PSF (sigma 0.5 HR px), BTV prior lambda 0.01, alpha 0.4, w 3,
eps 1e-3, 100 SCG iterations from multi-image interpolation.  One step = one full SR solve of
one projection (prepare, initial gradient, 100 fused SCG passes, output).  Synthetic data:
a seeded phantom, frames made with the library's forward operator plus Gaussian noise.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl misr|reference]

Under torchrun (N > 1) every rank solves its own projections (independent problems, no
collective on the data path); rank 0 prints one JSON line with the whole-job rate.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import gen  # noqa: E402

METRIC = "SR projections/s (2048^2->4096^2, 100 SCG it)"
UNIT = "projections/s"
WORKLOADS = {
    "detector": dict(h=2048, w=2048, f=2, iters=100, seed=gen.CONFIG_SEEDS["detector"],
                     desc="4 x 2048^2 fp32 frames -> 4096^2 HR, f=2, half-pixel shifts, 5x5 Gaussian PSF "
                          "sigma 0.5, lambda 0.01, BTV alpha 0.4 w 3 eps 1e-3, 100 SCG iterations"),
    "tiny": dict(h=64, w=64, f=2, iters=50, seed=gen.CONFIG_SEEDS["tiny"],
                 desc="4 x 64^2 fp32 frames -> 128^2 HR, f=2, 50 SCG iterations"),
}
PASS_BYTES_PER_PX = 28  # fused pass: read x, r, p_old, Y; write x', r', p (float32)
# Frame-wise pass (frames that do not interleave), f = 2 with 4 frames (one LR sample per HR
# pixel), every image read or written once by each kernel that uses it: A reads x, r, p_old and
# writes x', p, lambda grad BTV (24); F1 reads x', p and writes their horizontal parts, 2 K H w
# floats (8 + 16); B reads those and the frames and writes DS psi_d', A p and (L1) psi_d''
# (16 + 4 + 12); C1 reads DS psi_d' and writes the adjoint's horizontal part, K h W floats
# (4 + 8); C2 reads that, lambda grad BTV, r, p and writes r' (8 + 16); F1 of r' (4 + 8); D reads
# its part, (L1) psi_d'', A p (16) and x', r', p (12).  156 B/px with the L1 term, 148 with L2.
GEN_PASS_BYTES_PER_PX_L1 = 156


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def load_traffic(kernel_tag, shape_name):
    """Per-launch DRAM bytes of the fused pass from the committed ncu summary, if it was
    taken on the current kernel source and tile shape."""
    try:
        with open(os.path.join(ROOT, "profiles", "scg_pass_traffic.json")) as fh:
            d = json.load(fh)
        if d.get("kernel_source_sha1") == kernel_tag and d.get("tile_shape") == shape_name:
            return float(d["dram_bytes_per_launch_4096"])
    except Exception:
        pass
    return None


def kernel_source_tag():
    """Hash of the fused pass's device code (its tile shapes included), comments and blank
    space left out: a traffic record stays valid across comment edits, not across code ones."""
    import hashlib
    import re
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2108_04315_b300", "csrc")
    for f in ("misr_types.cuh", "misr_device.cuh", "misr_stream.cuh", "tma.cuh"):
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()


# the B300's nominal HBM3e bandwidth (GB/s), beside the measured copy peak
SPEC_HBM_GBS = 7700.0

# MISR_TILE_* -> (tile rows, tile columns, threads per CTA); the streaming shape's items are 112
# columns wide, their height chosen per plan (0 here)
TILE_SHAPES = {1: (32, 64, 512), 2: (32, 32, 256), 3: (16, 64, 256), 4: (0, 112, 256)}


def shape_label(k):
    return "stream" if k == 4 else "%dx%d" % TILE_SHAPES[k][:2]


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu_index), "-lms", "100"], stdout=self.tmp,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.tmp is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for _, _, flags in rows for i, v in enumerate(flags) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def job_rate(units_per_rank, seconds, dist=None, device=None):
    """Whole-job rate over replicas: the units all ranks processed divided by the slowest rank's
    time (max over ranks).  Returns (rate, max seconds)."""
    world = 1
    if dist is not None:
        import torch
        world = dist.get_world_size()
        t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = float(t.item())
    return world * units_per_rank / seconds, seconds


def make_inputs(plan, wl, device):
    """Phantom and frames y = A x_true + noise, made on the device with the library's forward op."""
    import torch
    H, W = wl["f"] * wl["h"], wl["f"] * wl["w"]
    xt = torch.from_numpy(gen.phantom(H, W, wl["seed"]).astype(np.float32)).to(device)
    y = plan.forward(xt)
    noise = torch.from_numpy(gen.gaussian_noise((4, wl["h"], wl["w"]), 0.01, wl["seed"] + 1).astype(np.float32))
    y += noise.to(device)
    torch.cuda.synchronize()
    return xt, y


def measure_variant(args, wl, shifts, psf, tuned, xt, stream, dist, device, peak, iters, y=None, **kw):
    """The headline geometry solved with other model options (kw: Plan arguments): solve rate
    and per-pass time, timed as the headline (K solves of `iters` and of 0 iterations, CUDA
    events on the solve's stream).  Frames: y, else A x_true + N(0, 0.01^2) with this model's A."""
    import torch
    from paper_2108_04315_b300.binding import Plan
    H, W = wl["f"] * wl["h"], wl["f"] * wl["w"]
    kw = dict(dict(lam=0.01, btv_alpha=0.4, btv_w=3, eps=1e-3, tile_shape=tuned), **kw)
    p1 = Plan(wl["h"], wl["w"], wl["f"], shifts, psf, iters=iters, **kw)
    p0 = Plan(wl["h"], wl["w"], wl["f"], shifts, psf, iters=0, **kw)
    if y is None:
        y = p1.forward(xt)
        y += torch.from_numpy(gen.gaussian_noise(tuple(y.shape), 0.01, wl["seed"] + 1).astype(np.float32)).to(device)
    x = torch.empty((H, W), dtype=torch.float32, device=device)
    for _ in range(max(args.warmup, 3)):
        p1.solve(y, x, stats=False)
        p0.solve(y, x, stats=False)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    for _ in range(args.steps):
        p1.solve(y, x, stats=False)
    ev[1].record(stream)
    for _ in range(args.steps):
        p0.solve(y, x, stats=False)
    ev[2].record(stream)
    ev[2].synchronize()
    ms1, ms0 = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    pass_ms = max((ms1 - ms0) / args.steps / max(iters, 1), 1e-9)
    rate, _ = job_rate(args.steps, ms1 / 1e3, dist, device)
    xs, st = p1.solve(y, x, stats=True)
    err = float(torch.linalg.vector_norm(xs - xt) / torch.linalg.vector_norm(xt))
    p1.close()
    p0.close()
    achieved = PASS_BYTES_PER_PX * H * W / (pass_ms * 1e-3) / 1e9
    return {"value": rate, "unit": UNIT, "iters": iters, "ms_per_pass": pass_ms, "achieved_gbs": achieved,
            "frac": achieved / peak, "image_rel_error_vs_phantom": err,
            "solve": {"J_final": st["J_final"], "accepted": st["accepted"], "iters_done": st["iters_done"]},
            "timed_as": "K solves, CUDA events; per pass (T(%d it) - T(0 it)) / %d" % (iters, max(iters, 1))}


L1_DATA_EPS = 0.01   # smoothing of the L1 data term: the frames' noise sigma


def measure_l1(args, wl, shifts, psf, tuned, y, xt, stream, dist, device, peak):
    """The headline workload with the smoothed L1 data term (the paper's experiments)."""
    from paper_2108_04315_b300.binding import MISR_NORM_L1
    out = measure_variant(args, wl, shifts, psf, tuned, xt, stream, dist, device, peak, wl["iters"], y=y,
                          data_norm=MISR_NORM_L1, data_eps=L1_DATA_EPS)
    out.update({"data_norm": "L1, psi_d(t) = sqrt(t^2 + eps_d^2) - eps_d", "data_eps": L1_DATA_EPS})
    return out


def measure_paper_ct(args, wl, shifts, tuned, xt, stream, dist, device, peak):
    """The paper's CT reconstruction setting (Sec. 4) at the headline size: 3x3 Gaussian blur,
    lambda 0.05, alpha 0.4, 20 SCG iterations, the L1 data term, and the 2x2 binning D of the
    synthetic study (Sec. 4.1.1); frames made with that model."""
    from paper_2108_04315_b300.binding import MISR_DECIM_BIN, MISR_NORM_L1
    psf3 = gen.gaussian_psf(3, 0.5)
    out = measure_variant(args, wl, shifts, psf3, tuned, xt, stream, dist, device, peak, 20, lam=0.05,
                          data_norm=MISR_NORM_L1, data_eps=L1_DATA_EPS, decimation=MISR_DECIM_BIN)
    out["model"] = ("2048^2 -> 4096^2, f=2 half-pixel shifts, 3x3 Gaussian sigma 0.5, 2x2 binning D, L1 data "
                    "term eps_d 0.01, lambda 0.05, BTV alpha 0.4 w 3 eps 1e-3, 20 SCG iterations")
    return out


def measure_subpixel(args, wl, xt, stream, dist, device, peak):
    """Non-integer detector shifts (bilinear M_k, per-phase blur taps) at the headline size: the
    half-pixel pattern with stage errors of a few hundredths of a pixel (x stage 0.02 / 0.51,
    y stage 0.04 / 0.53 LR px), a 3x3 Gaussian PSF, 100 SCG iterations; frames made with that
    model.  The tile shape is 32x32 (the one compiled with per-phase taps)."""
    shifts = [(dx, dy) for dy in (0.04, 0.53) for dx in (0.02, 0.51)]
    out = measure_variant(args, wl, shifts, gen.gaussian_psf(3, 0.5), 2, xt, stream, dist, device, peak,
                          wl["iters"])
    out["model"] = ("2048^2 -> 4096^2, f=2, shifts (dx, dy) in {0.02, 0.51} x {0.04, 0.53} LR px (bilinear M_k), "
                    "3x3 Gaussian sigma 0.5, L2 data term, lambda 0.01, 100 SCG iterations")
    return out


def measure_study(args, wl, xt, stream, dist, device, peak):
    """The synthetic study's frame set (Sec. 4.1.1: one-pixel shifts right, down, left and up at
    2x, two frames on each of two HR phases, 2x2 binning D) in the paper's reconstruction
    setting (3x3 Gaussian blur, lambda 0.05, alpha 0.4, the L1 data term, 20 SCG iterations) at
    the headline size; frames made with that model.  These frames do not interleave into one HR
    image, so the plan runs the frame-wise pass."""
    from paper_2108_04315_b300.binding import MISR_DECIM_BIN, MISR_NORM_L1
    shifts = [(0.5, 0.0), (0.0, 0.5), (-0.5, 0.0), (0.0, -0.5)]
    H, W = wl["f"] * wl["h"], wl["f"] * wl["w"]
    out = measure_variant(args, wl, shifts, gen.gaussian_psf(3, 0.5), 0, xt, stream, dist, device, peak, 20,
                          lam=0.05, data_norm=MISR_NORM_L1, data_eps=L1_DATA_EPS, decimation=MISR_DECIM_BIN)
    gen_achieved = GEN_PASS_BYTES_PER_PX_L1 * H * W / (out["ms_per_pass"] * 1e-3) / 1e9
    out.update({"model": ("2048^2 -> 4096^2, f=2, shifts (dx, dy) (0.5, 0), (0, 0.5), (-0.5, 0), (0, -0.5) LR px, "
                          "2x2 binning D, 3x3 Gaussian sigma 0.5, L1 data term eps_d 0.01, lambda 0.05, BTV alpha "
                          "0.4 w 3 eps 1e-3, 20 SCG iterations"),
                "pass": "frame-wise (7 gather kernels and the reduction per SCG pass)",
                "pass_bytes_per_px": GEN_PASS_BYTES_PER_PX_L1, "pass_achieved_gbs": gen_achieved,
                "pass_frac": gen_achieved / peak,
                "frac_basis": "frac and achieved_gbs: the fused pass's 28 B/px; pass_frac: the frame-wise pass's "
                              "own 156 B/px"})
    return out


def measure_interpolation(args, wl, plan, y, xt, stream, dist, device, peak):
    """Multi-image interpolation (misr_interpolate), the paper's non-iterative comparator, on
    the same frames: rate, HBM bandwidth (frames read once, HR image written once) and the image
    error against the phantom beside that of the SCG solve."""
    import torch
    H, W = wl["f"] * wl["h"], wl["f"] * wl["w"]
    xi = torch.empty((H, W), dtype=torch.float32, device=device)
    for _ in range(max(args.warmup, 3)):
        plan.interpolate(y, xi)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    reps = 20 * args.steps
    # L2 flush before each call: a 256 MB write evicts the call's data, and a 256 MB read of
    # another buffer then evicts the written (dirty) lines, so that their write-back happens
    # here and not inside the timed call
    flush = torch.empty(64 * 2**20, dtype=torch.float32, device=device)
    flush_r = torch.zeros(64 * 2**20, dtype=torch.float32, device=device)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in evs:
        flush.zero_()
        flush_r.sum()
        e0.record(stream)
        plan.interpolate(y, xi)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs) / reps
    del flush, flush_r
    rate, _ = job_rate(reps, ms * reps / 1e3, dist, device)
    nbytes = y.numel() * 4 + H * W * 4
    xs = plan.solve(y)[0]
    err = lambda a: float(torch.linalg.vector_norm(a - xt) / torch.linalg.vector_norm(xt))
    return {"value": rate, "unit": UNIT, "ms": ms, "achieved_gbs": nbytes / (ms * 1e-3) / 1e9,
            "frac": nbytes / (ms * 1e-3) / 1e9 / peak, "bytes_per_call": nbytes,
            "image_rel_error_vs_phantom": {"interpolation": err(xi), "scg_%d_it" % wl["iters"]: err(xs)},
            "timed_as": "%d calls of misr_interpolate, each timed alone with CUDA events on the stream "
                        "after a 256 MB write and a 256 MB read of another buffer that flush L2 "
                        "(the written lines are evicted, and written back, before the call)" % reps}


ORACLE_SAMPLE_ITERS = 3


def oracle_timing(h, w, f, seed, iters):
    """Seconds of the FP64 oracle for one problem of h x w LR frames: (init, per SCG iteration).
    init = shift-and-add plus the initial gradient; the iteration time is (T(init + iters SCG
    iterations) - T(init)) / iters, so that the first iteration's extra work is averaged in."""
    from oracle import oracle
    P = oracle.Problem(h, w, f, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5), lam=0.01)
    xt = gen.phantom(P.H, P.W, seed)
    y = P.forward_all(xt) + gen.gaussian_noise((4, h, w), 0.01, seed + 1)
    del xt
    t = time.perf_counter()
    P.scg(y, P.shift_add(y), 0)
    t0 = time.perf_counter() - t
    t = time.perf_counter()
    P.scg(y, P.shift_add(y), iters)
    tk = time.perf_counter() - t
    return t0, max((tk - t0) / iters, 1e-9), oracle.threads()


def _one_core_timing(h, w, f, seed, iters):
    """oracle_timing in a child process whose OpenMP runtime has one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_timing(%d, %d, %d, %d, %d)))" % (ROOT, h, w, f, seed, iters))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(wl):
    """The FP64 oracle on the host cores at the workload's full size (init + 3 SCG iterations,
    extrapolated to the workload's iteration count), and on one core for a 1/16 crop of it
    (h/4 x w/4 LR frames, same recipe), scaled to full size by the HR pixel count (the oracle's
    work per iteration is linear in the pixels)."""
    t0, t_iter, cores = oracle_timing(wl["h"], wl["w"], wl["f"], wl["seed"], ORACLE_SAMPLE_ITERS)
    per_proj = t0 + wl["iters"] * t_iter
    out = {"value": 1.0 / per_proj, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"FP64 oracle, full-size problem: init {t0:.2f} s, then {ORACLE_SAMPLE_ITERS} SCG iterations "
                     f"at {t_iter:.2f} s each; projections/s = 1 / (init + {wl['iters']} iterations)"}
    # the tiny workload end to end (every SCG iteration run, nothing extrapolated)
    tw = WORKLOADS["tiny"]
    from oracle import oracle
    Pt = oracle.Problem(tw["h"], tw["w"], tw["f"], gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5), lam=0.01)
    yt = Pt.forward_all(gen.phantom(Pt.H, Pt.W, tw["seed"])) + gen.gaussian_noise((4, tw["h"], tw["w"]), 0.01,
                                                                                  tw["seed"] + 1)
    t = time.perf_counter()
    Pt.scg(yt, Pt.shift_add(yt), tw["iters"])
    t_tiny = time.perf_counter() - t
    out["tiny_end_to_end"] = {"value": 1.0 / t_tiny, "unit": UNIT, "cores": oracle.threads(),
                              "sample": f"{tw['desc']}: shift-and-add and the full {tw['iters']}-iteration solve, "
                                        f"{t_tiny * 1e3:.0f} ms"}
    h1, w1 = wl["h"] // 4, wl["w"] // 4
    one = _one_core_timing(h1, w1, wl["f"], wl["seed"], ORACLE_SAMPLE_ITERS)
    if one is not None:
        scale = (wl["h"] * wl["w"]) / (h1 * w1)
        per1 = scale * (one[0] + wl["iters"] * one[1])
        out["one_core"] = {"value": 1.0 / per1, "unit": UNIT, "cores": one[2],
                           "sample": f"{h1}x{w1} LR crop on one thread: init {one[0]:.2f} s, SCG iteration "
                                     f"{one[1]:.2f} s, x{scale:.0f} to full size"}
    return out


def run_reference(args, wl):
    """Reference arm: the FP64 oracle as it stands, on the host cores, with cpu_baseline's
    estimator.  Every step is one full-size sample (init + 3 SCG iterations); the line reports
    the median step's rate."""
    warm = max(0, min(args.warmup, 1))
    for _ in range(warm):
        oracle_timing(wl["h"], wl["w"], wl["f"], wl["seed"], 1)
    samples = [oracle_timing(wl["h"], wl["w"], wl["f"], wl["seed"], ORACLE_SAMPLE_ITERS) for _ in range(args.steps)]
    per = sorted(t0 + wl["iters"] * ti for t0, ti, _ in samples)
    per_proj = statistics.median(per)
    cores = samples[0][2] if samples else 0
    value = 1.0 / per_proj
    sample = (f"FP64 oracle, full-size problem; each step = init + {ORACLE_SAMPLE_ITERS} SCG iterations, "
              f"extrapolated to {wl['iters']} iterations (median of {len(per)} steps; "
              f"range {per[0]:.1f}-{per[-1]:.1f} s per projection)")
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": warm, "ms_per_step": per_proj * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": wl["desc"], "lr": [wl["h"], wl["w"]], "K": 4, "factor": wl["f"], "iters": wl["iters"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def batch_uneven_record(n, iters, steps, warmup):
    """The batch form on uneven projections: the first n of 64 seeded ROIs (LR sides
    U{512..2048}; alternately f=2/K=4 and f=3/K=9), `iters` SCG iterations each.  One batched
    solve (one fused-pass launch per SCG step over all n projections) against the same
    projections solved one after another with misr_solve, on the same GPU and stream."""
    import torch
    from paper_2108_04315_b300.binding import Batch, Plan
    device = torch.device("cuda", torch.cuda.current_device())
    rois = gen.batch_rois(gen.CONFIG_SEEDS["batch"], n=64)[:n]
    big = torch.from_numpy(gen.phantom(6144, 6144, gen.CONFIG_SEEDS["batch"]).astype(np.float32)).to(device)
    g = torch.Generator(device=device)
    g.manual_seed(gen.CONFIG_SEEDS["batch"])
    rng = np.random.default_rng(gen.CONFIG_SEEDS["batch"])
    plans, ys = [], []
    for r in rois:
        p = Plan(r["h"], r["w"], r["f"], r["shifts"], gen.gaussian_psf(5, 0.5), lam=0.01, iters=iters)
        oy = int(rng.integers(0, 6144 - p.H + 1))
        ox = int(rng.integers(0, 6144 - p.W + 1))
        xt = big[oy:oy + p.H, ox:ox + p.W].contiguous()
        y = p.forward(xt)
        y += 0.01 * torch.randn(y.shape, generator=g, device=device)
        plans.append(p)
        ys.append(y)
    del big
    xs = [torch.empty((p.H, p.W), dtype=torch.float32, device=device) for p in plans]
    batch = Batch(plans)
    stream = torch.cuda.current_stream()
    for _ in range(max(1, warmup)):
        batch.solve(ys, xs, stats=False)
        for p, y, x in zip(plans, ys, xs):
            p.solve(y, x, stats=False)
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    with ClockSampler(device.index) as clk:
        e0.record(stream)
        for _ in range(steps):
            batch.solve(ys, xs, stats=False)
        e1.record(stream)
        for _ in range(steps):
            for p, y, x in zip(plans, ys, xs):
                p.solve(y, x, stats=False)
        e2.record(stream)
        e2.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    t_plain = e1.elapsed_time(e2) / 1e3
    px = sum(p.H * p.W for p in plans)
    n_f3 = sum(1 for r in rois if r["f"] == 3)
    out = {"value": n * steps / t_batch, "unit": UNIT, "steps": steps, "warmup": max(1, warmup),
           "ms_per_step": t_batch / steps * 1e3, "api": "misr_batch_solve",
           "config": {"workload": f"{n} projections, LR sides U{{512..2048}}, {n - n_f3} x (f=2, K=4) + "
                                  f"{n_f3} x (f=3, K=9), {iters} SCG iterations",
                      "hr_pixels_total": px, "projections": n, "iters": iters},
           "plain": {"value": n * steps / t_plain, "unit": UNIT, "ms_per_step": t_plain / steps * 1e3,
                     "api": "misr_solve, one projection after another"},
           "over_plain": t_plain / t_batch,
           "hr_pixels_per_s": px * steps / t_batch,
           "clocks": clk.summary()}
    batch.close()
    for p in plans:
        p.close()
    return out


def run_batch(args):
    """`--workload batch`: the 64-projection uneven batch at 60 SCG iterations."""
    import torch
    torch.cuda.set_device(0)
    rec = batch_uneven_record(args.batch_n, 60, args.steps, min(args.warmup, 2))
    out = {"metric": "SR projections/s (64 uneven projections, 60 SCG it, batched)", "n_gpus": 1,
           "higher_is_better": True, "dtype": "f32", "data": "synthetic", "impl": "misr-batch", **rec}
    print(json.dumps(out), flush=True)


def precision_record(h, steps, warmup):
    """The precision form: 4 x h^2 uint16 counts (Poisson, I0 40000) of a seeded phantom,
    log-converted on the device, (2h)^2 HR, 100 SCG iterations; r and p stored in bf16 with the
    float master x, against the all-float solve of the same counts on the same GPU."""
    import torch
    from paper_2108_04315_b300.binding import MISR_BF16, MISR_F32, MISR_U16, Plan
    device = torch.device("cuda", torch.cuda.current_device())
    w = h
    f, iters, seed = 2, 100, gen.CONFIG_SEEDS["precision"]
    sh, psf = gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)
    plans = {name: Plan(h, w, f, sh, psf, lam=0.01, iters=iters, in_dtype=MISR_U16, flat_field=FLAT_FIELD,
                        iterate_dtype=dt) for name, dt in (("f32", MISR_F32), ("bf16", MISR_BF16))}
    xt = torch.from_numpy(gen.phantom(f * h, f * w, seed).astype(np.float32)).to(device)
    m = plans["f32"].forward(xt)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    c = torch.poisson(FLAT_FIELD * torch.exp(-m), generator=g).clamp_(1, 65535).to(torch.int32)
    y = torch.where(c > 32767, c - 65536, c).to(torch.int16).contiguous()
    del c, m, xt
    xs = {k: torch.empty((f * h, f * w), dtype=torch.float32, device=device) for k in plans}
    stream = torch.cuda.current_stream()
    for _ in range(max(warmup, 3)):
        for k, p in plans.items():
            p.solve(y, xs[k], stats=False)
    torch.cuda.synchronize()
    res = {}
    with ClockSampler(device.index) as clk:
        for k, p in plans.items():
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                p.solve(y, xs[k], stats=False)
            e1.record(stream)
            e1.synchronize()
            res[k] = e0.elapsed_time(e1) / steps
    st = {k: p.solve(y, xs[k])[1] for k, p in plans.items()}
    diff = float(torch.linalg.vector_norm(xs["bf16"] - xs["f32"]) / torch.linalg.vector_norm(xs["f32"]))
    out = {"value": 1e3 / res["bf16"], "unit": UNIT, "steps": steps, "warmup": max(warmup, 3),
           "ms_per_step": res["bf16"], "dtype": "f32 (x) + bf16 (r, p); u16 frames",
           "config": {"workload": f"4 x {h}^2 u16 counts (Poisson, I0 40000) -> {f * h}^2 HR, f=2, half-pixel "
                                  "shifts, lambda 0.01, 100 SCG iterations", "hr_pixels": f * h * f * w},
           "plain": {"value": 1e3 / res["f32"], "unit": UNIT, "ms_per_step": res["f32"],
                     "dtype": "f32 (x, r, p); u16 frames", "workspace_bytes": plans["f32"].workspace_bytes()},
           "over_plain": res["f32"] / res["bf16"],
           "workspace_bytes": plans["bf16"].workspace_bytes(),
           "workspace_over_plain": plans["bf16"].workspace_bytes() / plans["f32"].workspace_bytes(),
           "image_rel_l2_vs_plain": diff,
           "J_final_rel_vs_plain": abs(st["bf16"]["J_final"] - st["f32"]["J_final"]) / st["f32"]["J_final"],
           "accepted": {k: v["accepted"] for k, v in st.items()},
           "clocks": clk.summary()}
    for p in plans.values():
        p.close()
    return out


def run_precision(args):
    """`--workload precision`: the 3072^2 u16 workload at full length."""
    import torch
    torch.cuda.set_device(0)
    rec = precision_record(3072, args.steps, args.warmup)
    out = {"metric": "SR projections/s (3072^2 u16 -> 6144^2, 100 SCG it, bf16 r and p)", "n_gpus": 1,
           "higher_is_better": True, "data": "synthetic", "impl": "misr-precision", **rec}
    print(json.dumps(out), flush=True)


SERVE_SCANS = {
    # scan A: full detector, f=2, K=4 half-pixel shifts; scan B: ROIs at f=3, K=9 third-pixel shifts
    "A": dict(h=1536, w=1920, f=2, shifts=gen.half_pixel_shifts()),
    "B": dict(h=768, w=960, f=3, shifts=gen.third_pixel_shifts()),
}
SERVE_ITERS = 80
SERVE_RATE = 30.0   # projections arriving per second (A and B alternate)
SERVE_SPIN_US = 50000   # the served arm's worker polls this long for the next request once idle
FLAT_FIELD = 40000.0


def _serving_inputs(device, n_pool):
    """Per scan: a plan (u16 frames, log-converted on the device) and a pool of projections,
    counts = clamp(Poisson(I0 exp(-A_k x)), 1, 65535) of a seeded phantom, stored as uint16 bits."""
    import torch
    from paper_2108_04315_b300.binding import MISR_U16, Plan
    seed = gen.CONFIG_SEEDS["serving"]
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    psf = gen.gaussian_psf(5, 0.5)
    out = {}
    for i, (name, sc) in enumerate(SERVE_SCANS.items()):
        plan = Plan(sc["h"], sc["w"], sc["f"], sc["shifts"], psf, lam=0.01, iters=SERVE_ITERS, in_dtype=MISR_U16,
                    flat_field=FLAT_FIELD)
        xt = torch.from_numpy(gen.phantom(plan.H, plan.W, seed + i).astype(np.float32)).to(device)
        m = plan.forward(xt)
        pool = []
        for _ in range(n_pool):
            c = torch.poisson(FLAT_FIELD * torch.exp(-m), generator=g).clamp_(1, 65535).to(torch.int32)
            pool.append(torch.where(c > 32767, c - 65536, c).to(torch.int16).contiguous())
        out[name] = dict(plan=plan, pool=pool, psf=psf, **sc)
    torch.cuda.synchronize()
    return out


def _pct(v, q):
    return float(np.percentile(np.asarray(v), q)) * 1e3 if v else None


def serving_record(n, slots, tick):
    """Simulated CT acquisition (the served form): a projection every 1/30 s, scan A and scan B
    alternating, 80 SCG iterations each from uint16 counts.  Served = misr_submit at arrival
    (continuous batching on the device); plain = one misr_solve at a time in arrival order.
    Then an open-loop overload run (all requests at once) for the peak served rate."""
    import torch
    from paper_2108_04315_b300.binding import MISR_U16, Server, make_desc
    device = torch.device("cuda", torch.cuda.current_device())
    scans = _serving_inputs(device, n_pool=4)
    names = ["A" if i % 2 == 0 else "B" for i in range(n)]
    xs = [torch.empty((scans[k]["plan"].H, scans[k]["plan"].W), dtype=torch.float32, device=device) for k in names]
    ys = [scans[k]["pool"][(i // 2) % len(scans[k]["pool"])] for i, k in enumerate(names)]
    srv = Server(max_slots=slots, passes_per_tick=tick, idle_spin_us=SERVE_SPIN_US)
    # one descriptor per scan, made once (as the plain arm's plans are)
    descs = {k: make_desc(sc["h"], sc["w"], sc["f"], sc["shifts"], sc["psf"], lam=0.01, iters=SERVE_ITERS,
                          in_dtype=MISR_U16, flat_field=FLAT_FIELD) for k, sc in scans.items()}

    def submit(i):
        return srv.submit_desc(ys[i], descs[names[i]], xs[i])

    # warm-up: one untimed burst of every request, so that the server's slot pool (a plan per
    # slot, kept between requests as a running server keeps it) exists before the timed runs;
    # and both classes solved plainly
    for t in [submit(i) for i in range(n)]:
        srv.wait(t, 600.0)
    for i in range(min(2, n)):
        scans[names[i]]["plan"].solve(ys[i], xs[i], stats=False)
    torch.cuda.synchronize()

    clocks = ClockSampler(device.index)
    with clocks:
        # 1. served, paced arrivals
        t0 = time.monotonic() + 0.05
        arrive = [t0 + i / SERVE_RATE for i in range(n)]
        tickets = []
        for i in range(n):
            d = arrive[i] - time.monotonic()
            if d > 0:
                time.sleep(d)
            tickets.append(submit(i))
        lat_srv, t_last = [], 0.0
        for i, t in enumerate(tickets):
            x, st, times = srv.wait(t, 600.0)
            lat_srv.append(times[2] - arrive[i])
            t_last = max(t_last, times[2])
        served_rate = n / (t_last - arrive[0])
        # 2. plain, same arrivals
        stream = torch.cuda.current_stream()
        t0 = time.monotonic() + 0.05
        arrive = [t0 + i / SERVE_RATE for i in range(n)]
        lat_plain, t_last = [], 0.0
        for i in range(n):
            d = arrive[i] - time.monotonic()
            if d > 0:
                time.sleep(d)
            scans[names[i]]["plan"].solve(ys[i], xs[i], stats=False)
            stream.synchronize()
            t_last = time.monotonic()
            lat_plain.append(t_last - arrive[i])
        plain_rate = n / (t_last - arrive[0])
        # 3. overload: every request at once, served vs back-to-back plain solves
        tickets = [submit(i) for i in range(n)]
        t_first, t_last = None, 0.0
        for t in tickets:
            x, st, times = srv.wait(t, 600.0)
            t_first = times[0] if t_first is None else min(t_first, times[0])
            t_last = max(t_last, times[2])
        peak_served = n / (t_last - t_first)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(n):
            scans[names[i]]["plan"].solve(ys[i], xs[i], stats=False)
        e1.record(stream)
        e1.synchronize()
        peak_plain = n / (e0.elapsed_time(e1) / 1e3)
    counters = srv.counters()
    srv.close()
    out = {"value": served_rate, "unit": UNIT, "steps": n, "warmup": n,
           "config": {"workload": "scan A: 4 x 1536x1920 u16 counts, f=2, half-pixel shifts; scan B: 9 x 768x960 u16 "
                                  "counts, f=3, third-pixel shifts; I0 40000, lambda 0.01, 80 SCG iterations; one "
                                  f"projection every {1 / SERVE_RATE:.4f} s alternating A/B; {n} projections",
                      "max_slots": slots, "passes_per_tick": tick, "idle_spin_us": SERVE_SPIN_US,
                      "inputs": "resident in HBM (frames > L2 per projection)",
                      "warmup": "one untimed burst of all requests (the slot pool is made), 2 plain solves"},
           "api": "misr_submit at arrival, misr_wait",
           "latency_ms": {"served_p50": _pct(lat_srv, 50), "served_p99": _pct(lat_srv, 99),
                          "plain_p50": _pct(lat_plain, 50), "plain_p99": _pct(lat_plain, 99),
                          # per scan (the two scans' latencies are far apart, so the medians of
                          # the mix above jump between them)
                          "by_scan": {k: {"served_p50": _pct([l for l, q in zip(lat_srv, names) if q == k], 50),
                                          "served_p99": _pct([l for l, q in zip(lat_srv, names) if q == k], 99),
                                          "plain_p50": _pct([l for l, q in zip(lat_plain, names) if q == k], 50),
                                          "plain_p99": _pct([l for l, q in zip(lat_plain, names) if q == k], 99)}
                                      for k in sorted(set(names))}},
           "plain": {"value": plain_rate, "unit": UNIT, "api": "misr_solve at arrival, one at a time",
                     "latency_p50_ms": _pct(lat_plain, 50), "latency_p99_ms": _pct(lat_plain, 99)},
           "p50_over_plain": _pct(lat_plain, 50) / _pct(lat_srv, 50),
           "p99_over_plain": _pct(lat_plain, 99) / _pct(lat_srv, 99),
           "overload": {"served": peak_served, "plain": peak_plain, "served_over_plain": peak_served / peak_plain,
                        "unit": UNIT},
           "server_counters": counters, "clocks": clocks.summary()}
    for sc in scans.values():
        sc["plan"].close()
    return out


def run_serving(args):
    """`--workload serving`: the paced acquisition with --serve-n projections."""
    import torch
    torch.cuda.set_device(0)
    rec = serving_record(args.serve_n, args.serve_slots, args.serve_tick)
    out = {"metric": "served SR projections/s (CT acquisition at 30/s, scans A/B alternating, 80 SCG it)",
           "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic", "impl": "misr-serve", **rec}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="misr", choices=["misr", "reference"])
    ap.add_argument("--workload", default="detector", choices=sorted(WORKLOADS) + ["batch", "serving", "precision"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the serving, precision and uneven-batch records of the default run")
    ap.add_argument("--batch-n", type=int, default=64)
    ap.add_argument("--serve-n", type=int, default=240)
    ap.add_argument("--serve-slots", type=int, default=32)
    ap.add_argument("--serve-tick", type=int, default=8)
    ap.add_argument("--tile-shape", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="0: autotune (default); 1: 32x64, 2: 32x32, 3: 16x64, 4: row-streaming")
    args = ap.parse_args()
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    if args.workload == "precision":
        run_precision(args)
        return
    wl = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, wl)), flush=True)
        return

    import torch
    from paper_2108_04315_b300.binding import Plan

    torch.cuda.set_device(local_rank)
    device = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    stream = torch.cuda.current_stream()
    H, W = wl["f"] * wl["h"], wl["f"] * wl["w"]
    shifts, psf = gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)
    # the autotuner times each tile shape on this geometry; the plans below get the fastest
    # (--tile-shape fixes one instead, e.g. for profiling runs where timings are distorted)
    from paper_2108_04315_b300.binding import make_desc, misr_autotune
    if args.tile_shape:
        tuned, tune_ms = args.tile_shape, [None] * len(TILE_SHAPES)
    else:
        tuned, tune_ms = misr_autotune(make_desc(wl["h"], wl["w"], wl["f"], shifts, psf, iters=1), passes=10)
    th, tw, nt = TILE_SHAPES[tuned]
    shape_name = shape_label(tuned)
    plan = Plan(wl["h"], wl["w"], wl["f"], shifts, psf, lam=0.01, btv_alpha=0.4, btv_w=3, eps=1e-3,
                iters=wl["iters"], tile_shape=tuned)
    plan0 = Plan(wl["h"], wl["w"], wl["f"], shifts, psf, lam=0.01, btv_alpha=0.4, btv_w=3, eps=1e-3, iters=0,
                 tile_shape=tuned)
    xt, y = make_inputs(plan, wl, device)
    x = torch.empty((H, W), dtype=torch.float32, device=device)

    for _ in range(max(args.warmup, 3)):
        plan.solve(y, x, stats=False)
        plan0.solve(y, x, stats=False)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # timed region: K full solves, inputs resident in HBM (working set 470 MB > 126 MB L2)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            plan.solve(y, x, stats=False)
        ev1.record(stream)
        ev1.synchronize()
        barrier()
    ms_total = ev0.elapsed_time(ev1)
    clocks = clk.summary()
    # per-pass time: the same solves with 0 SCG iterations, on the same stream
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(args.steps):
        plan0.solve(y, x, stats=False)
    ev3.record(stream)
    ev3.synchronize()
    ms0 = ev2.elapsed_time(ev3)
    pass_ms = max((ms_total - ms0) / args.steps / wl["iters"], 1e-9)
    st = plan.solve(y, x, stats=True)[1]

    value, s_total = job_rate(args.steps, ms_total / 1e3, dist, device)
    ms_total = s_total * 1e3

    # end to end through the C ABI with host buffers (page-locked): every step copies its
    # frames to the device and its image back.  misr_solve_host_many streams the steps'
    # projections through the plan, the copies of one overlapping the solve of another;
    # misr_solve_host (copy, solve, copy, one projection per call) is reported beside it.
    y_hosts = [y.cpu().pin_memory() for _ in range(2)]
    x_hosts = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(2)]
    yh = [t.numpy() for t in y_hosts]
    xh = [t.numpy() for t in x_hosts]
    plan.solve_host_many(yh, xh, stats=False)
    barrier()
    t = time.perf_counter()
    plan.solve_host_many([yh[k & 1] for k in range(args.steps)], [xh[k & 1] for k in range(args.steps)],
                         stats=False)
    e2e_rate, _ = job_rate(args.steps, time.perf_counter() - t, dist, device)
    barrier()
    t = time.perf_counter()
    for k in range(args.steps):
        plan.solve_host(yh[k & 1], xh[k & 1])
    serial_rate, _ = job_rate(args.steps, time.perf_counter() - t, dist, device)
    e2e = {"value": e2e_rate, "unit": UNIT, "h2d_bytes_per_step": int(y.numel() * 4),
           "d2h_bytes_per_step": int(H * W * 4), "api": "misr_solve_host_many (copies overlapped with solves)",
           "one_call_per_step": {"value": serial_rate, "unit": UNIT, "api": "misr_solve_host"}}

    # the batch form on this configuration: NB projections advanced by one pass launch per SCG
    # step (misr_batch_solve), against the plain one-projection-at-a-time rate above
    from paper_2108_04315_b300.binding import Batch
    NB = 4
    plans_b = [Plan(wl["h"], wl["w"], wl["f"], shifts, psf, lam=0.01, btv_alpha=0.4, btv_w=3, eps=1e-3,
                    iters=wl["iters"], tile_shape=tuned) for _ in range(NB)]
    batch = Batch(plans_b)
    xs_b = [torch.empty((H, W), dtype=torch.float32, device=device) for _ in range(NB)]
    batch.solve([y] * NB, xs_b, stats=False)
    n_b = max(1, (args.steps + NB - 1) // NB)
    ev4, ev5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev4.record(stream)
    for _ in range(n_b):
        batch.solve([y] * NB, xs_b, stats=False)
    ev5.record(stream)
    ev5.synchronize()
    batched_rate, _ = job_rate(n_b * NB, ev4.elapsed_time(ev5) / 1e3, dist, device)
    batch.close()
    for pb in plans_b:
        pb.close()
    batched = {"value": batched_rate, "unit": UNIT, "projections": NB, "over_plain": batched_rate / value,
               "api": "misr_batch_solve (%d projections of this configuration; each fills the GPU, so each runs its "
                      "own pass launches on a stream of its own, overlapped within every step)" % NB}

    peak, peak_kind = load_peaks()
    achieved = PASS_BYTES_PER_PX * H * W / (pass_ms * 1e-3) / 1e9
    # the L1 lines run on the shape tuned for this image size (every shape takes the L1 term)
    l1 = measure_l1(args, wl, shifts, psf, tuned, y, xt, stream, dist, device, peak)
    paper_ct = measure_paper_ct(args, wl, shifts, tuned, xt, stream, dist, device, peak)
    subpixel = measure_subpixel(args, wl, xt, stream, dist, device, peak)
    study = measure_study(args, wl, xt, stream, dist, device, peak)
    interp = measure_interpolation(args, wl, plan, y, xt, stream, dist, device, peak)
    # the three forms beside their plain counterparts, at sizes that keep the default run
    # within minutes: the paced acquisition (60 projections), the 3072^2 u16 precision
    # workload (3 solves per arm) and 16 of the 64 uneven projections (2 batched steps)
    forms = None
    if world == 1 and not args.no_forms and args.workload == "detector":
        forms = {"serving": serving_record(60, args.serve_slots, args.serve_tick),
                 "precision": precision_record(3072, 3, 3),
                 "batch_uneven": batch_uneven_record(16, 60, 2, 1)}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["desc"], "lr": [wl["h"], wl["w"]], "K": 4, "factor": wl["f"],
                   "iters": wl["iters"], "hr_pixels": H * W,
                   "l2": "no flush: per-solve working set 7 HR float32 images = %d MB > 126 MB L2"
                         % (7 * H * W * 4 // 2**20),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": load_traffic(kernel_source_tag(), shape_name),
                     "kernel": ("scg_stream_kernel<false>" if tuned == 4 else f"scg_pass_kernel<{th},{tw},{nt}>"),
                     "peak_kind": peak_kind,
                     "spec_peak": SPEC_HBM_GBS, "frac_of_spec": achieved / SPEC_HBM_GBS,
                     "algorithmic_bytes_per_launch": PASS_BYTES_PER_PX * H * W,
                     "ms_per_launch": pass_ms,
                     "timed_as": "one SCG pass (the fused pass kernel with its reduction: in the pass for the "
                                 "streaming kernel, a reduction kernel after it for the tile shapes), "
                                 "(T(100 it) - T(0 it)) / 100 with CUDA events on the solve's stream"},
        "e2e": e2e,
        "batched": batched,
        "l1": l1,
        "paper_ct_setting": paper_ct,
        "subpixel": subpixel,
        "synthetic_study_frames": study,
        "interpolation": interp,
        "forms": forms,
        # per solve: prepare, the initial pass and every SCG pass (the fused pass kernel, and
        # for the tile shapes its reduction kernel; the streaming pass reduces in the pass),
        # finalize
        "gpu_launches": args.steps * ((wl["iters"] + 1) * (1 if tuned == 4 else 2) + 2),
        "tile_shape": {"tuned": shape_name, "threads": nt,
                       "ms_per_pass_by_shape": {shape_label(k): (None if v is None else round(float(v), 5))
                                                for k, v in zip(sorted(TILE_SHAPES), tune_ms)}},
        "clocks": clocks,
        "solve": {"J_final": st["J_final"], "accepted": st["accepted"], "iters_done": st["iters_done"]},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl)
    if rank == 0:
        print(json.dumps(out), flush=True)
    plan.close()
    plan0.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
