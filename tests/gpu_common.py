"""Shared set-up of the GPU parity tests: the same seeded inputs for the CUDA library (float32)
and for the FP64 oracle (the float32 values widened)."""
import numpy as np

import gen

RTOL_OP = 1e-5      # operator applications and per-pass sums (relative L2)
RTOL_X = 1e-3       # final SR image after a fixed iteration count (relative L2)
RTOL_J = 1e-5       # objective


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def asym_separable_psf(seed, size=5):
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.1, 1.0, size)
    v = rng.uniform(0.1, 1.0, size)
    k = np.outer(u, v)
    return k / k.sum()


# Geometries of the parity tests: name -> (h, w, f, shifts, psf)
PARITY_CASES = {
    "tiny_f2": (64, 64, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)),
    "ragged_f2_asym": (37, 53, 2, gen.half_pixel_shifts(), asym_separable_psf(3)),
    "ragged_f3_k9": (23, 29, 3, gen.third_pixel_shifts(), gen.gaussian_psf(5, 0.5)),
    "partial_f2_k3": (30, 41, 2, [(0.0, 0.0), (0.5, 0.0), (0.5, 0.5)], asym_separable_psf(4, 3)),
    "f3_k5_psf3": (19, 40, 3, [(0.0, 0.0), (2 / 3, 0.0), (1 / 3, 1 / 3), (0.0, 2 / 3), (2 / 3, 2 / 3)],
                   gen.gaussian_psf(3, 0.7)),
    "f1_denoise": (45, 70, 1, [(0.0, 0.0)], gen.gaussian_psf(5, 0.6)),
    "f4_k16": (17, 21, 4, gen.phase_shifts(4), gen.gaussian_psf(5, 1.0)),
    "single_pixel": (1, 1, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)),
    "thin_strip": (1, 97, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)),
}

# Iteration counts of the solves on the extra geometries (seed 400) and of the u16 solve.
# tests/test_fp32_sensitivity.py shows, with the oracle alone, that up to these counts storing
# the SCG state in FP32 moves the FP64 run's objective by at most a fifth of the 1e-5 bar at
# every count (and its image by far less than 1e-3), and that at the longer counts used before
# (partial_f2_k3: 10, ragged_f2_asym: 30, u16: 20) that floor is above a fifth of the bar or the
# bar itself, for any FP32-state implementation.
OTHER_GEOMETRY_ITERS = {"ragged_f3_k9": 25, "partial_f2_k3": 6, "f1_denoise": 20, "f4_k16": 15,
                        "ragged_f2_asym": 18}
OTHER_GEOMETRY_SEED = 400
U16_ITERS = 10


def oracle_case(orc, h, w, f, shifts, psf, seed, lam=0.01, eps=1e-3, noise=0.01, **problem_kw):
    """(oracle problem, x_true, y float32) for one seeded acquisition (no GPU needed)."""
    P = orc.Problem(h, w, f, shifts, psf, lam=lam, eps=eps, **problem_kw)
    xt = gen.phantom(f * h, f * w, seed)
    y = P.forward_all(xt) + gen.gaussian_noise((len(shifts), h, w), noise, seed + 1)
    return P, xt, y.astype(np.float32)


def u16_case(orc, **problem_kw):
    """The u16 detector-count case: (oracle problem, counts, y = the oracle's log conversion)."""
    h, w, f = 48, 40, 2
    P = orc.Problem(h, w, f, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5), lam=0.01, **problem_kw)
    xt = gen.phantom(f * h, f * w, 600)
    counts = gen.poisson_counts(P.forward_all(xt), 40000.0, 601)
    return P, counts, orc.log_convert(counts, 40000.0)


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a if dtype is None else a.astype(dtype)))
    return t.cuda()


def make_case(orc, h, w, f, shifts, psf, seed, lam=0.01, eps=1e-3, noise=0.01, iters=50, **plan_kw):
    """Return (oracle problem, GPU plan, x_true, y float32) for one seeded acquisition."""
    from paper_2108_04315_b300.binding import Plan
    P, xt, y32 = oracle_case(orc, h, w, f, shifts, psf, seed, lam=lam, eps=eps, noise=noise)
    plan = Plan(h, w, f, shifts, psf, lam=lam, eps=eps, iters=iters, **plan_kw)
    return P, plan, xt, y32


# Frame sets that do not interleave into one HR image (the frame-wise pass): name -> (h, w, f,
# shifts, psf, decimation: 0 point, 1 binning).  STUDY_SHIFTS: the synthetic study's one-pixel
# shifts right, down, left and up at 2x (Sec. 4.1.1), two frames on each of two phases.
STUDY_SHIFTS = [(0.5, 0.0), (0.0, 0.5), (-0.5, 0.0), (0.0, -0.5)]
GENERAL_CASES = {
    "study_bin_psf3": (40, 52, 2, STUDY_SHIFTS, gen.gaussian_psf(3, 0.6), 1),
    "study_point_psf5": (37, 45, 2, STUDY_SHIFTS, gen.gaussian_psf(5, 0.5), 0),
    "dup_phase_k6": (30, 41, 2, [(0.0, 0.0), (0.5, 0.0), (0.0, 0.5), (0.5, 0.5), (0.0, 0.0), (0.5, 0.5)],
                     asym_separable_psf(4), 0),
    "neg_large": (29, 33, 2, [(-0.5, -0.5), (1.0, 0.0), (0.0, 1.5), (0.5, -1.0)], gen.gaussian_psf(5, 0.5), 0),
    "off_lattice": (31, 27, 2, [(0.0, 0.0), (0.3, 0.0), (0.0, 0.55), (0.45, 0.6)], gen.gaussian_psf(5, 0.5), 0),
    "off_lattice_bin": (26, 30, 2, [(0.1, 0.2), (0.6, 0.05), (0.35, 0.7), (0.8, 0.9)], gen.gaussian_psf(3, 0.6), 1),
    "wide_bin_f3": (21, 25, 3, gen.third_pixel_shifts(), gen.gaussian_psf(5, 0.6), 1),
    "f1_subpixel": (45, 50, 1, [(0.0, 0.0), (0.5, 0.0), (0.0, 0.5), (0.5, 0.5)], gen.gaussian_psf(3, 0.7), 0),
    "far_shifts": (12, 14, 2, [(0.0, 0.0), (8.0, 0.0), (-3.5, 2.25), (30.0, -30.0)], gen.gaussian_psf(3, 0.6), 0),
    "thin_strip": (1, 61, 2, STUDY_SHIFTS, gen.gaussian_psf(3, 0.6), 1),
    "single_pixel": (1, 1, 2, STUDY_SHIFTS, gen.gaussian_psf(5, 0.5), 0),
}
# Solves on these geometries (seed GENERAL_SEED): the paper's setting (L1 data term with eps_d
# 0.01, lambda 0.05, alpha 0.4, 20 iterations, Sec. 4) and the squared L2 term at lambda 0.01
# for as many iterations as the FP32-state floor allows (tests/test_fp32_sensitivity.py: up to
# these counts it stays at a fifth of the objective bar and a tenth of the image bar).
GENERAL_SEED = 400
GENERAL_PAPER_ITERS = {"study_bin_psf3": 20, "study_point_psf5": 20, "dup_phase_k6": 20, "neg_large": 20,
                       "off_lattice": 20, "off_lattice_bin": 9, "wide_bin_f3": 20, "f1_subpixel": 20}
GENERAL_L2_ITERS = {"study_bin_psf3": 7, "study_point_psf5": 7, "dup_phase_k6": 9, "neg_large": 20,
                    "off_lattice": 20, "off_lattice_bin": 7, "wide_bin_f3": 9, "f1_subpixel": 20}
PAPER_SETTING = dict(lam=0.05, l1_eps=0.01)


def general_case(orc, name, seed, lam=0.01, l1_eps=None, iters=20, noise=0.01, oracle_only=False, **plan_kw):
    """(oracle problem, GPU plan or None, x_true, y float32) for a frame-wise geometry."""
    h, w, f, shifts, psf, dec = GENERAL_CASES[name]
    kw_o = dict(data_norm=orc.NORM_L1, data_eps=l1_eps) if l1_eps else {}
    P = orc.Problem(h, w, f, shifts, psf, lam=lam, decimation=dec, **kw_o)
    xt = gen.phantom(f * h, f * w, seed)
    y = (P.forward_all(xt) + gen.gaussian_noise((len(shifts), h, w), noise, seed + 1)).astype(np.float32)
    if oracle_only:
        return P, None, xt, y
    from paper_2108_04315_b300 import binding as B
    kw_p = dict(data_norm=B.MISR_NORM_L1, data_eps=l1_eps) if l1_eps else {}
    plan = B.Plan(h, w, f, shifts, psf, lam=lam, iters=iters, decimation=dec, **kw_p, **plan_kw)
    return P, plan, xt, y
