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
