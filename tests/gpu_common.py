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


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a if dtype is None else a.astype(dtype)))
    return t.cuda()


def make_case(orc, h, w, f, shifts, psf, seed, lam=0.01, eps=1e-3, noise=0.01, iters=50, **plan_kw):
    """Return (oracle problem, GPU plan, x_true, y float32) for one seeded acquisition."""
    from paper_2108_04315_b300.binding import Plan
    P = orc.Problem(h, w, f, shifts, psf, lam=lam, eps=eps)
    xt = gen.phantom(f * h, f * w, seed)
    y = P.forward_all(xt) + gen.gaussian_noise((len(shifts), h, w), noise, seed + 1)
    y32 = y.astype(np.float32)
    plan = Plan(h, w, f, shifts, psf, lam=lam, eps=eps, iters=iters, **plan_kw)
    return P, plan, xt, y32
