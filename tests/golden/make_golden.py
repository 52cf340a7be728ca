"""Write the oracle's SCG runs the tests compare against.  Calls only oracle/ and gen/.

tests/golden/tiny_scg_trace.json: the tiny workload (4 LR frames 64x64, half-pixel shifts,
f = 2, 5x5 Gaussian PSF sigma 0.5, lambda 0.01, BTV alpha 0.4, w 3, eps 1e-3, 50 iterations,
shift-and-add start).  Run from the repository root:  python -m tests.golden.make_golden

tests/golden/detector_100it.json: the detector workload (4 x 2048^2 frames -> 4096^2, the same
model, 100 iterations): the per-iteration trace, J_final, and the final image's sum, norm and
sums over 256 x 256 blocks.  About ten minutes of oracle time on 8 cores:
python -m tests.golden.make_golden --detector
"""
import json
import os

import numpy as np

import gen
from oracle import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "tiny_scg_trace.json")
OUT_DETECTOR = os.path.join(HERE, "detector_100it.json")
DETECTOR_ITERS = 100
BLOCK = 256


def tiny_problem():
    P = oracle.Problem(64, 64, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5),
                       lam=0.01, btv_alpha=0.4, btv_w=3, eps=1e-3)
    seed = gen.CONFIG_SEEDS["tiny"]
    xt = gen.phantom(128, 128, seed)
    y = P.forward_all(xt) + gen.gaussian_noise((4, 64, 64), 0.01, seed + 100)
    return P, xt, y.astype(np.float32).astype(np.float64)


def detector_problem():
    """The detector workload: 4 x 2048^2 frames of the seeded phantom through the oracle's
    D B M_k plus N(0, 0.01^2) noise, rounded to float32 (the frames the GPU reads)."""
    h = w = 2048
    P = oracle.Problem(h, w, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5),
                       lam=0.01, btv_alpha=0.4, btv_w=3, eps=1e-3)
    seed = gen.CONFIG_SEEDS["detector"]
    xt = gen.phantom(2 * h, 2 * w, seed)
    y = (P.forward_all(xt) + gen.gaussian_noise((4, h, w), 0.01, seed + 1)).astype(np.float32)
    return P, xt, y


def block_sums(x):
    H, W = x.shape
    return x.reshape(H // BLOCK, BLOCK, W // BLOCK, BLOCK).sum(axis=(1, 3))


def main_detector():
    P, xt, y = detector_problem()
    y = y.astype(np.float64)
    x, tr = P.scg(y, P.shift_add(y), DETECTOR_ITERS)
    rec = {
        "workload": "4 x 2048^2 fp32 frames -> 4096^2, f=2, half-pixel shifts, 5x5 Gaussian sigma 0.5, "
                    "lambda 0.01, alpha 0.4, w 3, eps 1e-3, 100 SCG iterations, x0 = shift-and-add",
        "trace": {k: [float(v) for v in tr[k]] for k in tr},
        "J_final": P.objective(x, y),
        "x_sum": float(x.sum()),
        "x_norm": float(np.linalg.norm(x)),
        "block": BLOCK,
        "block_sums": block_sums(x).tolist(),
    }
    with open(OUT_DETECTOR, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(OUT_DETECTOR)


def main():
    P, xt, y = tiny_problem()
    x, tr = P.scg(y, P.shift_add(y), 50)
    rec = {
        "workload": "4 x 64^2 fp32 frames -> 128^2, f=2, half-pixel shifts, 5x5 Gaussian sigma 0.5, "
                    "lambda 0.01, alpha 0.4, w 3, eps 1e-3, 50 SCG iterations, x0 = shift-and-add",
        "trace": {k: [float(v) for v in tr[k]] for k in tr},
        "J_final": P.objective(x, y),
        "x_sum": float(x.sum()),
        "x_norm": float(np.linalg.norm(x)),
    }
    with open(OUT, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(OUT)


if __name__ == "__main__":
    import sys
    main_detector() if "--detector" in sys.argv else main()
