"""Write tests/golden/tiny_scg_trace.json: the oracle's SCG run on the tiny workload
(4 LR frames 64x64, half-pixel shifts, f = 2, 5x5 Gaussian PSF sigma 0.5, lambda 0.01,
BTV alpha 0.4, w 3, eps 1e-3, 50 iterations, shift-and-add start).  Calls only oracle/ and
gen/.  Run from the repository root:  python -m tests.golden.make_golden
"""
import json
import os

import numpy as np

import gen
from oracle import oracle

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_scg_trace.json")


def tiny_problem():
    P = oracle.Problem(64, 64, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5),
                       lam=0.01, btv_alpha=0.4, btv_w=3, eps=1e-3)
    seed = gen.CONFIG_SEEDS["tiny"]
    xt = gen.phantom(128, 128, seed)
    y = P.forward_all(xt) + gen.gaussian_noise((4, 64, 64), 0.01, seed + 100)
    return P, xt, y.astype(np.float32).astype(np.float64)


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
    main()
