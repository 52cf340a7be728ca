"""Child process of tests/test_gpu_bounds.py: run the odd geometries through a given build of
the library (argv[1]: library path, argv[2]: output .npz) and print its bounds-check record."""
import json
import sys

import numpy as np


def cases():
    import gen
    from tests.gpu_common import asym_separable_psf
    return {
        # name: (h, w, f, shifts, psf)
        "tiny_f2": (64, 64, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)),
        "ragged_f2_asym": (37, 53, 2, gen.half_pixel_shifts(), asym_separable_psf(3)),
        "ragged_f3_k9": (23, 29, 3, gen.third_pixel_shifts(), gen.gaussian_psf(5, 0.5)),
        "partial_f2_k3": (30, 41, 2, [(0.0, 0.0), (0.5, 0.0), (0.5, 0.5)], asym_separable_psf(4, 3)),
        "f1_denoise": (45, 70, 1, [(0.0, 0.0)], gen.gaussian_psf(5, 0.6)),
        "f4_k16": (17, 21, 4, gen.phase_shifts(4), gen.gaussian_psf(5, 1.0)),
        "single_pixel": (1, 1, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)),
        "thin_strip": (1, 97, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)),
        "tall_strip": (90, 1, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)),
        # the streaming shape's item split: several waves of left-strip items; top items only
        "split_tall": (700, 64, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)),
        "split_short": (10, 150, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)),
    }


def frames(h, w, shifts, seed):
    import gen
    return gen.random_field((len(shifts), h, w), seed, 0.0, 2.0).astype(np.float32)


def run(lib_path):
    import torch
    import gen
    from paper_2108_04315_b300 import binding as B
    B.LIB_PATH = lib_path
    out = {}
    plans = []
    for i, (name, (h, w, f, shifts, psf)) in enumerate(sorted(cases().items())):
        y = torch.from_numpy(frames(h, w, shifts, 600 + i)).cuda()
        for shape in (1, 2, 3, 4):
            for dt in (B.MISR_F32, B.MISR_BF16):
                plan = B.Plan(h, w, f, shifts, psf, iters=4, tile_shape=shape, iterate_dtype=dt)
                x, _ = plan.solve(y)
                out[f"{name}_s{shape}_d{dt}"] = x.cpu().numpy()
                # the L1 data term's variant (its owned-residual buffer; on the streaming shape,
                # the ring rows of its curvature weights)
                p1 = B.Plan(h, w, f, shifts, psf, iters=4, tile_shape=shape, iterate_dtype=dt,
                            data_norm=B.MISR_NORM_L1, data_eps=0.05)
                x1, _ = p1.solve(y)
                out[f"{name}_s{shape}_d{dt}_l1"] = x1.cpu().numpy()
                p1.close()
                if dt == B.MISR_F32 and shape == 2:
                    J, g = plan.gradient(y, x)
                    out[f"{name}_grad"] = g.cpu().numpy()
                    plans.append((plan, y))
    # non-integer shifts (per-phase taps), float and bf16 directions, L2 and L1
    fr_shifts = [(dx, dy) for dy in (0.05, 0.6) for dx in (0.0, 0.55)]
    for name, (h, w) in (("frac_ragged", (37, 45)), ("frac_strip", (1, 61)), ("frac_pixel", (1, 1))):
        y = torch.from_numpy(frames(h, w, fr_shifts, 700 + h)).cuda()
        for dt in (B.MISR_F32, B.MISR_BF16):
            for norm in (B.MISR_NORM_L2, B.MISR_NORM_L1):
                p = B.Plan(h, w, 2, fr_shifts, gen.gaussian_psf(3, 0.6), iters=4, iterate_dtype=dt, data_norm=norm,
                           data_eps=0.05)
                x, _ = p.solve(y)
                out[f"{name}_d{dt}_n{norm}"] = x.cpu().numpy()
                p.close()
    # frame sets that run the frame-wise pass (several frames per phase, shifts outside [0, f),
    # off-lattice shifts, binning, one-pixel and one-row images, the three tap widths), L2 and
    # L1, the solve from the shift-and-add start point and the gradient
    study = [(0.5, 0.0), (0.0, 0.5), (-0.5, 0.0), (0.0, -0.5)]
    general = {
        "gen_study_bin": (21, 26, 2, study, gen.gaussian_psf(3, 0.6), B.MISR_DECIM_BIN),
        "gen_far": (12, 14, 2, [(0.0, 0.0), (8.0, 0.0), (-3.5, 2.25), (30.0, -30.0)], gen.gaussian_psf(3, 0.6),
                    B.MISR_DECIM_POINT),
        "gen_off_bin": (13, 15, 2, [(0.1, 0.2), (0.6, 0.05), (0.35, 0.7), (0.8, 0.9)], gen.gaussian_psf(3, 0.6),
                        B.MISR_DECIM_BIN),
        "gen_wide_f4": (9, 11, 4, [(0.1, 0.0), (0.6, 0.3), (0.3, 0.8), (-0.4, 0.5)], gen.gaussian_psf(5, 0.8),
                        B.MISR_DECIM_BIN),
        "gen_pixel": (1, 1, 2, study, gen.gaussian_psf(5, 0.5), B.MISR_DECIM_POINT),
        "gen_strip": (1, 61, 2, study, gen.gaussian_psf(3, 0.6), B.MISR_DECIM_BIN),
        "gen_column": (40, 1, 3, study, gen.gaussian_psf(3, 0.6), B.MISR_DECIM_POINT),
    }
    gen_plans = []
    for i, (name, (h, w, f, shifts, psf, dec)) in enumerate(sorted(general.items())):
        y = torch.from_numpy(frames(h, w, shifts, 800 + i)).cuda()
        for norm in (B.MISR_NORM_L2, B.MISR_NORM_L1):
            p = B.Plan(h, w, f, shifts, psf, iters=4, decimation=dec, data_norm=norm, data_eps=0.05)
            x, _ = p.solve(y)
            out[f"{name}_n{norm}"] = x.cpu().numpy()
            J, g = p.gradient(y, x)
            out[f"{name}_n{norm}_grad"] = g.cpu().numpy()
            if norm == B.MISR_NORM_L2:
                gen_plans.append((p, y))
            else:
                p.close()
    # a batch over mixed geometries, tile shapes and storage types, and two frame-wise problems
    sel = plans[:4] + gen_plans[:2]
    batch = B.Batch([p for p, _ in sel])
    xs, _ = batch.solve([y for _, y in sel])
    for k, x in enumerate(xs):
        out[f"batch_{k}"] = x.cpu().numpy()
    batch.close()
    torch.cuda.synchronize()
    try:
        bits, first = B.misr_debug_bounds()
    except B.MisrError as e:                       # the normal build has no checks to report
        assert e.status == B.MISR_ENOTIMPL
        bits, first = 0, [0, 0, 0, 0]
    return out, bits, first


if __name__ == "__main__":
    sys.path.insert(0, sys.argv[3] if len(sys.argv) > 3 else ".")
    images, bits, first = run(sys.argv[1])
    np.savez(sys.argv[2], **images)
    print(json.dumps({"bits": bits, "first": first}))
