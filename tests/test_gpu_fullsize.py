"""The detector workload at full size (4 x 2048^2 frames -> 4096^2 HR) in the launch
configuration bench.py times (its tile shape tuned first): the forward operator and the
gradient over the whole image, a short solve, the full 100-iteration solve against the
oracle's committed run (tests/golden/detector_100it.json, written by
tests/golden/make_golden.py from oracle calls alone) and a live 20-iteration solve element by
element, against the FP64 oracle; the precision workload's size (u16 counts -> 6144^2); and the
synthetic study's frame set at the headline size as bench.py times it (the frame-wise pass):
forward, gradient and a short solve against the oracle."""
import json

import numpy as np
import pytest

import gen
from tests.gpu_common import RTOL_J, RTOL_OP, RTOL_X, rel_l2, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def detector(orc):
    from paper_2108_04315_b300 import binding as B
    h = w = 2048
    f, sh, psf = 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)
    B.misr_autotune(B.make_desc(h, w, f, sh, psf, iters=1), passes=5)   # as bench.py does
    P = orc.Problem(h, w, f, sh, psf, lam=0.01)
    xt = gen.phantom(f * h, f * w, gen.CONFIG_SEEDS["detector"])
    y = (P.forward_all(xt) + gen.gaussian_noise((4, h, w), 0.01, gen.CONFIG_SEEDS["detector"] + 1)).astype(np.float32)
    return B, P, xt, y, (h, w, f, sh, psf)


def test_detector_forward_and_gradient(detector):
    B, P, xt, y, (h, w, f, sh, psf) = detector
    plan = B.Plan(h, w, f, sh, psf, lam=0.01, iters=1)
    yf = plan.forward(to_dev(xt.astype(np.float32)))
    assert rel_l2(yf.cpu().numpy(), P.forward_all(xt.astype(np.float32).astype(np.float64))) <= RTOL_OP
    x = (xt + 0.05 * gen.smooth_field(f * h, f * w, 71)).astype(np.float32)
    J, g = plan.gradient(to_dev(y), to_dev(x))
    Jr, gr = P.gradient(x.astype(np.float64), y.astype(np.float64))
    assert rel_l2(g.cpu().numpy(), gr) <= RTOL_OP
    assert J == pytest.approx(Jr, rel=RTOL_OP)
    plan.close()


def test_detector_short_solve(detector):
    B, P, xt, y, (h, w, f, sh, psf) = detector
    iters = 5
    plan = B.Plan(h, w, f, sh, psf, lam=0.01, iters=iters)
    x, st = plan.solve(to_dev(y))
    y64 = y.astype(np.float64)
    xr, _ = P.scg(y64, P.shift_add(y64), iters)
    xg = x.cpu().numpy().astype(np.float64)
    assert st["iters_done"] == iters
    assert rel_l2(xg, xr) <= RTOL_X
    assert abs(P.objective(xg, y64) - P.objective(xr, y64)) <= RTOL_J * P.objective(xr, y64)
    plan.close()


def test_detector_full_length_solve_against_golden(detector):
    """The number bench.py sells: 100 SCG iterations at 4096^2.  The oracle's run of the same
    frames is committed; the device's objective trace meets it at 1e-5 and J_final at 1e-5,
    the accept decisions agree wherever the step changes J by more than 1e-6 J (the FP32
    noise floor of the prior's sum), and the final image's sum, norm and 256 x 256 block sums
    meet the oracle's at the image tolerance."""
    B, P, xt, y, (h, w, f, sh, psf) = detector
    from tests.golden.make_golden import DETECTOR_ITERS, OUT_DETECTOR, block_sums
    ref = json.load(open(OUT_DETECTOR))
    tr = {k: np.asarray(v) for k, v in ref["trace"].items()}
    plan = B.Plan(h, w, f, sh, psf, lam=0.01, iters=DETECTOR_ITERS)
    x, st = plan.solve(to_dev(y))
    tg = plan.trace()
    xg = x.cpu().numpy().astype(np.float64)
    plan.close()
    assert st["iters_done"] == DETECTOR_ITERS == len(tr["E"])
    assert st["J_final"] == pytest.approx(ref["J_final"], rel=RTOL_J)
    np.testing.assert_allclose(tg["E"], tr["E"], rtol=RTOL_J)
    sig = np.abs(tr["E"] - tr["J_trial"]) > 1e-6 * np.abs(tr["E"])
    assert sig.sum() >= 20
    assert np.array_equal(tg["accept"][sig], tr["accept"][sig])
    np.testing.assert_allclose(tg["alpha"][sig], tr["alpha"][sig], rtol=1e-3)
    assert abs(xg.sum() - ref["x_sum"]) <= RTOL_X * abs(ref["x_sum"])
    assert abs(np.linalg.norm(xg) - ref["x_norm"]) <= RTOL_X * ref["x_norm"]
    assert rel_l2(block_sums(xg), np.asarray(ref["block_sums"])) <= RTOL_X
    # the objective at the device's own image, evaluated by the oracle
    assert P.objective(xg, y.astype(np.float64)) == pytest.approx(ref["J_final"], rel=RTOL_J)


def test_detector_20_iterations_element_by_element(detector):
    """Twenty iterations (the paper's longest runtime column, Table 4) at 4096^2, the image
    compared pixel by pixel with a live oracle run."""
    B, P, xt, y, (h, w, f, sh, psf) = detector
    iters = 20
    plan = B.Plan(h, w, f, sh, psf, lam=0.01, iters=iters)
    x, st = plan.solve(to_dev(y))
    xg = x.cpu().numpy().astype(np.float64)
    plan.close()
    y64 = y.astype(np.float64)
    xr, _ = P.scg(y64, P.shift_add(y64), iters)
    assert rel_l2(xg, xr) <= RTOL_X
    assert np.max(np.abs(xg - xr)) <= 1e-2 * np.max(np.abs(xr))
    assert st["J_final"] == pytest.approx(P.objective(xr, y64), rel=RTOL_J)


@pytest.mark.parametrize("model", ["l1", "paper_ct", "subpixel"])
def test_full_size_model_options(orc, model):
    """The other lines bench.py times, at their full size (4 x 2048^2 -> 4096^2): the L1 data
    term (eps_d 0.01), the paper's CT setting (3x3 PSF, binning D, L1, lambda 0.05) and
    non-integer shifts (x 0.02 / 0.51, y 0.04 / 0.53 LR px, 3x3 PSF): the forward operator and
    the gradient over the whole image against the FP64 oracle."""
    from paper_2108_04315_b300 import binding as B
    h = w = 2048
    f = 2
    psf3 = gen.gaussian_psf(3, 0.5)
    if model == "l1":
        sh, psf, lam = gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5), 0.01
        kp, ko = dict(data_norm=B.MISR_NORM_L1, data_eps=0.01), dict(data_norm=orc.NORM_L1, data_eps=0.01)
    elif model == "paper_ct":
        sh, psf, lam = gen.half_pixel_shifts(), psf3, 0.05
        kp = dict(data_norm=B.MISR_NORM_L1, data_eps=0.01, decimation=B.MISR_DECIM_BIN)
        ko = dict(data_norm=orc.NORM_L1, data_eps=0.01, decimation=orc.DECIM_BIN)
    else:
        sh, psf, lam = [(dx, dy) for dy in (0.04, 0.53) for dx in (0.02, 0.51)], psf3, 0.01
        kp, ko = dict(tile_shape=B.MISR_TILE_32x32), {}
    P = orc.Problem(h, w, f, sh, psf, lam=lam, **ko)
    plan = B.Plan(h, w, f, sh, psf, lam=lam, iters=1, **kp)
    xt = gen.phantom(f * h, f * w, gen.CONFIG_SEEDS["detector"])
    yf = plan.forward(to_dev(xt.astype(np.float32)))
    assert rel_l2(yf.cpu().numpy(), P.forward_all(xt.astype(np.float32).astype(np.float64))) <= RTOL_OP
    y = (P.forward_all(xt) + gen.gaussian_noise((4, h, w), 0.01, gen.CONFIG_SEEDS["detector"] + 1)).astype(np.float32)
    x = (xt + 0.05 * gen.smooth_field(f * h, f * w, 72)).astype(np.float32)
    J, g = plan.gradient(to_dev(y), to_dev(x))
    Jr, gr = P.gradient(x.astype(np.float64), y.astype(np.float64))
    # the L1 bar of tests/test_gpu_l1.py where the L1 term is used
    tol = RTOL_OP + (16 * 2.0 ** -24 * float(np.abs(y).max()) / 0.01 if model != "subpixel" else 0.0)
    assert rel_l2(g.cpu().numpy(), gr) <= tol
    assert J == pytest.approx(Jr, rel=RTOL_J)
    plan.close()


def test_full_size_interpolation_is_the_oracle_bitwise(detector):
    """misr_interpolate at the full size, in the bench's configuration: the oracle's
    shift-and-add rounded to float32, bit for bit."""
    B, P, xt, y, (h, w, f, sh, psf) = detector
    plan = B.Plan(h, w, f, sh, psf, lam=0.01, iters=1)
    xi = plan.interpolate(to_dev(y)).cpu().numpy()
    assert np.array_equal(xi, P.shift_add(y.astype(np.float64)).astype(np.float32))
    plan.close()


def test_precision_size_gradient_against_oracle(orc):
    """The precision workload's size (4 x 3072^2 u16 counts -> 6144^2 HR) on the shape its plans
    get by default: the device's log conversion and the gradient over the whole image against
    the FP64 oracle's (its items split into four waves of edge items and one of interior)."""
    from paper_2108_04315_b300 import binding as B
    h = w = 3072
    f, sh, psf, i0 = 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5), 40000.0
    seed = gen.CONFIG_SEEDS["precision"]
    P = orc.Problem(h, w, f, sh, psf, lam=0.01)
    xt = gen.phantom(f * h, f * w, seed)
    counts = gen.poisson_counts(P.forward_all(xt), i0, seed + 1)
    y64 = orc.log_convert(counts, i0)
    plan = B.Plan(h, w, f, sh, psf, lam=0.01, iters=1, in_dtype=B.MISR_U16, flat_field=i0)
    x = (xt + 0.05 * gen.smooth_field(f * h, f * w, 73)).astype(np.float32)
    J, g = plan.gradient(to_dev(counts.view(np.int16)), to_dev(x))
    Jr, gr = P.gradient(x.astype(np.float64), y64)
    assert rel_l2(g.cpu().numpy(), gr) <= RTOL_OP
    assert J == pytest.approx(Jr, rel=RTOL_J)
    plan.close()


def test_study_frames_full_size(orc):
    """bench.py's synthetic_study_frames workload: 4 x 2048^2 frames with the one-pixel shifts
    right, down, left and up, 2x2 binning, 3x3 Gaussian PSF sigma 0.5, the L1 data term (eps_d
    0.01), lambda 0.05 (the frame-wise pass): every frame of the forward operator, the gradient
    and a 5-iteration solve against the oracle."""
    from paper_2108_04315_b300 import binding as B
    from tests.gpu_common import STUDY_SHIFTS
    h = w = 2048
    f, psf, eps_d = 2, gen.gaussian_psf(3, 0.5), 0.01
    kw_o = dict(lam=0.05, decimation=orc.DECIM_BIN, data_norm=orc.NORM_L1, data_eps=eps_d)
    P = orc.Problem(h, w, f, STUDY_SHIFTS, psf, **kw_o)
    xt = gen.phantom(f * h, f * w, gen.CONFIG_SEEDS["detector"])
    y = (P.forward_all(xt) + gen.gaussian_noise((4, h, w), 0.01, gen.CONFIG_SEEDS["detector"] + 1)).astype(np.float32)
    kw_p = dict(lam=0.05, decimation=B.MISR_DECIM_BIN, data_norm=B.MISR_NORM_L1, data_eps=eps_d)
    plan = B.Plan(h, w, f, STUDY_SHIFTS, psf, iters=5, **kw_p)
    yf = plan.forward(to_dev(xt.astype(np.float32))).cpu().numpy()
    ref = P.forward_all(xt.astype(np.float32).astype(np.float64))
    for k in range(4):
        assert rel_l2(yf[k], ref[k]) <= RTOL_OP, k
    x = (xt + 0.05 * gen.smooth_field(f * h, f * w, 71)).astype(np.float32)
    J, g = plan.gradient(to_dev(y), to_dev(x))
    Jr, gr = P.gradient(x.astype(np.float64), y.astype(np.float64))
    tol = RTOL_OP + 16 * 2.0 ** -24 * float(np.abs(y).max()) / eps_d
    assert rel_l2(g.cpu().numpy(), gr) <= tol
    assert J == pytest.approx(Jr, rel=RTOL_J)
    xs, st = plan.solve(to_dev(y))
    y64 = y.astype(np.float64)
    xr, _ = P.scg(y64, P.shift_add(y64), 5)
    assert st["iters_done"] == 5
    assert rel_l2(xs.cpu().numpy(), xr) <= RTOL_X
    assert st["J_final"] == pytest.approx(P.objective(xr, y64), rel=RTOL_J)
    plan.close()
