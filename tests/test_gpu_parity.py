"""CUDA library vs the FP64 oracle, through the C ABI, on the same seeded inputs.

Tolerances: operator applications and per-pass sums relative L2 <= 1e-5; the SR image after a
fixed iteration count relative L2 <= 1e-3 and the objective within 1e-5 relative.
"""
import numpy as np
import pytest

import gen
from tests.gpu_common import (OTHER_GEOMETRY_ITERS, OTHER_GEOMETRY_SEED, PARITY_CASES, RTOL_J, RTOL_OP, RTOL_X,
                              U16_ITERS, make_case, rel_l2, to_dev, u16_case)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = PARITY_CASES
# the plan's default shape (the 32 x 32 tiles on these sizes) and the row-streaming kernel
SHAPES = [0, 4]


@pytest.mark.parametrize("name", sorted(CASES))
def test_forward_operator(orc, name):
    """y_k = D B M_k x (Eq. 1) for every frame."""
    h, w, f, shifts, psf = CASES[name]
    P, plan, xt, _ = make_case(orc, h, w, f, shifts, psf, seed=100)
    x = (xt + gen.random_field(xt.shape, 7, -0.5, 0.5)).astype(np.float32)
    y = plan.forward(to_dev(x)).cpu().numpy()
    ref = P.forward_all(x.astype(np.float64))
    for k in range(len(shifts)):
        assert rel_l2(y[k], ref[k]) <= RTOL_OP, (name, k)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("name", sorted(CASES))
def test_objective_and_gradient(orc, name, shape):
    """J(x) (Eq. 9) and grad J(x) = 2 sum_k A_k^T (A_k x - y_k) + lambda grad BTV(x)."""
    h, w, f, shifts, psf = CASES[name]
    P, plan, xt, y = make_case(orc, h, w, f, shifts, psf, seed=200, tile_shape=shape)
    x = (xt + gen.random_field(xt.shape, 8, -0.2, 0.2)).astype(np.float32)
    J, g = plan.gradient(to_dev(y), to_dev(x))
    Jr, gr = P.gradient(x.astype(np.float64), y.astype(np.float64))
    assert J == pytest.approx(Jr, rel=RTOL_J)
    assert rel_l2(g.cpu().numpy(), gr) <= RTOL_OP


@pytest.mark.parametrize("name", ["tiny_f2", "ragged_f2_asym", "ragged_f3_k9", "partial_f2_k3", "f1_denoise",
                                  "thin_strip"])
@pytest.mark.parametrize("alpha,beta", [(0.3, 0.7), (0.0, 0.0), (1.7, 0.05)])
@pytest.mark.parametrize("shape", SHAPES)
def test_fused_pass(orc, name, alpha, beta, shape):
    """One fused SCG pass: p = r + beta p_old, x' = x + alpha p, r' = -grad J(x'), and its sums:
    J_data(x'), J_data(x') - J_data(x), BTV(x'), |r'|^2, r'.r, p.r', |p|^2 and the curvature
    forms r'.H(x')r', r'.H(x')p, p.H(x')p with the exact Hessian H of J."""
    h, w, f, shifts, psf = CASES[name]
    P, plan, xt, y = make_case(orc, h, w, f, shifts, psf, seed=300, tile_shape=shape)
    P0 = orc.Problem(h, w, f, shifts, psf, lam=0.0)
    x = (xt + gen.random_field(xt.shape, 9, -0.1, 0.1)).astype(np.float32)
    r = gen.random_field(xt.shape, 10, -0.3, 0.3).astype(np.float32)
    po = gen.random_field(xt.shape, 11, -0.3, 0.3).astype(np.float32)
    xo, ro, pn, S = plan.pass_probe(to_dev(y), to_dev(x), to_dev(r), to_dev(po), alpha, beta)
    xo, ro, pn = (t.cpu().numpy().astype(np.float64) for t in (xo, ro, pn))
    x64, r64, po64, y64 = (a.astype(np.float64) for a in (x, r, po, y))
    p_ref = r64 + beta * po64
    assert rel_l2(pn, p_ref) <= 1e-6
    assert rel_l2(xo, x64 + alpha * pn) <= 1e-6
    # everything downstream is checked at the pass's own x' and p
    J, g = P.gradient(xo, y64)
    r_ref = -g
    assert rel_l2(ro, r_ref) <= RTOL_OP
    ref = {
        "J_data": P0.objective(xo, y64),
        "dJ_data": P0.objective(x64 + alpha * pn, y64) - P0.objective(x64, y64),
        "R_btv": P.reg_value(xo),
        "rr": float(np.sum(r_ref * r_ref)),
        "rr_cross": float(np.sum(r_ref * r64)),
        "pr": float(np.sum(pn * r_ref)),
        "pp": float(np.sum(pn * pn)),
        "a": P.curvature(xo, r_ref),
        "b": float(np.sum(r_ref * P.hessvec(xo, pn))),
        "c": P.curvature(xo, pn),
    }
    scale = {"dJ_data": abs(ref["J_data"]) * 1e-7, "b": np.sqrt(abs(ref["a"] * ref["c"])) * 1e-6,
             "rr_cross": np.sqrt(ref["rr"] * np.sum(r64 * r64)) * 1e-6, "pr": np.sqrt(ref["rr"] * ref["pp"]) * 1e-6}
    for k, v in ref.items():
        assert abs(S[k] - v) <= RTOL_OP * abs(v) + scale.get(k, 0.0) + 1e-30, (k, S[k], v)


def _check_decisions(tg, tr):
    """Accept decisions must agree wherever the objective change is above the FP32 noise
    floor of the device's prior sum; below it (converged runs) a few may differ."""
    sig = np.abs(tr["E"] - tr["J_trial"]) > 1e-6 * np.abs(tr["E"])
    assert np.array_equal(tg["accept"][sig], tr["accept"][sig])
    assert int(np.sum(tg["accept"] != tr["accept"])) <= max(2, (~sig).sum() // 4)


def _compare_solve(P, plan, y, iters, x0=None):
    y64 = y.astype(np.float64)
    yd = to_dev(y)
    if x0 is None:
        x0 = P.shift_add(y64)
        xg, st = plan.solve(yd)
    else:
        xg = to_dev(x0.astype(np.float32))
        xg, st = plan.solve(yd, x_out=xg)
        x0 = x0.astype(np.float32).astype(np.float64)
    xr, tr = P.scg(y64, x0, iters)
    xg = xg.cpu().numpy()
    tg = plan.trace()
    return xg, st, tg, xr, tr


@pytest.mark.parametrize("shape", SHAPES)
def test_solve_tiny_workload(orc, shape):
    """4 x 64^2 frames -> 128^2, half-pixel shifts, 5x5 Gaussian sigma 0.5, lambda 0.01,
    50 SCG iterations from multi-image interpolation: image, objective and accept trace."""
    h, w, f, shifts, psf = CASES["tiny_f2"]
    P, plan, xt, y = make_case(orc, h, w, f, shifts, psf, seed=gen.CONFIG_SEEDS["tiny"], iters=50, tile_shape=shape)
    xg, st, tg, xr, tr = _compare_solve(P, plan, y, 50)
    assert st["iters_done"] == 50
    assert rel_l2(xg, xr) <= RTOL_X
    assert st["J_final"] == pytest.approx(P.objective(xr, y.astype(np.float64)), rel=RTOL_J)
    assert st["J_final"] == pytest.approx(P.objective(xg.astype(np.float64), y.astype(np.float64)), rel=RTOL_J)
    # Moller's comparison parameter Delta = 2 delta (E - J') / mu^2 is computed on the device
    # from FP32 per-pixel terms summed in FP64: the data part as a per-pixel difference, the
    # prior part as two direct sums whose FP32 noise is ~1e-9 of J on this problem.  Where
    # E - J' is above 1e-6 J the decisions (accept, lambda schedule) must agree with the FP64
    # oracle; below it Delta is noise-limited and a decision may differ without moving the
    # image (checked above).
    sig = np.abs(tr["E"] - tr["J_trial"]) > 1e-6 * np.abs(tr["E"])
    assert sig.sum() >= 10
    assert np.array_equal(tg["accept"][sig], tr["accept"][sig])
    np.testing.assert_allclose(tg["Delta"][sig], tr["Delta"][sig], rtol=1e-2, atol=1e-3)
    np.testing.assert_allclose(tg["E"], tr["E"], rtol=RTOL_J)
    np.testing.assert_allclose(tg["alpha"][sig], tr["alpha"][sig], rtol=1e-3)
    first_floor = int(np.argmin(sig)) if not sig.all() else len(sig)
    floor = 1e-9 * np.median(tr["delta"] / tr["pn2"])
    np.testing.assert_allclose(tg["lam"][:first_floor], tr["lam"][:first_floor], rtol=1e-3, atol=floor)
    flips = int(np.sum(tg["accept"] != tr["accept"]))
    assert flips <= max(2, (~sig).sum() // 4), flips


# Iteration counts stay where storing the SCG state (x, r, p) in FP32 moves the FP64 run by
# far less than the parity bars (tests/test_fp32_sensitivity.py, oracle only).  With one HR
# phase unsampled (partial_f2_k3) the near-L1 prior leaves the problem ill-conditioned: there,
# rounding x, r and p to FP32 after every step of the FP64 algorithm moves the objective by
# ~1e-7 after 6 iterations but by ~2e-4 after 10, for any FP32-state implementation.
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("name,iters", sorted(OTHER_GEOMETRY_ITERS.items()))
def test_solve_other_geometries(orc, name, iters, shape):
    h, w, f, shifts, psf = CASES[name]
    P, plan, xt, y = make_case(orc, h, w, f, shifts, psf, seed=OTHER_GEOMETRY_SEED, iters=iters, tile_shape=shape)
    xg, st, tg, xr, tr = _compare_solve(P, plan, y, iters)
    y64 = y.astype(np.float64)
    assert rel_l2(xg, xr) <= RTOL_X
    # the device's objective at its own image, to the accuracy of its FP32 terms
    assert st["J_final"] == pytest.approx(P.objective(xg.astype(np.float64), y64), rel=1e-6)
    assert st["J_final"] == pytest.approx(P.objective(xr, y64), rel=RTOL_J)
    _check_decisions(tg, tr)


@pytest.mark.parametrize("mode", ["zero", "given"])
def test_solve_start_modes(orc, mode):
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts, psf = CASES["ragged_f2_asym"]
    x0_mode = B.MISR_X0_ZERO if mode == "zero" else B.MISR_X0_GIVEN
    P, plan, xt, y = make_case(orc, h, w, f, shifts, psf, seed=500, iters=20, x0_mode=x0_mode)
    x0 = np.zeros_like(xt) if mode == "zero" else xt + gen.random_field(xt.shape, 12, -0.3, 0.3)
    xg, st, tg, xr, tr = _compare_solve(P, plan, y, 20, x0=x0)
    assert rel_l2(xg, xr) <= RTOL_X
    _check_decisions(tg, tr)


def test_uint16_counts_log_converted_on_device(orc):
    """uint16 detector counts c, y = ln I0 - ln max(c, 1) on the device (Sec. 4 inputs are
    16-bit projections), then the solve; compared with the oracle on the oracle's own
    log conversion of the same counts."""
    from paper_2108_04315_b300 import binding as B
    P, counts, y64 = u16_case(orc)
    h, w, f = P.h, P.w, P.f
    shifts, psf = gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)
    # 10 iterations: the 12th step of this problem lowers J by 2.6e-10 of J, below the FP32
    # evaluation floor of the objective (~1e-9 J), and by 20 iterations FP32 storage of the
    # state alone moves the FP64 objective by ~2e-4 (tests/test_fp32_sensitivity.py)
    iters = U16_ITERS
    plan = B.Plan(h, w, f, shifts, psf, lam=0.01, iters=iters, in_dtype=B.MISR_U16, flat_field=40000.0)
    xg, st = plan.solve(to_dev(counts.view(np.int16)))
    xr, tr = P.scg(y64, P.shift_add(y64), iters)
    _check_decisions(plan.trace(), tr)
    assert rel_l2(xg.cpu().numpy(), xr) <= RTOL_X
    assert st["J_final"] == pytest.approx(P.objective(xr, y64), rel=RTOL_J)


def test_solve_is_deterministic_and_plan_reusable(orc):
    h, w, f, shifts, psf = CASES["ragged_f3_k9"]
    P, plan, xt, y = make_case(orc, h, w, f, shifts, psf, seed=700, iters=12)
    yd = to_dev(y)
    a, sa = plan.solve(yd)
    b, sb = plan.solve(yd)
    assert torch.equal(a, b) and sa == sb
    y2 = (y + gen.gaussian_noise(y.shape, 0.01, 701)).astype(np.float32)
    c, _ = plan.solve(to_dev(y2))
    xr, _ = P.scg(y2.astype(np.float64), P.shift_add(y2.astype(np.float64)), 12)
    assert rel_l2(c.cpu().numpy(), xr) <= RTOL_X


def test_solve_host_buffers(orc):
    """misr_solve_host: host frames in, host image out, same result as the device call."""
    h, w, f, shifts, psf = CASES["tiny_f2"]
    P, plan, xt, y = make_case(orc, h, w, f, shifts, psf, seed=800, iters=10)
    xd, _ = plan.solve(to_dev(y))
    xh = np.zeros((f * h, f * w), dtype=np.float32)
    st = plan.solve_host(np.ascontiguousarray(y), xh)
    assert st["iters_done"] == 10
    np.testing.assert_array_equal(xh, xd.cpu().numpy())


def test_zero_iterations_returns_start_point(orc):
    h, w, f, shifts, psf = CASES["tiny_f2"]
    P, plan, xt, y = make_case(orc, h, w, f, shifts, psf, seed=900, iters=0)
    xg, st = plan.solve(to_dev(y))
    assert st["iters_done"] == 0
    np.testing.assert_array_equal(xg.cpu().numpy(), P.shift_add(y.astype(np.float64)).astype(np.float32))
    assert st["J_final"] == pytest.approx(P.objective(P.shift_add(y.astype(np.float64)), y.astype(np.float64)),
                                          rel=RTOL_J)
