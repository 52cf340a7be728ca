"""Binning decimation (misr_desc.decimation = MISR_DECIM_BIN): each LR pixel the mean of its
f x f block of B M_k x, as in the synthetic study (Sec. 4.1.1).  The library folds D_bin B
into one blur with psf_size + f - 1 taps per axis; the FP64 oracle applies the block mean
literally, so the two share no arithmetic.  Same bars as the point-sampled path (and the L1
bars of tests/test_gpu_l1.py where the L1 term is used)."""
import numpy as np
import pytest

import gen
from tests.gpu_common import RTOL_J, RTOL_OP, RTOL_X, asym_separable_psf, rel_l2, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U = 2.0 ** -24
CASES = {
    # name: (h, w, f, shifts, psf) -- taps psf_size + f - 1 <= 5
    "ct_f2_psf3": (40, 52, 2, gen.half_pixel_shifts(), gen.gaussian_psf(3, 0.6)),
    "f2_asym3_partial": (30, 41, 2, [(0.0, 0.0), (0.5, 0.0), (0.5, 0.5)], asym_separable_psf(4, 3)),
    "f2_delta": (33, 27, 2, gen.half_pixel_shifts(), np.ones((1, 1))),
    "f3_delta_k9": (21, 25, 3, gen.third_pixel_shifts(), np.ones((1, 1))),
    "f1_psf5": (45, 70, 1, [(0.0, 0.0)], gen.gaussian_psf(5, 0.6)),
    "thin_strip": (1, 61, 2, gen.half_pixel_shifts(), gen.gaussian_psf(3, 0.6)),
}


def binned_case(orc, name, seed, iters=20, lam=0.01, l1_eps=None, **plan_kw):
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts, psf = CASES[name]
    kw_o = dict(data_norm=orc.NORM_L1, data_eps=l1_eps) if l1_eps else {}
    kw_p = dict(data_norm=B.MISR_NORM_L1, data_eps=l1_eps) if l1_eps else {}
    P = orc.Problem(h, w, f, shifts, psf, lam=lam, decimation=orc.DECIM_BIN, **kw_o)
    xt = gen.phantom(f * h, f * w, seed)
    y = P.forward_all(xt) + gen.gaussian_noise((len(shifts), h, w), 0.01, seed + 1)
    plan = B.Plan(h, w, f, shifts, psf, lam=lam, iters=iters, decimation=B.MISR_DECIM_BIN, **kw_p, **plan_kw)
    return P, plan, xt, y.astype(np.float32)


@pytest.mark.parametrize("name", sorted(CASES))
def test_binned_forward_operator(orc, name):
    P, plan, xt, _ = binned_case(orc, name, 100)
    x = (xt + gen.random_field(xt.shape, 7, -0.5, 0.5)).astype(np.float32)
    y = plan.forward(to_dev(x)).cpu().numpy()
    ref = P.forward_all(x.astype(np.float64))
    for k in range(P.K):
        assert rel_l2(y[k], ref[k]) <= RTOL_OP, (name, k)


@pytest.mark.parametrize("name", sorted(CASES))
def test_binned_objective_and_gradient(orc, name):
    P, plan, xt, y = binned_case(orc, name, 200)
    x = (xt + gen.random_field(xt.shape, 8, -0.2, 0.2)).astype(np.float32)
    J, g = plan.gradient(to_dev(y), to_dev(x))
    Jr, gr = P.gradient(x.astype(np.float64), y.astype(np.float64))
    assert J == pytest.approx(Jr, rel=RTOL_J)
    assert rel_l2(g.cpu().numpy(), gr) <= RTOL_OP


@pytest.mark.parametrize("name", ["ct_f2_psf3", "f3_delta_k9", "f2_asym3_partial"])
@pytest.mark.parametrize("l1_eps", [None, 0.05])
@pytest.mark.parametrize("shape", [0, 4])   # the size default (tiles) and MISR_TILE_STREAM
def test_binned_fused_pass(orc, name, l1_eps, shape):
    """One fused pass with binning: r' and the ten sums, curvature forms included."""
    alpha, beta = 0.3, 0.7
    P, plan, xt, y = binned_case(orc, name, 300, l1_eps=l1_eps, tile_shape=shape)
    x = (xt + gen.random_field(xt.shape, 9, -0.1, 0.1)).astype(np.float32)
    r = gen.random_field(xt.shape, 10, -0.3, 0.3).astype(np.float32)
    po = gen.random_field(xt.shape, 11, -0.3, 0.3).astype(np.float32)
    xo, ro, pn, S = plan.pass_probe(to_dev(y), to_dev(x), to_dev(r), to_dev(po), alpha, beta)
    xo, ro, pn = (t.cpu().numpy().astype(np.float64) for t in (xo, ro, pn))
    x64, r64, y64 = (a.astype(np.float64) for a in (x, r, y))
    h, w, f, shifts, psf = CASES[name]
    kw = dict(data_norm=orc.NORM_L1, data_eps=l1_eps) if l1_eps else {}
    P0 = orc.Problem(h, w, f, shifts, psf, lam=0.0, decimation=orc.DECIM_BIN, **kw)
    tol = RTOL_OP + (16 * U * float(np.abs(y).max()) / l1_eps if l1_eps else 0.0)
    J, g = P.gradient(xo, y64)
    r_ref = -g
    assert rel_l2(ro, r_ref) <= tol
    ref = {
        "J_data": P0.objective(xo, y64),
        "dJ_data": P0.objective(x64 + alpha * pn, y64) - P0.objective(x64, y64),
        "R_btv": P.reg_value(xo),
        "rr": float(np.sum(r_ref * r_ref)),
        "pr": float(np.sum(pn * r_ref)),
        "pp": float(np.sum(pn * pn)),
        "a": P.curvature(xo, r_ref, y64),
        "b": float(np.sum(r_ref * P.hessvec(xo, pn, y64))),
        "c": P.curvature(xo, pn, y64),
    }
    scale = {"dJ_data": abs(ref["J_data"]) * 1e-7, "b": np.sqrt(abs(ref["a"] * ref["c"])) * tol,
             "pr": np.sqrt(ref["rr"] * ref["pp"]) * tol}
    for k, v in ref.items():
        rt = 2 * tol if k in ("rr", "pr", "a", "b", "c") else RTOL_OP
        assert abs(S[k] - v) <= rt * abs(v) + scale.get(k, 0.0) + 1e-30, (k, S[k], v)


@pytest.mark.parametrize("name,iters", [("ct_f2_psf3", 20), ("f3_delta_k9", 12), ("f2_delta", 15)])
@pytest.mark.parametrize("shape", [0, 4])
def test_binned_solve_matches_oracle(orc, name, iters, shape):
    P, plan, xt, y = binned_case(orc, name, 400, iters=iters, tile_shape=shape)
    y64 = y.astype(np.float64)
    xg, st = plan.solve(to_dev(y))
    xr, tr = P.scg(y64, P.shift_add(y64), iters)
    assert rel_l2(xg.cpu().numpy(), xr) <= RTOL_X
    assert st["J_final"] == pytest.approx(P.objective(xr, y64), rel=1e-4)
    tg = plan.trace()
    sig = np.abs(tr["E"] - tr["J_trial"]) > 1e-6 * np.abs(tr["E"])
    assert np.array_equal(tg["accept"][sig], tr["accept"][sig])


def test_paper_ct_setting_matches_oracle(orc):
    """The paper's CT reconstruction setting (Sec. 4): 2x with half-pixel detector shifts, a
    3x3 Gaussian blur, lambda 0.05, alpha 0.4, 20 SCG iterations and the L1 data term, here with
    the binning D of the synthetic study, against the oracle."""
    P, plan, xt, y = binned_case(orc, "ct_f2_psf3", 500, iters=20, lam=0.05, l1_eps=0.01)
    y64 = y.astype(np.float64)
    xg, st = plan.solve(to_dev(y))
    xr, tr = P.scg(y64, P.shift_add(y64), 20)
    assert st["iters_done"] == 20
    assert rel_l2(xg.cpu().numpy(), xr) <= RTOL_X
    assert st["J_final"] == pytest.approx(P.objective(xr, y64), rel=1e-4)


def test_binned_and_point_in_one_batch_equal_each_alone(orc):
    from paper_2108_04315_b300 import binding as B
    from tests.gpu_common import make_case
    cases = [binned_case(orc, "ct_f2_psf3", 600, iters=8),
             make_case(orc, 40, 52, 2, gen.half_pixel_shifts(), gen.gaussian_psf(3, 0.6), seed=601, iters=9),
             binned_case(orc, "f3_delta_k9", 602, iters=7, l1_eps=0.05)]
    plans = [c[1] for c in cases]
    ys = [to_dev(c[3]) for c in cases]
    alone = [tuple(v.clone() if i == 0 else v for i, v in enumerate(p.solve(y))) for p, y in zip(plans, ys)]
    batch = B.Batch(plans)
    xs, stats = batch.solve(ys)
    for (xa, sa), xb, sb in zip(alone, xs, stats):
        assert torch.equal(xa, xb) and sa == sb
    batch.close()
