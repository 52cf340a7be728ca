"""The prior's options through the C ABI against the FP64 oracle: lambda 0 (the data term
alone), BTV windows w = 1 (no offsets), 2 and 3, decay alpha from 0.4 to 1, and the
smoothing eps from 1e-3 to 0.1 (Eq. 8, 9).  Gradient, the fused pass's sums and a short solve,
with the bars of tests/test_gpu_parity.py."""
import numpy as np
import pytest

import gen
from tests.gpu_common import RTOL_J, RTOL_OP, RTOL_X, asym_separable_psf, rel_l2, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

OPTIONS = [
    # (lambda, btv_w, btv_alpha, eps)
    (0.0, 3, 0.4, 1e-3),
    (0.01, 1, 0.4, 1e-3),
    (0.01, 2, 0.7, 1e-3),
    (0.05, 3, 1.0, 0.1),
    (1.0, 3, 0.4, 1e-2),
]


def case(orc, opt, seed, iters=10, shape=0):
    """shape: a MISR_TILE_* shape, or "frame" for the synthetic study's frame set with binning
    (the frame-wise pass, whose prior kernels are its own)"""
    from paper_2108_04315_b300 import binding as B
    from tests.gpu_common import STUDY_SHIFTS
    lam, w_, a_, eps = opt
    h, w, f, shifts, psf = 37, 53, 2, gen.half_pixel_shifts(), asym_separable_psf(3)
    kw_o, kw_p = {}, {"tile_shape": shape}
    if shape == "frame":
        shifts, psf = STUDY_SHIFTS, asym_separable_psf(3, 3)
        kw_o, kw_p = {"decimation": orc.DECIM_BIN}, {"decimation": B.MISR_DECIM_BIN}
    P = orc.Problem(h, w, f, shifts, psf, lam=lam, btv_alpha=a_, btv_w=w_, eps=eps, **kw_o)
    xt = gen.phantom(f * h, f * w, seed)
    y = (P.forward_all(xt) + gen.gaussian_noise((4, h, w), 0.01, seed + 1)).astype(np.float32)
    plan = B.Plan(h, w, f, shifts, psf, lam=lam, btv_alpha=a_, btv_w=w_, eps=eps, iters=iters, **kw_p)
    return P, plan, xt, y


@pytest.mark.parametrize("shape", [0, 4, "frame"])   # the size default (tiles), MISR_TILE_STREAM, frame-wise
@pytest.mark.parametrize("opt", OPTIONS, ids=[f"lam{o[0]}_w{o[1]}_a{o[2]}_eps{o[3]}" for o in OPTIONS])
def test_prior_options_gradient_and_pass(orc, opt, shape):
    P, plan, xt, y = case(orc, opt, 100, shape=shape)
    x = (xt + gen.random_field(xt.shape, 9, -0.1, 0.1)).astype(np.float32)
    J, g = plan.gradient(to_dev(y), to_dev(x))
    Jr, gr = P.gradient(x.astype(np.float64), y.astype(np.float64))
    assert J == pytest.approx(Jr, rel=RTOL_J)
    assert rel_l2(g.cpu().numpy(), gr) <= RTOL_OP
    r = gen.random_field(xt.shape, 10, -0.3, 0.3).astype(np.float32)
    po = gen.random_field(xt.shape, 11, -0.3, 0.3).astype(np.float32)
    alpha, beta = 0.3, 0.7
    xo, ro, pn, S = plan.pass_probe(to_dev(y), to_dev(x), to_dev(r), to_dev(po), alpha, beta)
    xo, pn = xo.cpu().numpy().astype(np.float64), pn.cpu().numpy().astype(np.float64)
    _, g2 = P.gradient(xo, y.astype(np.float64))
    ref = {"R_btv": P.reg_value(xo), "a": P.curvature(xo, -g2), "c": P.curvature(xo, pn),
           "b": float(np.sum(-g2 * P.hessvec(xo, pn)))}
    for k, v in ref.items():
        slack = np.sqrt(abs(ref["a"] * ref["c"])) * 1e-6 if k == "b" else 1e-30
        assert abs(S[k] - v) <= RTOL_OP * abs(v) + slack, (k, S[k], v)


@pytest.mark.parametrize("shape", [0, 4, "frame"])
@pytest.mark.parametrize("opt", OPTIONS, ids=[f"lam{o[0]}_w{o[1]}_a{o[2]}_eps{o[3]}" for o in OPTIONS])
def test_prior_options_solve(orc, opt, shape):
    iters = 7 if shape == "frame" else 10   # the study's frames: the FP32-state floor of the L2 term
    P, plan, xt, y = case(orc, opt, 200, iters=iters, shape=shape)
    y64 = y.astype(np.float64)
    xg, st = plan.solve(to_dev(y))
    xr, tr = P.scg(y64, P.shift_add(y64), iters)
    assert rel_l2(xg.cpu().numpy(), xr) <= RTOL_X
    assert st["J_final"] == pytest.approx(P.objective(xr, y64), rel=1e-4)
