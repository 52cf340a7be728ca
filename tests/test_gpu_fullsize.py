"""The detector workload at full size (4 x 2048^2 frames -> 4096^2 HR) in the launch
configuration bench.py times (its tile shape tuned first): the forward operator and the
gradient over the whole image, and a short solve, against the FP64 oracle."""
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
