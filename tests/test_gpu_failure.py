"""Failure path of the fused pass without a GPU fault: with the tile-load wait limit at 0 every
load is reported late, the projection is flagged and its solve returns MISR_ETIMEOUT, the copies
in flight are drained, and the context stays usable (the default limit then gives the healthy
result again, bit for bit)."""
import numpy as np
import pytest

import gen
from tests.gpu_common import make_case, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PSF = gen.gaussian_psf(5, 0.5)


@pytest.mark.parametrize("tile_shape", [1, 2, 3])
@pytest.mark.parametrize("iterate", ["f32", "bf16"])
def test_late_tile_load_is_reported_and_context_survives(orc, tile_shape, iterate):
    from paper_2108_04315_b300 import binding as B
    dt = B.MISR_BF16 if iterate == "bf16" else B.MISR_F32
    P, plan, xt, y = make_case(orc, 37, 53, 2, gen.half_pixel_shifts(), PSF, seed=4000, iters=6,
                               tile_shape=tile_shape, iterate_dtype=dt)
    yd = to_dev(y)
    x_ok, st_ok = plan.solve(yd)
    x_ok = x_ok.clone()
    B.misr_plan_set_wait_limit(plan.handle, 0)
    with pytest.raises(B.MisrError) as e:
        plan.solve(yd)
    assert e.value.status == B.MISR_ETIMEOUT
    B.misr_plan_set_wait_limit(plan.handle, B.TMA_WAIT_TRIES_DEFAULT)
    x2, st2 = plan.solve(yd)
    assert torch.equal(x2, x_ok) and st2 == st_ok
    torch.cuda.synchronize()


def test_late_tile_load_in_a_probe_pass(orc):
    from paper_2108_04315_b300 import binding as B
    P, plan, xt, y = make_case(orc, 30, 41, 2, gen.half_pixel_shifts(), PSF, seed=4100, iters=3)
    yd = to_dev(y)
    g = torch.Generator("cuda").manual_seed(7)
    x = torch.rand((plan.H, plan.W), device="cuda", generator=g)
    r = torch.randn((plan.H, plan.W), device="cuda", generator=g)
    p = torch.randn((plan.H, plan.W), device="cuda", generator=g)
    ref = plan.pass_probe(yd, x, r, p, 0.5, 0.3)
    B.misr_plan_set_wait_limit(plan.handle, 0)
    with pytest.raises(B.MisrError) as e:
        plan.pass_probe(yd, x, r, p, 0.5, 0.3)
    assert e.value.status == B.MISR_ETIMEOUT
    B.misr_plan_set_wait_limit(plan.handle, B.TMA_WAIT_TRIES_DEFAULT)
    again = plan.pass_probe(yd, x, r, p, 0.5, 0.3)
    for a, b in zip(ref[:3], again[:3]):
        assert torch.equal(a, b)
    assert np.array_equal(np.asarray(ref[3]), np.asarray(again[3]))
