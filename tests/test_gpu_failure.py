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


@pytest.mark.parametrize("variant", ["l1", "subpixel", "subpixel_l1_bf16", "binned_l1"])
def test_late_tile_load_in_the_other_kernel_variants(orc, variant):
    """The same failure path in the L1, per-phase-tap and binning variants of the pass."""
    from paper_2108_04315_b300 import binding as B
    psf3 = gen.gaussian_psf(3, 0.6)
    frac = [(dx, dy) for dy in (0.05, 0.6) for dx in (0.0, 0.55)]
    kw = {
        "l1": (gen.half_pixel_shifts(), PSF, dict(data_norm=B.MISR_NORM_L1, data_eps=0.02)),
        "subpixel": (frac, psf3, dict()),
        "subpixel_l1_bf16": (frac, psf3, dict(data_norm=B.MISR_NORM_L1, data_eps=0.05, iterate_dtype=B.MISR_BF16)),
        "binned_l1": (gen.half_pixel_shifts(), psf3, dict(data_norm=B.MISR_NORM_L1, data_eps=0.02,
                                                          decimation=B.MISR_DECIM_BIN)),
    }[variant]
    shifts, psf, opts = kw
    plan = B.Plan(37, 53, 2, shifts, psf, lam=0.01, iters=6, **opts)
    yd = to_dev(gen.random_field((4, 37, 53), 4200, 0.0, 2.0).astype(np.float32))
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
