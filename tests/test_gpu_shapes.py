"""Shapes of the fused pass (three tile shapes and the row-streaming kernel) and their
autotuner.  Every compiled shape must give the oracle's gradient and solve (the tiling changes
only the order of the pass's sums); a batch mixing shapes must give each projection its own
solve bit for bit; misr_autotune must time every shape and make the fastest the default of
later plans of that HR size."""
import numpy as np
import pytest

import gen
from tests.gpu_common import RTOL_OP, RTOL_X, asym_separable_psf, rel_l2, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = (1, 2, 3, 4)   # MISR_TILE_32x64, MISR_TILE_32x32, MISR_TILE_16x64, MISR_TILE_STREAM


@pytest.mark.parametrize("shape", SHAPES)
def test_every_shape_matches_the_oracle(orc, shape):
    from paper_2108_04315_b300 import binding as B
    h, w, f = 45, 71, 3
    sh, psf = gen.third_pixel_shifts(), asym_separable_psf(31)
    P = orc.Problem(h, w, f, sh, psf, lam=0.01)
    xt = gen.phantom(f * h, f * w, 32)
    y = (P.forward_all(xt) + gen.gaussian_noise((len(sh), h, w), 0.01, 33)).astype(np.float32)
    y64 = y.astype(np.float64)
    plan = B.Plan(h, w, f, sh, psf, lam=0.01, iters=12, tile_shape=shape)
    x = gen.smooth_field(f * h, f * w, 34).astype(np.float32)
    J, g = plan.gradient(to_dev(y), to_dev(x))
    Jr, gr = P.gradient(x.astype(np.float64), y64)
    assert rel_l2(g.cpu().numpy(), gr) <= RTOL_OP
    assert J == pytest.approx(Jr, rel=RTOL_OP)
    xs, st = plan.solve(to_dev(y))
    xr, _ = P.scg(y64, P.shift_add(y64), 12)
    assert rel_l2(xs.cpu().numpy(), xr) <= RTOL_X
    plan.close()


def test_batch_mixing_shapes_equals_each_alone(orc):
    from paper_2108_04315_b300 import binding as B
    psf = gen.gaussian_psf(5, 0.5)
    plans, ys = [], []
    for i, shape in enumerate((1, 2, 3, 4, 2, 4)):
        h, w = 30 + 6 * i, 50 - 4 * i
        P = orc.Problem(h, w, 2, gen.half_pixel_shifts(), psf, lam=0.01)
        y = (P.forward_all(gen.phantom(2 * h, 2 * w, 40 + i)) + gen.gaussian_noise((4, h, w), 0.01, 50 + i))
        plans.append(B.Plan(h, w, 2, gen.half_pixel_shifts(), psf, lam=0.01, iters=10, tile_shape=shape))
        ys.append(to_dev(y.astype(np.float32)))
    alone = [p.solve(y)[0].clone() for p, y in zip(plans, ys)]
    batch = B.Batch(plans)
    xs, _ = batch.solve(ys)
    for a, b in zip(alone, xs):
        assert torch.equal(a, b)
    batch.close()


def test_autotune_picks_a_shape_that_later_plans_use(orc):
    from paper_2108_04315_b300 import binding as B
    h, w, f = 96, 128, 2
    sh, psf = gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)
    shape, ms = B.misr_autotune(B.make_desc(h, w, f, sh, psf, iters=1), passes=5)
    assert shape in SHAPES
    assert np.all(ms > 0) and ms[shape - 1] == ms.min()
    P = orc.Problem(h, w, f, sh, psf, lam=0.01)
    y = to_dev((P.forward_all(gen.phantom(f * h, f * w, 60)) + gen.gaussian_noise((4, h, w), 0.01, 61))
               .astype(np.float32))
    auto = B.Plan(h, w, f, sh, psf, lam=0.01, iters=8)
    explicit = B.Plan(h, w, f, sh, psf, lam=0.01, iters=8, tile_shape=shape)
    assert torch.equal(auto.solve(y)[0], explicit.solve(y)[0])
    with pytest.raises(B.MisrError) as e:
        B.misr_autotune(B.make_desc(h, w, f, sh, psf), passes=0)
    assert e.value.status == B.MISR_EINVAL


# Geometries of the streaming shape's item split: one strip (no interior items), images no
# taller than one edge item (the top items hold every row), a row more than that, a tall thin
# image whose left strip takes several waves of edge items, and a wide short one.
STREAM_GEOMETRIES = {
    "one_strip": (40, 50, 2),       # HR 80 x 100
    "short": (10, 150, 2),          # HR 20 x 300
    "edge_plus_one": (25, 120, 1),  # HR 25 x 120
    "tall_thin": (700, 64, 2),      # HR 1400 x 128
    "wide_short": (20, 900, 2),     # HR 40 x 1800
}


@pytest.mark.parametrize("name", sorted(STREAM_GEOMETRIES))
def test_streaming_item_split_matches_the_oracle(orc, name):
    from paper_2108_04315_b300 import binding as B
    h, w, f = STREAM_GEOMETRIES[name]
    sh = gen.half_pixel_shifts() if f == 2 else [(0.0, 0.0)]
    psf = gen.gaussian_psf(5, 0.5)
    P = orc.Problem(h, w, f, sh, psf, lam=0.01)
    xt = gen.phantom(f * h, f * w, 70)
    y = (P.forward_all(xt) + gen.gaussian_noise((len(sh), h, w), 0.01, 71)).astype(np.float32)
    x = gen.smooth_field(f * h, f * w, 72).astype(np.float32)
    plan = B.Plan(h, w, f, sh, psf, lam=0.01, iters=6, tile_shape=4)
    J, g = plan.gradient(to_dev(y), to_dev(x))
    Jr, gr = P.gradient(x.astype(np.float64), y.astype(np.float64))
    assert rel_l2(g.cpu().numpy(), gr) <= RTOL_OP
    assert J == pytest.approx(Jr, rel=RTOL_OP)
    # the pass's ten sums equal those of the 32 x 32 tile shape (same arithmetic, other order)
    tile = B.Plan(h, w, f, sh, psf, lam=0.01, iters=6, tile_shape=2)
    r = gen.random_field(xt.shape, 73, -0.3, 0.3).astype(np.float32)
    po = gen.random_field(xt.shape, 74, -0.3, 0.3).astype(np.float32)
    sums = [p.pass_probe(to_dev(y), to_dev(x), to_dev(r), to_dev(po), 0.3, 0.7)[3] for p in (plan, tile)]
    for k in sums[1]:
        assert sums[0][k] == pytest.approx(sums[1][k], rel=1e-5, abs=1e-6 * abs(sums[1]["J_data"]) + 1e-12), k
    xs, st = plan.solve(to_dev(y))
    xr, _ = P.scg(y.astype(np.float64), P.shift_add(y.astype(np.float64)), 6)
    assert rel_l2(xs.cpu().numpy(), xr) <= RTOL_X
    plan.close()
    tile.close()


def test_streaming_batch_mixing_variants_equals_each_alone(orc):
    """A batch of streaming-shape problems with the L1 term, bf16 directions and the L2 term
    (one launch per variant group, the reduction kernel after them) gives each projection its
    own solve (whose single launch reduces in the pass) bit for bit."""
    from paper_2108_04315_b300 import binding as B
    psf = gen.gaussian_psf(5, 0.5)
    variants = [dict(), dict(data_norm=B.MISR_NORM_L1, data_eps=0.02), dict(iterate_dtype=B.MISR_BF16),
                dict(data_norm=B.MISR_NORM_L1, data_eps=0.05, iterate_dtype=B.MISR_BF16), dict()]
    plans, ys = [], []
    for i, kw in enumerate(variants):
        h, w = 36 + 8 * i, 60 + 20 * i
        P = orc.Problem(h, w, 2, gen.half_pixel_shifts(), psf, lam=0.01)
        y = P.forward_all(gen.phantom(2 * h, 2 * w, 80 + i)) + gen.gaussian_noise((4, h, w), 0.01, 90 + i)
        plans.append(B.Plan(h, w, 2, gen.half_pixel_shifts(), psf, lam=0.01, iters=10, tile_shape=4, **kw))
        ys.append(to_dev(y.astype(np.float32)))
    alone = [p.solve(y)[0].clone() for p, y in zip(plans, ys)]
    batch = B.Batch(plans)
    xs, _ = batch.solve(ys)
    for i, (a, b) in enumerate(zip(alone, xs)):
        assert torch.equal(a, b), f"projection {i} ({variants[i]})"
    batch.close()
