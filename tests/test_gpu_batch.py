"""Batched solves (misr_batch_*): several projections of uneven sizes, magnification factors,
frame counts and iteration counts advanced by one fused-pass launch per SCG step (and the
projections that fill the GPU on their own by their own passes on streams of their own).  Each
projection keeps its own state and fixed-order reductions, so its result must equal its own
misr_solve bit for bit, and both must match the FP64 oracle."""
import numpy as np
import pytest

import gen
from tests.gpu_common import RTOL_X, make_case, rel_l2, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GEOMS = [
    # (h, w, f, shifts, iters)
    (64, 64, 2, gen.half_pixel_shifts(), 20),
    (37, 53, 2, gen.half_pixel_shifts(), 12),
    (23, 29, 3, gen.third_pixel_shifts(), 16),
    (48, 30, 3, gen.third_pixel_shifts(), 20),
    (17, 90, 2, gen.half_pixel_shifts(), 9),
]


def test_batch_equals_individual_solves_and_oracle(orc):
    from paper_2108_04315_b300 import binding as B
    psf = gen.gaussian_psf(5, 0.5)
    cases = [make_case(orc, h, w, f, sh, psf, seed=1000 + i, iters=it) for i, (h, w, f, sh, it) in enumerate(GEOMS)]
    plans = [c[1] for c in cases]
    ys = [to_dev(c[3]) for c in cases]
    alone = []
    for plan, y in zip(plans, ys):
        x, st = plan.solve(y)
        alone.append((x.clone(), st))
    batch = B.Batch(plans)
    xs, stats = batch.solve(ys)
    for i, ((P, plan, xt, y), (xa, sa), xb, sb) in enumerate(zip(cases, alone, xs, stats)):
        assert torch.equal(xa, xb), f"projection {i} differs between batch and alone"
        assert sa == sb
        assert sb["iters_done"] == GEOMS[i][4]
        y64 = y.astype(np.float64)
        xr, _ = P.scg(y64, P.shift_add(y64), GEOMS[i][4])
        assert rel_l2(xb.cpu().numpy(), xr) <= RTOL_X
    # a second solve of the same batch with new frames reuses the graph and the tables
    ys2 = [y + 0.01 * torch.ones_like(y) for y in ys]
    xs2, stats2 = batch.solve(ys2)
    for plan, y2, xb2 in zip(plans, ys2, xs2):
        xa2, _ = plan.solve(y2)
        assert torch.equal(xa2, xb2)
    batch.close()


def test_batch_rejects_duplicate_plans(orc):
    from paper_2108_04315_b300 import binding as B
    P, plan, xt, y = make_case(orc, 16, 16, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5), seed=7, iters=2)
    with pytest.raises(B.MisrError) as e:
        B.Batch([plan, plan])
    assert e.value.status == B.MISR_EINVAL


def _large_frames(h, w, seed):
    """Frames of a 2h x 2w projection made on the device (the oracle is not needed here: the
    check is bitwise equality with the projection's own misr_solve)."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return (0.5 + 0.1 * torch.rand((4, h, w), device="cuda", generator=g)).contiguous()


def test_grid_filling_projections_on_their_own_streams_equal_each_alone():
    """Projections that fill the GPU on their own (streaming shape, 2048^2 and 2560 x 2048 HR)
    run their plans' own passes on streams of their own inside the batch step and in the server's
    ticks, beside a small projection that shares the step's launches: every result equals its
    own misr_solve bit for bit."""
    from paper_2108_04315_b300 import binding as B
    psf = gen.gaussian_psf(5, 0.5)
    geoms = [(1024, 1024, 6), (1280, 1024, 5), (40, 52, 7)]
    plans = [B.Plan(h, w, 2, gen.half_pixel_shifts(), psf, iters=it,
                    tile_shape=B.MISR_TILE_STREAM if h > 100 else B.MISR_TILE_AUTO) for h, w, it in geoms]
    ys = [_large_frames(h, w, 70 + i) for i, (h, w, _) in enumerate(geoms)]
    alone = []
    for p, y in zip(plans, ys):
        x, st = p.solve(y)
        alone.append((x.clone(), st))
    batch = B.Batch(plans)
    for _ in range(2):   # the step graph replayed
        xs, stats = batch.solve(ys)
        for (xa, sa), xb, sb in zip(alone, xs, stats):
            assert torch.equal(xa, xb) and sa == sb
    batch.close()
    srv = B.Server(max_slots=4, passes_per_tick=2)
    tickets = [srv.submit(y, h, w, 2, gen.half_pixel_shifts(), psf, iters=it,
                          tile_shape=B.MISR_TILE_STREAM if h > 100 else B.MISR_TILE_AUTO)
               for (h, w, it), y in zip(geoms, ys)]
    for t, (xa, sa) in zip(tickets, alone):
        x, st, _ = srv.wait(t, timeout_s=120.0)
        assert torch.equal(x, xa) and st == sa
    srv.close()
    for p in plans:
        p.close()
