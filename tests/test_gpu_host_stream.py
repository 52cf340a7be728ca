"""misr_solve_host_many: a stream of projections from host memory, the copies of one overlapped
with the solve of another.  Each projection is solved alone on the plan, so its image and
statistics must equal its own misr_solve_host bit for bit, with page-locked or pageable host
buffers, with a given start point, and for any count (0, 1, odd, even)."""
import numpy as np
import pytest

import gen
from tests.gpu_common import RTOL_X, make_case, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PSF = gen.gaussian_psf(5, 0.5)


def _frames(orc, n, h=37, w=53, iters=12, **kw):
    P, plan, xt, y0 = make_case(orc, h, w, 2, gen.half_pixel_shifts(), PSF, seed=3000, iters=iters, **kw)
    ys = [y0] + [(y0 + gen.gaussian_noise(y0.shape, 0.05, 3100 + k)).astype(np.float32) for k in range(1, n)]
    return P, plan, ys


def _pinned(a):
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return t, t.numpy()


@pytest.mark.parametrize("n,shape", [(1, 0), (2, 0), (5, 0), (3, 4)])   # 4: MISR_TILE_STREAM
def test_stream_equals_one_at_a_time(orc, n, shape):
    P, plan, ys = _frames(orc, n, tile_shape=shape)
    H, W = plan.H, plan.W
    alone = []
    for y in ys:
        x = np.empty((H, W), dtype=np.float32)
        st = plan.solve_host(np.ascontiguousarray(y), x)
        alone.append((x, st))
    keep = [_pinned(y) for y in ys]                    # page-locked frames
    outs = [_pinned(np.zeros((H, W), dtype=np.float32)) for _ in ys]
    stats = plan.solve_host_many([k[1] for k in keep], [o[1] for o in outs])
    for k in range(n):
        assert np.array_equal(outs[k][1], alone[k][0]), f"projection {k}"
        assert stats[k] == alone[k][1]
    # the first projection also matches the FP64 oracle
    y64 = ys[0].astype(np.float64)
    xr, _ = P.scg(y64, P.shift_add(y64), plan.iters)
    assert rel_l2(outs[0][1], xr) <= RTOL_X


def test_stream_pageable_buffers_and_reuse(orc):
    P, plan, ys = _frames(orc, 3, h=23, w=29)
    H, W = plan.H, plan.W
    ref = []
    for y in ys:
        x = np.empty((H, W), dtype=np.float32)
        plan.solve_host(np.ascontiguousarray(y), x)
        ref.append(x)
    for _ in range(2):                                 # the plan's stream buffers are reused
        outs = [np.full((H, W), np.nan, dtype=np.float32) for _ in ys]
        plan.solve_host_many([np.ascontiguousarray(y) for y in ys], outs, stats=False)
        for k in range(3):
            assert np.array_equal(outs[k], ref[k])
    assert plan.solve_host_many([], []) == []


def test_stream_given_start_points(orc):
    from paper_2108_04315_b300 import binding as B
    P, plan, ys = _frames(orc, 3, h=30, w=41, iters=8, x0_mode=B.MISR_X0_GIVEN)
    H, W = plan.H, plan.W
    x0s = [gen.random_field((H, W), 50 + k, 0.0, 1.0).astype(np.float32) for k in range(3)]
    ref = []
    for y, x0 in zip(ys, x0s):
        x = x0.copy()
        st = plan.solve_host(np.ascontiguousarray(y), x)
        ref.append((x, st))
    outs = [x0.copy() for x0 in x0s]
    stats = plan.solve_host_many([np.ascontiguousarray(y) for y in ys], outs)
    for k in range(3):
        assert np.array_equal(outs[k], ref[k][0]) and stats[k] == ref[k][1]


def test_stream_rejects_null_entries():
    from paper_2108_04315_b300 import binding as B
    plan = B.Plan(16, 16, 2, gen.half_pixel_shifts(), PSF, iters=2)
    y = np.zeros((4, 16, 16), dtype=np.float32)
    with pytest.raises(B.MisrError) as e:
        B.misr_solve_host_many(plan.handle, [y.ctypes.data, 0], [0, 0])
    assert e.value.status == B.MISR_EINVAL


def test_stream_frame_wise_projections(orc):
    """The synthetic study's frame set (the frame-wise pass) streamed from host memory: each
    projection equals its own misr_solve_host bit for bit, the first one the oracle."""
    from tests.gpu_common import GENERAL_SEED, general_case
    P, plan, xt, y0 = general_case(orc, "study_bin_psf3", GENERAL_SEED, iters=7)
    ys = [y0] + [(y0 + gen.gaussian_noise(y0.shape, 0.05, 3200 + k)).astype(np.float32) for k in range(1, 3)]
    H, W = plan.H, plan.W
    alone = []
    for y in ys:
        x = np.empty((H, W), dtype=np.float32)
        st = plan.solve_host(np.ascontiguousarray(y), x)
        alone.append((x, st))
    keep = [_pinned(y) for y in ys]
    outs = [_pinned(np.zeros((H, W), dtype=np.float32)) for _ in ys]
    stats = plan.solve_host_many([k[1] for k in keep], [o[1] for o in outs])
    for k in range(len(ys)):
        assert np.array_equal(outs[k][1], alone[k][0]), f"projection {k}"
        assert stats[k] == alone[k][1]
    y64 = ys[0].astype(np.float64)
    xr, _ = P.scg(y64, P.shift_add(y64), 7)
    assert rel_l2(outs[0][1], xr) <= RTOL_X
    plan.close()
