"""Checkpoint and resume: a solve stopped after N1 iterations, exported, imported into a plan of
the same geometry with N iterations and resumed, gives the image, statistics and trace of one
uninterrupted N-iteration solve bit for bit (float and bf16 directions, two tile shapes and the
streaming one), and the checkpoint survives a solve of other data on the plan in between.
Malformed checkpoints fail
with a status."""
import numpy as np
import pytest

import gen
from tests.gpu_common import make_case, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PSF = gen.gaussian_psf(5, 0.5)


@pytest.mark.parametrize("iterate,tile_shape", [("f32", 2), ("bf16", 2), ("f32", 3), ("f32", 4), ("bf16", 4)])
def test_resume_equals_uninterrupted(orc, iterate, tile_shape):
    from paper_2108_04315_b300 import binding as B
    dt = B.MISR_BF16 if iterate == "bf16" else B.MISR_F32
    N, N1 = 14, 6
    kw = dict(tile_shape=tile_shape, iterate_dtype=dt)
    P, full, xt, y = make_case(orc, 37, 53, 2, gen.half_pixel_shifts(), PSF, seed=5000, iters=N, **kw)
    yd = to_dev(y)
    x_full, st_full = full.solve(yd)
    tr_full = full.trace()
    short = B.Plan(37, 53, 2, gen.half_pixel_shifts(), PSF, iters=N1, **kw)
    short.solve(yd)
    ck = short.export_state()
    assert ck.nbytes == B.misr_state_bytes(short.handle)
    cont = B.Plan(37, 53, 2, gen.half_pixel_shifts(), PSF, iters=N, **kw)
    cont.import_state(ck)
    x_res, st_res = cont.resume(yd)
    assert torch.equal(x_res, x_full)
    assert st_res == st_full
    tr = cont.trace()
    assert tr.keys() == tr_full.keys()
    for k in tr:                                   # rows of the iterations run on this plan
        assert len(tr[k]) == len(tr_full[k]) == N
        assert np.array_equal(tr[k][N1:], tr_full[k][N1:]), k
        assert not np.any(tr[k][:N1]), k


def test_checkpoint_survives_other_work_and_reimport(orc):
    from paper_2108_04315_b300 import binding as B
    N, N1 = 10, 4
    P, full, xt, y = make_case(orc, 30, 41, 2, gen.half_pixel_shifts(), PSF, seed=5100, iters=N)
    yd = to_dev(y)
    x_full, st_full = full.solve(yd)
    plan = B.Plan(30, 41, 2, gen.half_pixel_shifts(), PSF, iters=N1)
    plan.solve(yd)
    ck = plan.export_state()
    # other data through the same plan, then the checkpoint back (into the N1 plan: its count
    # is reached, so the resume only writes the image out)
    other = (y + 0.3).astype(np.float32)
    plan.solve(to_dev(other))
    plan.import_state(ck)
    x4, st4 = plan.resume(yd)
    assert st4["iters_done"] == N1
    # and on into a plan with the full count
    cont = B.Plan(30, 41, 2, gen.half_pixel_shifts(), PSF, iters=N)
    cont.import_state(ck)
    x_res, st_res = cont.resume(yd)
    assert torch.equal(x_res, x_full) and st_res == st_full


def test_bad_checkpoints_rejected():
    from paper_2108_04315_b300 import binding as B
    a = B.Plan(16, 16, 2, gen.half_pixel_shifts(), PSF, iters=2)
    b = B.Plan(16, 24, 2, gen.half_pixel_shifts(), PSF, iters=2)
    c = B.Plan(16, 16, 2, gen.half_pixel_shifts(), PSF, iters=2, iterate_dtype=B.MISR_BF16)
    a.solve(torch.zeros((4, 16, 16), dtype=torch.float32, device="cuda"))
    ck = a.export_state()
    for plan in (b, c):                                  # other geometry, other storage type
        with pytest.raises(B.MisrError) as e:
            plan.import_state(ck)
        assert e.value.status == B.MISR_EINVAL
    with pytest.raises(B.MisrError) as e:                # truncated
        a.import_state(ck[:-1])
    assert e.value.status == B.MISR_EINVAL
    bad = ck.copy()
    bad[0] ^= 0xff                                       # not a checkpoint
    with pytest.raises(B.MisrError) as e:
        a.import_state(bad)
    assert e.value.status == B.MISR_EINVAL
    for other in (dict(psf=gen.gaussian_psf(5, 0.8)), dict(lam=0.02), dict(eps=2e-3),
                  dict(shifts=[(0.0, 0.0), (0.5, 0.0), (0.0, 0.5)]), dict(psf=gen.gaussian_psf(3, 0.5),
                                                                           decimation=B.MISR_DECIM_BIN)):
        kw = dict(shifts=gen.half_pixel_shifts(), psf=PSF, lam=0.01, eps=1e-3)
        kw.update(other)
        d = B.Plan(16, 16, 2, kw.pop("shifts"), kw.pop("psf"), iters=2, **kw)
        with pytest.raises(B.MisrError) as e:            # another model of the same geometry
            d.import_state(ck)
        assert e.value.status == B.MISR_EINVAL
    B.Plan(16, 16, 2, gen.half_pixel_shifts(), PSF, iters=7).import_state(ck)   # another count: fine
    a.import_state(ck)                                   # the real one still loads
