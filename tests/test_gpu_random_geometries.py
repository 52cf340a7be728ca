"""Seeded random geometries against the FP64 oracle: factor 1..4, a random subset of the HR
phases (one frame each), random separable PSFs of size 1, 3 or 5, point or binning D, L2 or L1
data term, integer or non-integer (product-lattice) shifts, ragged LR sizes from 1 to 40.  Each
draw is checked on the forward operator and the gradient (the L2 path's bars; the L1 bars of
tests/test_gpu_l1.py where the L1 term is used).  Draws whose combined blur is too wide for the
fused passes' taps (binning or non-integer shifts with a wide PSF) run the frame-wise pass and
meet the same bars.  A second family draws frame sets anywhere: shifts in [-1.5, 1.5] LR px,
several frames per phase, K up to 2 f^2 (the frame-wise pass)."""
import numpy as np
import pytest

import gen
from tests.gpu_common import RTOL_J, RTOL_OP, rel_l2, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U = 2.0 ** -24


def draw(seed):
    rng = np.random.default_rng(seed)
    f = int(rng.integers(1, 5))
    h, w = (int(v) for v in rng.integers(1, 41, size=2))
    phases = [(py, px) for py in range(f) for px in range(f)]
    K = int(rng.integers(1, f * f + 1))
    pick = [phases[i] for i in rng.choice(len(phases), size=K, replace=False)]
    frac = bool(rng.integers(0, 2)) and f > 1
    ay = rng.uniform(0.0, 0.9, size=f) if frac else np.zeros(f)
    ax = rng.uniform(0.0, 0.9, size=f) if frac else np.zeros(f)
    shifts = [((px + ax[px]) / f, (py + ay[py]) / f) for py, px in pick]
    size = int(rng.choice([1, 3, 5]))
    u, v = rng.uniform(0.1, 1.0, size=(2, size))
    psf = np.outer(u, v)
    binned = bool(rng.integers(0, 2))
    l1 = bool(rng.integers(0, 2))
    return dict(f=f, h=h, w=w, shifts=shifts, psf=psf / psf.sum(), binned=binned, l1=l1, frac=frac)


def fits(d):
    R = d["psf"].shape[0] // 2
    widen = (d["f"] - 1 if d["binned"] else 0) + (1 if d["frac"] else 0)
    return R + widen <= 2


@pytest.mark.parametrize("seed", range(40))
def test_random_geometry_matches_oracle(orc, seed):
    from paper_2108_04315_b300 import binding as B
    d = draw(9000 + seed)
    kw_p = dict(lam=0.01, iters=1)
    kw_o = dict(lam=0.01)
    if d["binned"]:
        kw_p["decimation"] = B.MISR_DECIM_BIN
        kw_o["decimation"] = orc.DECIM_BIN
    eps_d = 0.05
    if d["l1"]:
        kw_p.update(data_norm=B.MISR_NORM_L1, data_eps=eps_d)
        kw_o.update(data_norm=orc.NORM_L1, data_eps=eps_d)
    plan = B.Plan(d["h"], d["w"], d["f"], d["shifts"], d["psf"], **kw_p)
    P = orc.Problem(d["h"], d["w"], d["f"], d["shifts"], d["psf"], **kw_o)
    x = (gen.phantom(P.H, P.W, seed) + gen.random_field((P.H, P.W), seed + 1, -0.2, 0.2)).astype(np.float32)
    y = (P.forward_all(x.astype(np.float64)) + gen.gaussian_noise((P.K, d["h"], d["w"]), 0.05, seed + 2)
         ).astype(np.float32)
    yd = plan.forward(to_dev(x)).cpu().numpy()
    ref = P.forward_all(x.astype(np.float64))
    for k in range(P.K):
        assert rel_l2(yd[k], ref[k]) <= RTOL_OP, (d, k)
    J, g = plan.gradient(to_dev(y), to_dev(x))
    Jr, gr = P.gradient(x.astype(np.float64), y.astype(np.float64))
    tol = RTOL_OP + (16 * U * float(np.abs(y).max()) / eps_d if d["l1"] else 0.0)
    assert J == pytest.approx(Jr, rel=RTOL_J), d
    assert rel_l2(g.cpu().numpy(), gr) <= tol, d
    plan.close()
    if not d["frac"] and fits(d):   # integer shifts: the streaming shape too
        plan = B.Plan(d["h"], d["w"], d["f"], d["shifts"], d["psf"], tile_shape=B.MISR_TILE_STREAM, **kw_p)
        J, g = plan.gradient(to_dev(y), to_dev(x))
        assert J == pytest.approx(Jr, rel=RTOL_J), d
        assert rel_l2(g.cpu().numpy(), gr) <= tol, d
        plan.close()


def draw_general(seed):
    rng = np.random.default_rng(seed)
    f = int(rng.integers(1, 5))
    h, w = (int(v) for v in rng.integers(1, 41, size=2))
    K = int(rng.integers(1, 2 * f * f + 1))
    integer = bool(rng.integers(0, 2))
    if integer:
        shifts = [tuple(float(v) / f for v in rng.integers(-f - f // 2, f + f // 2 + 1, size=2)) for _ in range(K)]
    else:
        shifts = [tuple(float(v) for v in rng.uniform(-1.5, 1.5, size=2)) for _ in range(K)]
    size = int(rng.choice([1, 3, 5]))
    u, v = rng.uniform(0.1, 1.0, size=(2, size))
    psf = np.outer(u, v)
    return dict(f=f, h=h, w=w, shifts=shifts, psf=psf / psf.sum(), binned=bool(rng.integers(0, 2)),
                l1=bool(rng.integers(0, 2)))


@pytest.mark.parametrize("seed", range(30))
def test_random_frame_set_matches_oracle(orc, seed):
    from paper_2108_04315_b300 import binding as B
    d = draw_general(9500 + seed)
    kw_p = dict(lam=0.01, iters=1)
    kw_o = dict(lam=0.01)
    if d["binned"]:
        kw_p["decimation"] = B.MISR_DECIM_BIN
        kw_o["decimation"] = orc.DECIM_BIN
    eps_d = 0.05
    if d["l1"]:
        kw_p.update(data_norm=B.MISR_NORM_L1, data_eps=eps_d)
        kw_o.update(data_norm=orc.NORM_L1, data_eps=eps_d)
    plan = B.Plan(d["h"], d["w"], d["f"], d["shifts"], d["psf"], **kw_p)
    P = orc.Problem(d["h"], d["w"], d["f"], d["shifts"], d["psf"], **kw_o)
    x = (gen.phantom(P.H, P.W, seed) + gen.random_field((P.H, P.W), seed + 1, -0.2, 0.2)).astype(np.float32)
    y = (P.forward_all(x.astype(np.float64)) + gen.gaussian_noise((P.K, d["h"], d["w"]), 0.05, seed + 2)
         ).astype(np.float32)
    yd = plan.forward(to_dev(x)).cpu().numpy()
    ref = P.forward_all(x.astype(np.float64))
    for k in range(P.K):
        if np.any(ref[k]):
            assert rel_l2(yd[k], ref[k]) <= RTOL_OP, (d, k)
        else:   # the frame sees no pixel of the grid
            assert not np.any(yd[k]), (d, k)
    J, g = plan.gradient(to_dev(y), to_dev(x))
    Jr, gr = P.gradient(x.astype(np.float64), y.astype(np.float64))
    tol = RTOL_OP + (16 * U * float(np.abs(y).max()) / eps_d if d["l1"] else 0.0)
    assert J == pytest.approx(Jr, rel=RTOL_J), d
    assert rel_l2(g.cpu().numpy(), gr) <= tol, d
    x0 = plan.interpolate(to_dev(y)).cpu().numpy()
    # a weighted mean of at most 4 K samples: (4 K + 8) rounding errors of max |y| at most
    assert float(np.abs(x0 - P.shift_add(y.astype(np.float64))).max()) <= (4 * P.K + 8) * U * float(np.abs(y).max()), d
    plan.close()
