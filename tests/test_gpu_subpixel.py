"""Non-integer detector shifts (bilinear M_k, reading of Eq. 1): each frame's HR shift t = n + a
per axis, the samples at HR phase n and the blur widened by the bilinear's second tap, with the
taps per phase (a product lattice of shifts, as x and y stages give) and the bilinear's first
part alone where its second part would read B's padding.  CUDA library vs the FP64 oracle's
bilinear M_k, through the C ABI; the same bars as the integer-shift path."""
import numpy as np
import pytest

import gen
from tests.gpu_common import RTOL_J, RTOL_OP, RTOL_X, asym_separable_psf, rel_l2, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def lattice(xs, ys):
    """Frames on the product of x shifts and y shifts (LR px)."""
    return [(dx, dy) for dy in ys for dx in xs]


CASES = {
    # name: (h, w, f, shifts, psf, binned)
    "f2_frac": (37, 45, 2, lattice([0.0, 0.55], [0.05, 0.6]), gen.gaussian_psf(3, 0.6), False),
    "f3_frac_k9": (23, 29, 3, lattice([0.02, 0.36, 0.7], [0.1, 0.4, 0.75]), asym_separable_psf(6, 3), False),
    "f2_frac_partial": (30, 41, 2, lattice([0.0, 0.55], [0.05, 0.6])[:3], asym_separable_psf(7, 3), False),
    "f2_frac_x_only": (33, 40, 2, lattice([0.1, 0.65], [0.0, 0.5]), gen.gaussian_psf(3, 0.5), False),
    "f2_frac_bin_delta": (35, 38, 2, lattice([0.0, 0.55], [0.05, 0.6]), np.ones((1, 1)), True),
    "f1_frac": (45, 70, 1, [(0.3, 0.7)], gen.gaussian_psf(3, 0.6), False),
    "thin_strip": (1, 61, 2, lattice([0.0, 0.55], [0.05, 0.6]), gen.gaussian_psf(3, 0.6), False),
}


def frac_case(orc, name, seed, iters=20, lam=0.01, l1_eps=None, **plan_kw):
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts, psf, binned = CASES[name]
    kw_o, kw_p = {}, {}
    if l1_eps:
        kw_o.update(data_norm=orc.NORM_L1, data_eps=l1_eps)
        kw_p.update(data_norm=B.MISR_NORM_L1, data_eps=l1_eps)
    if binned:
        kw_o.update(decimation=orc.DECIM_BIN)
        kw_p.update(decimation=B.MISR_DECIM_BIN)
    P = orc.Problem(h, w, f, shifts, psf, lam=lam, **kw_o)
    xt = gen.phantom(f * h, f * w, seed)
    y = P.forward_all(xt) + gen.gaussian_noise((len(shifts), h, w), 0.01, seed + 1)
    plan = B.Plan(h, w, f, shifts, psf, lam=lam, iters=iters, **kw_p, **plan_kw)
    return P, plan, xt, y.astype(np.float32)


@pytest.mark.parametrize("name", sorted(CASES))
def test_subpixel_forward_operator(orc, name):
    P, plan, xt, _ = frac_case(orc, name, 100)
    x = (xt + gen.random_field(xt.shape, 7, -0.5, 0.5)).astype(np.float32)
    y = plan.forward(to_dev(x)).cpu().numpy()
    ref = P.forward_all(x.astype(np.float64))
    for k in range(P.K):
        assert rel_l2(y[k], ref[k]) <= RTOL_OP, (name, k)


@pytest.mark.parametrize("name", sorted(CASES))
def test_subpixel_objective_and_gradient(orc, name):
    P, plan, xt, y = frac_case(orc, name, 200)
    x = (xt + gen.random_field(xt.shape, 8, -0.2, 0.2)).astype(np.float32)
    J, g = plan.gradient(to_dev(y), to_dev(x))
    Jr, gr = P.gradient(x.astype(np.float64), y.astype(np.float64))
    assert J == pytest.approx(Jr, rel=RTOL_J)
    assert rel_l2(g.cpu().numpy(), gr) <= RTOL_OP


@pytest.mark.parametrize("name", ["f2_frac", "f3_frac_k9", "f2_frac_bin_delta", "f1_frac"])
def test_subpixel_fused_pass(orc, name):
    alpha, beta = 0.3, 0.7
    P, plan, xt, y = frac_case(orc, name, 300)
    x = (xt + gen.random_field(xt.shape, 9, -0.1, 0.1)).astype(np.float32)
    r = gen.random_field(xt.shape, 10, -0.3, 0.3).astype(np.float32)
    po = gen.random_field(xt.shape, 11, -0.3, 0.3).astype(np.float32)
    xo, ro, pn, S = plan.pass_probe(to_dev(y), to_dev(x), to_dev(r), to_dev(po), alpha, beta)
    xo, ro, pn = (t.cpu().numpy().astype(np.float64) for t in (xo, ro, pn))
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    h, w, f, shifts, psf, binned = CASES[name]
    P0 = orc.Problem(h, w, f, shifts, psf, lam=0.0, **(dict(decimation=orc.DECIM_BIN) if binned else {}))
    J, g = P.gradient(xo, y64)
    r_ref = -g
    assert rel_l2(ro, r_ref) <= RTOL_OP
    ref = {
        "J_data": P0.objective(xo, y64),
        "dJ_data": P0.objective(x64 + alpha * pn, y64) - P0.objective(x64, y64),
        "R_btv": P.reg_value(xo),
        "rr": float(np.sum(r_ref * r_ref)),
        "pp": float(np.sum(pn * pn)),
        "a": P.curvature(xo, r_ref),
        "b": float(np.sum(r_ref * P.hessvec(xo, pn))),
        "c": P.curvature(xo, pn),
    }
    scale = {"dJ_data": abs(ref["J_data"]) * 1e-7, "b": np.sqrt(abs(ref["a"] * ref["c"])) * 1e-6}
    for k, v in ref.items():
        assert abs(S[k] - v) <= RTOL_OP * abs(v) + scale.get(k, 0.0) + 1e-30, (k, S[k], v)


@pytest.mark.parametrize("name,iters,l1_eps", [("f2_frac", 20, None), ("f3_frac_k9", 12, None),
                                               ("f2_frac_bin_delta", 15, None), ("f2_frac", 15, 0.02)])
def test_subpixel_solve_matches_oracle(orc, name, iters, l1_eps):
    P, plan, xt, y = frac_case(orc, name, 400, iters=iters, l1_eps=l1_eps)
    y64 = y.astype(np.float64)
    xg, st = plan.solve(to_dev(y))
    xr, tr = P.scg(y64, P.shift_add(y64), iters)
    assert st["iters_done"] == iters
    assert rel_l2(xg.cpu().numpy(), xr) <= RTOL_X
    assert st["J_final"] == pytest.approx(P.objective(xr, y64), rel=1e-4)
    sig = np.abs(tr["E"] - tr["J_trial"]) > 1e-6 * np.abs(tr["E"])
    assert np.array_equal(plan.trace()["accept"][sig], tr["accept"][sig])


@pytest.mark.parametrize("name", ["f2_frac", "f3_frac_k9", "f2_frac_partial", "f1_frac"])
def test_subpixel_interpolation_and_start_point(orc, name):
    """misr_interpolate and a zero-iteration solve give the oracle's bilinear shift-and-add
    (FP32 weights and division: a few ulps)."""
    from paper_2108_04315_b300 import binding as B
    P, plan, xt, y = frac_case(orc, name, 500, iters=0)
    ref = P.shift_add(y.astype(np.float64))
    xi = plan.interpolate(to_dev(y)).cpu().numpy()
    np.testing.assert_allclose(xi, ref, rtol=2e-6, atol=1e-6)
    x0, _ = plan.solve(to_dev(y))
    assert np.array_equal(x0.cpu().numpy(), xi)


def test_subpixel_routing():
    """Shift sets the per-phase-tap pass cannot take run the frame-wise pass (checked against the
    oracle in tests/test_gpu_general.py); an explicit tile shape other than 32x32 for a product
    lattice of non-integer shifts is refused."""
    from paper_2108_04315_b300 import binding as B
    psf3 = gen.gaussian_psf(3, 0.5)
    for sh, psf in (([(0.0, 0.0), (0.55, 0.0), (0.0, 0.5), (0.6, 0.5)], psf3),     # not a product lattice
                    (lattice([0.0, 0.55], [0.0, 0.5]), gen.gaussian_psf(5, 0.5)),  # 5x5 PSF: 6 taps
                    ([(1.0, 0.0)], psf3)):                                           # a whole LR pixel
        assert B.misr_autotune(B.make_desc(16, 16, 2, sh, psf, iters=1), 1)[0] == B.MISR_TILE_AUTO
        p = B.Plan(16, 16, 2, sh, psf, iters=1)
        y = torch.zeros((len(sh), 16, 16), dtype=torch.float32, device="cuda")
        x, st = p.solve(y)
        assert st["iters_done"] == 0 and not torch.any(x)   # zero frames: the gradient at x_1 = 0 is 0
        p.close()
    with pytest.raises(B.MisrError) as e:              # per-phase taps on another tile shape
        B.Plan(16, 16, 2, lattice([0.0, 0.55], [0.0, 0.5]), psf3, iters=1, tile_shape=B.MISR_TILE_32x64)
    assert e.value.status == B.MISR_ENOTIMPL


def test_subpixel_and_integer_in_one_batch_equal_each_alone(orc):
    from paper_2108_04315_b300 import binding as B
    from tests.gpu_common import make_case
    cases = [frac_case(orc, "f2_frac", 600, iters=8),
             make_case(orc, 37, 45, 2, gen.half_pixel_shifts(), gen.gaussian_psf(3, 0.6), seed=601, iters=9),
             frac_case(orc, "f3_frac_k9", 602, iters=7, l1_eps=0.05, iterate_dtype=B.MISR_BF16)]
    plans = [c[1] for c in cases]
    ys = [to_dev(c[3]) for c in cases]
    alone = []
    for p, y in zip(plans, ys):
        x, st = p.solve(y)
        alone.append((x.clone(), st))
    batch = B.Batch(plans)
    xs, stats = batch.solve(ys)
    for (xa, sa), xb, sb in zip(alone, xs, stats):
        assert torch.equal(xa, xb) and sa == sb
    batch.close()


def test_subpixel_gradient_noalloc_equals_plan_gradient(orc):
    import ctypes as C
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts, psf, binned = CASES["f3_frac_k9"]
    P, plan, xt, y = frac_case(orc, "f3_frac_k9", 1110)
    yd, xd = to_dev(y), to_dev(xt.astype(np.float32))
    J_ref, g_ref = plan.gradient(yd, xd)
    fn = B.lib().misr_gradient_noalloc
    fn.argtypes = [C.POINTER(B.misr_desc), C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]
    fn.restype = C.c_int
    desc = B.make_desc(h, w, f, shifts, psf, lam=0.01, iters=1)
    g = torch.full_like(xd, float("nan"))
    J = C.c_double()
    rc = fn(C.byref(desc), yd.data_ptr(), xd.data_ptr(), g.data_ptr(), C.byref(J),
            torch.cuda.current_stream().cuda_stream)
    assert rc == B.MISR_OK, B.misr_last_error()
    assert rel_l2(g.cpu().numpy(), g_ref.cpu().numpy()) <= RTOL_OP
    assert J.value == pytest.approx(J_ref, rel=RTOL_OP)
