"""The smoothed L1 data term (misr_desc.data_norm = MISR_NORM_L1): the data term of the paper's
experiments (Sec. 3.1), each residual t smoothed as psi_d(t) = sqrt(t^2 + eps_d^2) - eps_d.
CUDA library vs the FP64 oracle's L1 term, through the C ABI, on frames with Gaussian noise
and sparse outliers (defective detector pixels, the case an L1 data term is for).

Tolerances.  The device forms each residual e = (B x)(c) - y(c) in FP32, a few ulps of the
blurred value: |de| <= 8 u max|y| (u = 2^-24).  The L1 term's gradient takes psi_d'(e), whose
slope is at most psi_d'' <= 1/eps_d, and its curvature weights psi_d''(e), whose relative slope
|d ln psi_d''/de| is at most sqrt(2)/eps_d; so the L2 path's bars (RTOL_OP for operator
applications and pass sums) widen by 16 u max|y| / eps_d here.
"""
import numpy as np
import pytest

import gen
from tests.gpu_common import RTOL_J, RTOL_OP, RTOL_X, asym_separable_psf, rel_l2, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U = 2.0 ** -24

CASES = {
    # name: (h, w, f, shifts, psf)
    "tiny_f2": (64, 64, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)),
    "ragged_f2_asym": (37, 53, 2, gen.half_pixel_shifts(), asym_separable_psf(3)),
    "ragged_f3_k9": (23, 29, 3, gen.third_pixel_shifts(), gen.gaussian_psf(5, 0.5)),
    "partial_f2_k3": (30, 41, 2, [(0.0, 0.0), (0.5, 0.0), (0.5, 0.5)], asym_separable_psf(4, 3)),
    "f1_denoise": (45, 70, 1, [(0.0, 0.0)], gen.gaussian_psf(5, 0.6)),
    "thin_strip": (1, 97, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)),
}


def tol_l1(y, eps_d):
    return RTOL_OP + 16 * U * float(np.abs(y).max()) / eps_d


def l1_case(orc, name, seed, eps_d, iters=20, lam=0.01, **plan_kw):
    """(oracle problem with the L1 term, GPU plan, x_true, y float32): frames with Gaussian
    noise (sigma 0.01) and 2 % outliers of +-0.5."""
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts, psf = CASES[name]
    P = orc.Problem(h, w, f, shifts, psf, lam=lam, data_norm=orc.NORM_L1, data_eps=eps_d)
    xt = gen.phantom(f * h, f * w, seed)
    K = len(shifts)
    y = P.forward_all(xt) + gen.gaussian_noise((K, h, w), 0.01, seed + 1) + \
        gen.impulse_noise((K, h, w), 0.02, 0.5, seed + 2)
    plan = B.Plan(h, w, f, shifts, psf, lam=lam, iters=iters, data_norm=B.MISR_NORM_L1, data_eps=eps_d, **plan_kw)
    return P, plan, xt, y.astype(np.float32)


@pytest.mark.parametrize("shape", [2, 4])   # MISR_TILE_32x32, MISR_TILE_STREAM
@pytest.mark.parametrize("eps_d", [0.01, 0.1])
@pytest.mark.parametrize("name", sorted(CASES))
def test_l1_objective_and_gradient(orc, name, eps_d, shape):
    """J(x) = sum psi_d(A_k x - y_k) + lambda BTV(x) and grad J = sum A_k^T psi_d'(.) + lambda grad BTV."""
    P, plan, xt, y = l1_case(orc, name, 210, eps_d, tile_shape=shape)
    x = (xt + gen.random_field(xt.shape, 8, -0.2, 0.2)).astype(np.float32)
    J, g = plan.gradient(to_dev(y), to_dev(x))
    Jr, gr = P.gradient(x.astype(np.float64), y.astype(np.float64))
    assert J == pytest.approx(Jr, rel=RTOL_J)
    assert rel_l2(g.cpu().numpy(), gr) <= tol_l1(y, eps_d)


@pytest.mark.parametrize("name", ["tiny_f2", "ragged_f2_asym", "ragged_f3_k9", "partial_f2_k3", "f1_denoise",
                                  "thin_strip"])
@pytest.mark.parametrize("alpha,beta", [(0.3, 0.7), (0.0, 0.0), (1.7, 0.05)])
@pytest.mark.parametrize("shape", [2, 4])   # MISR_TILE_32x32, MISR_TILE_STREAM
def test_l1_fused_pass(orc, name, alpha, beta, shape):
    """One fused SCG pass with the L1 term: r' = -grad J(x') and the sums, the curvature forms
    with the L1 term's Hessian sum_k A_k^T diag(psi_d''(A_k x' - y_k)) A_k + lambda H_BTV(x')."""
    eps_d = 0.02
    P, plan, xt, y = l1_case(orc, name, 310, eps_d, tile_shape=shape)
    x = (xt + gen.random_field(xt.shape, 9, -0.1, 0.1)).astype(np.float32)
    r = gen.random_field(xt.shape, 10, -0.3, 0.3).astype(np.float32)
    po = gen.random_field(xt.shape, 11, -0.3, 0.3).astype(np.float32)
    xo, ro, pn, S = plan.pass_probe(to_dev(y), to_dev(x), to_dev(r), to_dev(po), alpha, beta)
    xo, ro, pn = (t.cpu().numpy().astype(np.float64) for t in (xo, ro, pn))
    x64, r64, po64, y64 = (a.astype(np.float64) for a in (x, r, po, y))
    assert rel_l2(pn, r64 + beta * po64) <= 1e-6
    assert rel_l2(xo, x64 + alpha * pn) <= 1e-6
    h, w, f, shifts, psf = CASES[name]
    P0 = orc.Problem(h, w, f, shifts, psf, lam=0.0, data_norm=orc.NORM_L1, data_eps=eps_d)
    J, g = P.gradient(xo, y64)
    r_ref = -g
    tol = tol_l1(y, eps_d)
    assert rel_l2(ro, r_ref) <= tol
    ref = {
        "J_data": P0.objective(xo, y64),
        "dJ_data": P0.objective(x64 + alpha * pn, y64) - P0.objective(x64, y64),
        "R_btv": P.reg_value(xo),
        "rr": float(np.sum(r_ref * r_ref)),
        "rr_cross": float(np.sum(r_ref * r64)),
        "pr": float(np.sum(pn * r_ref)),
        "pp": float(np.sum(pn * pn)),
        "a": P.curvature(xo, r_ref, y64),
        "b": float(np.sum(r_ref * P.hessvec(xo, pn, y64))),
        "c": P.curvature(xo, pn, y64),
    }
    # the sums that take the gradient (rr, rr_cross, pr) or the curvature weights (a, b, c)
    # get the L1 bar; the others keep the L2 path's
    wide = {"rr", "rr_cross", "pr", "a", "b", "c"}
    scale = {"dJ_data": abs(ref["J_data"]) * 1e-7, "b": np.sqrt(abs(ref["a"] * ref["c"])) * tol,
             "rr_cross": np.sqrt(ref["rr"] * np.sum(r64 * r64)) * tol, "pr": np.sqrt(ref["rr"] * ref["pp"]) * tol}
    for k, v in ref.items():
        rt = 2 * tol if k in wide else RTOL_OP
        assert abs(S[k] - v) <= rt * abs(v) + scale.get(k, 0.0) + 1e-30, (k, S[k], v)


def _decisions_agree(tg, tr):
    sig = np.abs(tr["E"] - tr["J_trial"]) > 1e-6 * np.abs(tr["E"])
    assert np.array_equal(tg["accept"][sig], tr["accept"][sig])
    assert int(np.sum(tg["accept"] != tr["accept"])) <= max(2, (~sig).sum() // 4)
    return sig


@pytest.mark.parametrize("name,iters,eps_d", [("tiny_f2", 20, 0.02), ("ragged_f2_asym", 15, 0.05),
                                              ("ragged_f3_k9", 12, 0.02), ("f1_denoise", 12, 0.05)])
@pytest.mark.parametrize("shape", [2, 4])   # MISR_TILE_32x32, MISR_TILE_STREAM
def test_l1_solve_matches_oracle(orc, name, iters, eps_d, shape):
    """SCG with the L1 term from multi-image interpolation: image, objective and decisions."""
    P, plan, xt, y = l1_case(orc, name, 410, eps_d, iters=iters, tile_shape=shape)
    y64 = y.astype(np.float64)
    xg, st = plan.solve(to_dev(y))
    xg = xg.cpu().numpy()
    xr, tr = P.scg(y64, P.shift_add(y64), iters)
    assert st["iters_done"] == iters
    assert rel_l2(xg, xr) <= RTOL_X
    assert st["J_final"] == pytest.approx(P.objective(xg.astype(np.float64), y64), rel=1e-6)
    assert st["J_final"] == pytest.approx(P.objective(xr, y64), rel=1e-4)
    tg = plan.trace()
    sig = _decisions_agree(tg, tr)
    np.testing.assert_allclose(tg["E"][sig], tr["E"][sig], rtol=1e-4)


def test_l1_is_robust_to_outliers_where_l2_is_not(orc):
    """What the L1 term is for: with 2 % outliers of +-0.5 in the frames, the L1 solve
    (lambda 0.2, eps_d 0.01) lands closer to the true image than the L2 solve of the same
    frames at any lambda of a sweep (the FP64 oracle gives 0.071 against 0.107 at best, at
    lambda 0.2; the prior supplies the redundancy the L1 fit needs to reject outliers when
    K = f^2 frames sample each HR pixel once)."""
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts, psf = CASES["tiny_f2"]
    P, plan1, xt, y = l1_case(orc, "tiny_f2", 510, 0.01, iters=60, lam=0.2)
    yd = to_dev(y)
    x1, _ = plan1.solve(yd)
    e1 = rel_l2(x1.cpu().numpy(), xt)
    e2 = {}
    for lam in (0.01, 0.1, 0.2, 0.5):
        x2, _ = B.Plan(h, w, f, shifts, psf, lam=lam, iters=60).solve(yd)
        e2[lam] = rel_l2(x2.cpu().numpy(), xt)
    assert e1 < 0.8 * min(e2.values()), (e1, e2)


@pytest.mark.parametrize("shape", [1, 2, 3, 4])
def test_l1_every_tile_shape(orc, shape):
    P, plan, xt, y = l1_case(orc, "ragged_f2_asym", 610, 0.02, iters=10, tile_shape=shape)
    y64 = y.astype(np.float64)
    xg, st = plan.solve(to_dev(y))
    xr, tr = P.scg(y64, P.shift_add(y64), 10)
    assert rel_l2(xg.cpu().numpy(), xr) <= RTOL_X
    _decisions_agree(plan.trace(), tr)


@pytest.mark.parametrize("shape", [2, 4])   # MISR_TILE_32x32, MISR_TILE_STREAM
def test_l1_bf16_directions(orc, shape):
    """bf16 r and p with the L1 term: the same image and objective bars as the float run."""
    from paper_2108_04315_b300 import binding as B
    P, plan, xt, y = l1_case(orc, "tiny_f2", 710, 0.05, iters=15, iterate_dtype=B.MISR_BF16, tile_shape=shape)
    y64 = y.astype(np.float64)
    xg, st = plan.solve(to_dev(y))
    xr, _ = P.scg(y64, P.shift_add(y64), 15)
    xg = xg.cpu().numpy().astype(np.float64)
    assert rel_l2(xg, xr) <= RTOL_X
    assert abs(P.objective(xg, y64) - P.objective(xr, y64)) <= 1e-4 * P.objective(xr, y64)


def test_l1_and_l2_in_one_batch_equal_each_alone(orc):
    """A batch of L1 and L2 problems (float and bf16 directions) runs one pass launch per
    kernel variant; each result equals its own solve bit for bit."""
    from paper_2108_04315_b300 import binding as B
    from tests.gpu_common import make_case
    psf = gen.gaussian_psf(5, 0.5)
    cases = [
        l1_case(orc, "ragged_f2_asym", 810, 0.02, iters=9),
        make_case(orc, 37, 53, 2, gen.half_pixel_shifts(), psf, seed=811, iters=11),
        l1_case(orc, "ragged_f3_k9", 812, 0.05, iters=7, iterate_dtype=B.MISR_BF16),
        make_case(orc, 23, 29, 3, gen.third_pixel_shifts(), psf, seed=813, iters=8, iterate_dtype=B.MISR_BF16),
    ]
    plans = [c[1] for c in cases]
    ys = [to_dev(c[3]) for c in cases]
    alone = []
    for plan, yd in zip(plans, ys):
        x, st = plan.solve(yd)
        alone.append((x.clone(), st))
    batch = B.Batch(plans)
    xs, stats = batch.solve(ys)
    for i, ((xa, sa), xb, sb) in enumerate(zip(alone, xs, stats)):
        assert torch.equal(xa, xb), f"problem {i}"
        assert sa == sb
    batch.close()


def test_l1_served_beside_l2_equals_alone(orc):
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts, psf = CASES["ragged_f2_asym"]
    P, plan, xt, y = l1_case(orc, "ragged_f2_asym", 910, 0.02, iters=12)
    yd = to_dev(y)
    x_alone, st_alone = plan.solve(yd)
    x_l2, st_l2 = B.Plan(h, w, f, shifts, psf, lam=0.01, iters=12).solve(yd)
    srv = B.Server(max_slots=4, passes_per_tick=3)
    t1 = srv.submit(yd, h, w, f, shifts, psf, lam=0.01, iters=12, data_norm=B.MISR_NORM_L1, data_eps=0.02)
    t2 = srv.submit(yd, h, w, f, shifts, psf, lam=0.01, iters=12)
    x1, s1, _ = srv.wait(t1, timeout_s=60.0)
    x2, s2, _ = srv.wait(t2, timeout_s=60.0)
    assert torch.equal(x1, x_alone) and s1 == st_alone
    assert torch.equal(x2, x_l2) and s2 == st_l2
    srv.close()


def test_l1_checkpoint_resume_and_norm_mismatch(orc):
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts, psf = CASES["ragged_f2_asym"]
    N, N1 = 12, 5
    P, full, xt, y = l1_case(orc, "ragged_f2_asym", 1010, 0.02, iters=N)
    yd = to_dev(y)
    x_full, st_full = full.solve(yd)
    kw = dict(lam=0.01, data_norm=B.MISR_NORM_L1, data_eps=0.02)
    short = B.Plan(h, w, f, shifts, psf, iters=N1, **kw)
    short.solve(yd)
    ck = short.export_state()
    cont = B.Plan(h, w, f, shifts, psf, iters=N, **kw)
    cont.import_state(ck)
    x_res, st_res = cont.resume(yd)
    assert torch.equal(x_res, x_full) and st_res == st_full
    l2 = B.Plan(h, w, f, shifts, psf, lam=0.01, iters=N)
    with pytest.raises(B.MisrError) as e:
        l2.import_state(ck)
    assert e.value.status == B.MISR_EINVAL


def test_l1_gradient_noalloc_equals_plan_gradient(orc):
    import ctypes as C
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts, psf = CASES["ragged_f3_k9"]
    P, plan, xt, y = l1_case(orc, "ragged_f3_k9", 1110, 0.02)
    yd, xd = to_dev(y), to_dev(xt.astype(np.float32))
    J_ref, g_ref = plan.gradient(yd, xd)
    fn = B.lib().misr_gradient_noalloc
    fn.argtypes = [C.POINTER(B.misr_desc), C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]
    fn.restype = C.c_int
    desc = B.make_desc(h, w, f, shifts, psf, lam=0.01, iters=1, data_norm=B.MISR_NORM_L1, data_eps=0.02)
    g = torch.full_like(xd, float("nan"))
    J = C.c_double()
    rc = fn(C.byref(desc), yd.data_ptr(), xd.data_ptr(), g.data_ptr(), C.byref(J),
            torch.cuda.current_stream().cuda_stream)
    assert rc == B.MISR_OK, B.misr_last_error()
    assert rel_l2(g.cpu().numpy(), g_ref.cpu().numpy()) <= RTOL_OP
    assert J.value == pytest.approx(J_ref, rel=RTOL_OP)


@pytest.mark.parametrize("eps_d", [1e-15, 1e15])
def test_l1_extreme_smoothing_stays_finite(orc, eps_d):
    """At the ends of the accepted range of eps_d (the L1 term's psi_d'' reaches 1/eps_d at a
    zero residual) the solve stays finite and never raises the objective beyond the FP32 noise
    of its direct sums (1e-6 of J; the accept test itself uses the per-pixel difference)."""
    P, plan, xt, y = l1_case(orc, "ragged_f2_asym", 1210, eps_d, iters=15)
    x, st = plan.solve(to_dev(y))
    tr = plan.trace()
    assert torch.isfinite(x).all() and np.isfinite(st["J_final"])
    E_next = np.where(tr["accept"] == 1, tr["J_trial"], tr["E"])
    E_all = np.concatenate([tr["E"][:1], E_next])
    assert np.all(np.isfinite(E_next)) and np.all(np.diff(E_all) <= 1e-6 * np.abs(E_all[:-1]))
    # at eps_d = 1e15 the L1 term is the L2 term over 2 eps_d: the objective at the device's
    # image is the oracle's
    if eps_d > 1:
        assert st["J_final"] == pytest.approx(P.objective(x.cpu().numpy().astype(np.float64), y.astype(np.float64)),
                                              rel=1e-5)
