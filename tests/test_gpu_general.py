"""The frame-wise pass: frame sets that do not interleave into one HR image (several frames on
one HR phase, such as the synthetic study's one-pixel shifts right, down, left and up, Sec.
4.1.1; shifts outside [0, 1) LR px, negative or beyond a pixel; non-integer shifts off a product
lattice; K above f^2; binning whose combined blur is wider than the fused passes' taps).  The
library builds per-frame, per-row tap tables of D B M_k on the host and gathers them on the
device; the FP64 oracle applies M_k, B and D literally, so the two share no arithmetic.  Same
bars as the fused passes: forward and gradient at 1e-5, the pass's sums at 1e-5 (L1: the bars
of tests/test_gpu_l1.py), solves at 1e-3 on the image and 1e-5 on the objective, decisions
where the objective change is above the FP32 noise floor."""
import numpy as np
import pytest

import gen
from tests.gpu_common import (GENERAL_CASES, GENERAL_L2_ITERS, GENERAL_PAPER_ITERS, GENERAL_SEED, PAPER_SETTING,
                              RTOL_J, RTOL_OP, RTOL_X, general_case, rel_l2, to_dev)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U = 2.0 ** -24


def _close(a, ref, tol):
    """rel_l2 within tol, or (a frame that sees no pixel of the grid) both zero"""
    if not np.any(ref):
        return float(np.abs(a).max()) <= 1e-30
    return rel_l2(a, ref) <= tol


@pytest.mark.parametrize("name", sorted(GENERAL_CASES))
def test_general_forward_operator(orc, name):
    P, plan, xt, _ = general_case(orc, name, 100)
    x = (xt + gen.random_field(xt.shape, 7, -0.5, 0.5)).astype(np.float32)
    y = plan.forward(to_dev(x)).cpu().numpy()
    ref = P.forward_all(x.astype(np.float64))
    for k in range(P.K):
        assert _close(y[k], ref[k], RTOL_OP), (name, k)
    plan.close()


@pytest.mark.parametrize("name", sorted(GENERAL_CASES))
@pytest.mark.parametrize("l1_eps", [None, 0.05])
def test_general_objective_and_gradient(orc, name, l1_eps):
    P, plan, xt, y = general_case(orc, name, 200, l1_eps=l1_eps)
    x = (xt + gen.random_field(xt.shape, 8, -0.2, 0.2)).astype(np.float32)
    J, g = plan.gradient(to_dev(y), to_dev(x))
    Jr, gr = P.gradient(x.astype(np.float64), y.astype(np.float64))
    tol = RTOL_OP + (16 * U * float(np.abs(y).max()) / l1_eps if l1_eps else 0.0)
    assert J == pytest.approx(Jr, rel=RTOL_J)
    assert rel_l2(g.cpu().numpy(), gr) <= tol
    plan.close()


@pytest.mark.parametrize("name", ["study_bin_psf3", "dup_phase_k6", "neg_large", "off_lattice", "wide_bin_f3",
                                  "far_shifts", "thin_strip"])
@pytest.mark.parametrize("l1_eps", [None, 0.05])
def test_general_pass(orc, name, l1_eps):
    """One frame-wise pass: p, x', r' and the ten sums, curvature forms included."""
    alpha, beta = 0.3, 0.7
    P, plan, xt, y = general_case(orc, name, 300, l1_eps=l1_eps)
    x = (xt + gen.random_field(xt.shape, 9, -0.1, 0.1)).astype(np.float32)
    r = gen.random_field(xt.shape, 10, -0.3, 0.3).astype(np.float32)
    po = gen.random_field(xt.shape, 11, -0.3, 0.3).astype(np.float32)
    xo, ro, pn, S = plan.pass_probe(to_dev(y), to_dev(x), to_dev(r), to_dev(po), alpha, beta)
    xo, ro, pn = (t.cpu().numpy().astype(np.float64) for t in (xo, ro, pn))
    x64, r64, po64, y64 = (a.astype(np.float64) for a in (x, r, po, y))
    assert rel_l2(pn, r64 + beta * po64) <= 1e-6
    assert rel_l2(xo, x64 + alpha * pn) <= 1e-6
    h, w, f, shifts, psf, dec = GENERAL_CASES[name]
    kw = dict(data_norm=orc.NORM_L1, data_eps=l1_eps) if l1_eps else {}
    P0 = orc.Problem(h, w, f, shifts, psf, lam=0.0, decimation=dec, **kw)
    tol = RTOL_OP + (16 * U * float(np.abs(y).max()) / l1_eps if l1_eps else 0.0)
    J, g = P.gradient(xo, y64)
    r_ref = -g
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
    scale = {"dJ_data": abs(ref["J_data"]) * 1e-7, "b": np.sqrt(abs(ref["a"] * ref["c"])) * tol,
             "rr_cross": np.sqrt(ref["rr"] * np.sum(r64 * r64)) * tol, "pr": np.sqrt(ref["rr"] * ref["pp"]) * tol}
    for k, v in ref.items():
        rt = 2 * tol if k in ("rr", "pr", "a", "b", "c") else RTOL_OP
        assert abs(S[k] - v) <= rt * abs(v) + scale.get(k, 0.0) + 1e-30, (k, S[k], v)
    plan.close()


def _solve_vs_oracle(orc, name, iters, lam, l1_eps):
    P, plan, xt, y = general_case(orc, name, GENERAL_SEED, lam=lam, l1_eps=l1_eps, iters=iters)
    y64 = y.astype(np.float64)
    xg, st = plan.solve(to_dev(y))
    xr, tr = P.scg(y64, P.shift_add(y64), iters)
    assert st["iters_done"] == iters
    assert rel_l2(xg.cpu().numpy(), xr) <= RTOL_X
    assert st["J_final"] == pytest.approx(P.objective(xr, y64), rel=RTOL_J)
    tg = plan.trace()
    sig = np.abs(tr["E"] - tr["J_trial"]) > 1e-6 * np.abs(tr["E"])
    assert np.array_equal(tg["accept"][sig], tr["accept"][sig])
    plan.close()


@pytest.mark.parametrize("name", sorted(GENERAL_PAPER_ITERS))
def test_general_solve_paper_setting(orc, name):
    """The paper's setting (L1 data term, lambda 0.05, alpha 0.4, 20 iterations) against the
    oracle's SCG from the same shift-and-add start point."""
    _solve_vs_oracle(orc, name, GENERAL_PAPER_ITERS[name], PAPER_SETTING["lam"], PAPER_SETTING["l1_eps"])


@pytest.mark.parametrize("name", sorted(GENERAL_L2_ITERS))
def test_general_solve_l2(orc, name):
    _solve_vs_oracle(orc, name, GENERAL_L2_ITERS[name], 0.01, None)


@pytest.mark.parametrize("name", sorted(GENERAL_CASES))
def test_general_start_point(orc, name):
    """Multi-image interpolation: every sample placed (bilinearly for non-integer shifts) where
    it was taken, several samples of one pixel averaged, 0 where none falls; and a solve of 0
    iterations returns it."""
    from paper_2108_04315_b300 import binding as B
    P, plan, xt, y = general_case(orc, name, 500, iters=0)
    ref = P.shift_add(y.astype(np.float64))
    x0 = plan.interpolate(to_dev(y)).cpu().numpy()
    # a weighted mean of at most 4 K samples: (4 K + 8) rounding errors of max |y| at most
    assert float(np.abs(x0 - ref).max()) <= (4 * P.K + 8) * U * float(np.abs(y).max())
    xs, st = plan.solve(to_dev(y))
    assert st["iters_done"] == 0
    assert torch.equal(xs.cpu(), torch.from_numpy(x0))
    plan.close()
    assert B.MISR_TILE_AUTO == 0


def test_general_u16_counts(orc):
    """u16 detector counts on the synthetic study's geometry: converted on the device, then the
    gradient against the oracle's log conversion."""
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts, psf, dec = GENERAL_CASES["study_bin_psf3"]
    P = orc.Problem(h, w, f, shifts, psf, lam=0.01, decimation=dec)
    xt = gen.phantom(f * h, f * w, 600)
    counts = gen.poisson_counts(P.forward_all(xt), 40000.0, 601)
    y = orc.log_convert(counts, 40000.0)
    plan = B.Plan(h, w, f, shifts, psf, lam=0.01, iters=5, decimation=dec, in_dtype=B.MISR_U16, flat_field=40000.0)
    x = (xt + gen.random_field(xt.shape, 8, -0.2, 0.2)).astype(np.float32)
    J, g = plan.gradient(to_dev(counts.astype(np.uint16).view(np.int16)), to_dev(x))
    Jr, gr = P.gradient(x.astype(np.float64), y)
    assert J == pytest.approx(Jr, rel=RTOL_J)
    assert rel_l2(g.cpu().numpy(), gr) <= RTOL_OP
    plan.close()


def test_general_and_fused_in_one_batch_equal_each_alone(orc):
    from paper_2108_04315_b300 import binding as B
    from tests.gpu_common import make_case
    cases = [general_case(orc, "study_bin_psf3", 610, iters=8),
             make_case(orc, 40, 52, 2, gen.half_pixel_shifts(), gen.gaussian_psf(3, 0.6), seed=611, iters=9),
             general_case(orc, "off_lattice", 612, iters=7, l1_eps=0.05),
             make_case(orc, 37, 45, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5), seed=613, iters=6,
                       tile_shape=B.MISR_TILE_STREAM)]
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


def test_general_served_equals_alone(orc):
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts, psf, dec = GENERAL_CASES["study_bin_psf3"]
    P, plan, xt, y = general_case(orc, "study_bin_psf3", 620, iters=9)
    yd = to_dev(y)
    x_alone, st_alone = plan.solve(yd)
    x_alone = x_alone.clone()
    srv = B.Server(max_slots=4, passes_per_tick=2)
    tickets = [srv.submit(yd, h, w, f, shifts, psf, iters=9, decimation=dec) for _ in range(3)]
    for t in tickets:
        x, st, times = srv.wait(t, timeout_s=60.0)
        assert torch.equal(x, x_alone) and st == st_alone
    srv.close()
    plan.close()


def test_general_resume_equals_uninterrupted(orc):
    from paper_2108_04315_b300 import binding as B
    N, N1 = 12, 5
    h, w, f, shifts, psf, dec = GENERAL_CASES["dup_phase_k6"]
    P, full, xt, y = general_case(orc, "dup_phase_k6", 630, iters=N)
    yd = to_dev(y)
    x_full, st_full = full.solve(yd)
    short = B.Plan(h, w, f, shifts, psf, iters=N1, decimation=dec)
    short.solve(yd)
    ck = short.export_state()
    cont = B.Plan(h, w, f, shifts, psf, iters=N, decimation=dec)
    cont.import_state(ck)
    x_res, st_res = cont.resume(yd)
    assert torch.equal(x_res, x_full) and st_res == st_full
    for p in (full, short, cont):
        p.close()


def test_general_refusals(orc):
    """bf16 directions and the allocation-free gradient are not offered for these geometries:
    refused with MISR_ENOTIMPL before any device work."""
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts, psf, dec = GENERAL_CASES["study_bin_psf3"]
    with pytest.raises(B.MisrError) as e:
        B.Plan(h, w, f, shifts, psf, decimation=dec, iterate_dtype=B.MISR_BF16)
    assert e.value.status == B.MISR_ENOTIMPL
    P, plan, xt, y = general_case(orc, "study_bin_psf3", 640)
    desc = B.make_desc(h, w, f, shifts, psf, decimation=dec)
    g = torch.empty((f * h, f * w), dtype=torch.float32, device="cuda")
    with pytest.raises(B.MisrError) as e:
        B.misr_gradient_noalloc(desc, to_dev(y).data_ptr(), to_dev(xt.astype(np.float32)).data_ptr(), g.data_ptr())
    assert e.value.status == B.MISR_ENOTIMPL
    plan.close()


def test_general_checkpoint_refused_on_another_model(orc):
    """A frame-wise checkpoint resumes only on a plan of the same model: another PSF, another
    fractional shift, point sampling instead of binning, or the fused passes' geometry refuse it
    with MISR_EINVAL."""
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts, psf, dec = GENERAL_CASES["study_bin_psf3"]
    P, plan, xt, y = general_case(orc, "study_bin_psf3", 650, iters=3)
    plan.solve(to_dev(y))
    ck = plan.export_state()
    others = [B.Plan(h, w, f, shifts, gen.gaussian_psf(3, 0.9), iters=5, decimation=dec),
              B.Plan(h, w, f, [(0.5, 0.0), (0.0, 0.5), (-0.5, 0.0), (0.0, -0.45)], psf, iters=5, decimation=dec),
              B.Plan(h, w, f, shifts, psf, iters=5),
              B.Plan(h, w, f, gen.half_pixel_shifts(), psf, iters=5, decimation=dec)]
    for o in others:
        with pytest.raises(B.MisrError) as e:
            o.import_state(ck)
        assert e.value.status == B.MISR_EINVAL
        o.close()
    same = B.Plan(h, w, f, shifts, psf, iters=5, decimation=dec)
    same.import_state(ck)
    same.close()
    plan.close()
