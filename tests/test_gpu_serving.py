"""Serving (misr_server_*, misr_submit, misr_poll): projections submitted while others are on
the GPU join the next fused-pass launch.  Each keeps its own state and fixed-order reductions,
so its image and statistics must equal its own misr_solve bit for bit whatever it shared the
GPU with; admission respects the HBM budget; malformed requests fail with a status."""
import time

import numpy as np
import pytest

import gen
from tests.gpu_common import RTOL_X, make_case, rel_l2, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PSF = gen.gaussian_psf(5, 0.5)
GEOMS = [
    # (h, w, f, shifts, iters)
    (64, 64, 2, gen.half_pixel_shifts(), 20),
    (37, 53, 2, gen.half_pixel_shifts(), 12),
    (23, 29, 3, gen.third_pixel_shifts(), 16),
]


def _cases(orc):
    return [make_case(orc, h, w, f, sh, PSF, seed=2000 + i, iters=it) for i, (h, w, f, sh, it) in enumerate(GEOMS)]


def test_serving_mix_equals_alone_and_oracle(orc):
    from paper_2108_04315_b300 import binding as B
    cases = _cases(orc)
    ys = [to_dev(c[3]) for c in cases]
    alone = []
    for (P, plan, xt, y), yd in zip(cases, ys):
        x, st = plan.solve(yd)
        alone.append((x.clone(), st))
    srv = B.Server(max_slots=8, passes_per_tick=3)
    # a stream of requests over three geometry classes, arriving while earlier ones run; every
    # other one submitted with its class's descriptor made once (submit_desc)
    descs = [B.make_desc(h, w, f, sh, PSF, iters=it) for h, w, f, sh, it in GEOMS]
    order = [0, 1, 2, 0, 0, 2, 1, 0, 2]
    tickets = []
    for n, i in enumerate(order):
        h, w, f, sh, it = GEOMS[i]
        if n % 2:
            tickets.append((i, srv.submit_desc(ys[i], descs[i])))
        else:
            tickets.append((i, srv.submit(ys[i], h, w, f, sh, PSF, iters=it)))
        if n % 3 == 2:
            time.sleep(0.002)
    for i, t in tickets:
        x, st, times = srv.wait(t, timeout_s=60.0)
        assert torch.equal(x, alone[i][0]), f"class {i}: served image differs from misr_solve"
        assert st == alone[i][1]
        assert st["iters_done"] == GEOMS[i][4]
        assert times[0] <= times[1] <= times[2]
    c = srv.counters()
    assert c["queued"] == 0 and c["running"] == 0 and 1 <= c["slots"] <= 8 and c["passes_launched"] > 0
    # the served result also matches the FP64 oracle
    P, plan, xt, y = cases[0]
    y64 = y.astype(np.float64)
    xr, _ = P.scg(y64, P.shift_add(y64), GEOMS[0][4])
    assert rel_l2(alone[0][0].cpu().numpy(), xr) <= RTOL_X
    srv.close()


def test_serving_respects_hbm_budget(orc):
    from paper_2108_04315_b300 import binding as B
    (P, plan, xt, y) = _cases(orc)[0]
    yd = to_dev(y)
    h, w, f, sh, it = GEOMS[0]
    x_alone, st_alone = plan.solve(yd)
    probe = B.Server(max_slots=4)
    probe.wait(probe.submit(yd, h, w, f, sh, PSF, iters=it))
    one_slot = probe.counters()["slot_bytes"]
    probe.close()
    assert one_slot > 0
    srv = B.Server(max_slots=4, passes_per_tick=2, hbm_budget_bytes=int(one_slot * 1.5))
    tickets = [srv.submit(yd, h, w, f, sh, PSF, iters=it) for _ in range(4)]
    peak = 0
    for t in tickets:
        while True:
            peak = max(peak, srv.counters()["slots"])
            r = srv.poll(t)
            if r is not None:
                break
            time.sleep(0.0005)
        assert torch.equal(r[0], x_alone) and r[1] == st_alone
    assert peak == 1 and srv.counters()["slot_bytes"] == one_slot
    # a projection larger than the whole budget fails instead of waiting forever
    big = torch.zeros((4, 256, 256), dtype=torch.float32, device="cuda")
    t = srv.submit(big, 256, 256, 2, gen.half_pixel_shifts(), PSF, iters=2)
    with pytest.raises(B.MisrError) as e:
        srv.wait(t, timeout_s=60.0)
    assert e.value.status == B.MISR_ENOMEM
    srv.close()


def test_serving_errors_and_timeouts():
    from paper_2108_04315_b300 import binding as B
    srv = B.Server(max_slots=2, passes_per_tick=1)
    y = torch.zeros((4, 32, 32), dtype=torch.float32, device="cuda")
    with pytest.raises(B.MisrError) as e:   # frames off a product lattice (frame-wise pass) with bf16 r, p
        srv.submit(y, 32, 32, 2, [(0, 0), (0.6, 0), (0, 0.5), (0.55, 0.5)], gen.gaussian_psf(3, 0.5),
                   iterate_dtype=B.MISR_BF16)
    assert e.value.status == B.MISR_ENOTIMPL
    with pytest.raises(B.MisrError) as e:   # a shift that is not finite
        srv.submit(y, 32, 32, 2, [(0, 0), (0, float("nan")), (0, 0.5), (0.5, 0.5)], PSF)
    assert e.value.status == B.MISR_EINVAL
    with pytest.raises(B.MisrError) as e:   # even PSF size
        srv.submit(y, 32, 32, 2, gen.half_pixel_shifts(), np.full((4, 4), 1 / 16.0), iters=1)
    assert e.value.status == B.MISR_EINVAL
    with pytest.raises(B.MisrError) as e:
        B.misr_poll(srv.handle, 12345)
    assert e.value.status == B.MISR_EINVAL
    with pytest.raises(B.MisrError) as e:
        B.misr_server_wait(srv.handle, 12345, 0.0)
    assert e.value.status == B.MISR_EINVAL
    with pytest.raises(B.MisrError):
        B.Server(max_slots=0)
    # a long solve is not finished after 0 s, then finishes
    yl = torch.rand((4, 256, 256), dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    t = srv.submit(yl, 256, 256, 2, gen.half_pixel_shifts(), PSF, iters=3000)
    with pytest.raises(B.MisrError) as e:
        B.misr_server_wait(srv.handle, t, 0.0)
    assert e.value.status == B.MISR_ETIMEOUT
    x, st, _ = srv.wait(t, timeout_s=120.0)
    assert st["iters_done"] >= 1 and np.isfinite(st["J_final"])
    with pytest.raises(B.MisrError):   # forgotten once reported
        B.misr_poll(srv.handle, t)
    srv.close()


def test_serving_destroy_with_requests_in_flight():
    from paper_2108_04315_b300 import binding as B
    srv = B.Server(max_slots=2, passes_per_tick=2)
    y = torch.rand((4, 128, 128), dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(9))
    for _ in range(5):
        srv.submit(y, 128, 128, 2, gen.half_pixel_shifts(), PSF, iters=500)
    time.sleep(0.01)
    srv.close()
    torch.cuda.synchronize()


def test_serving_cancel_queued_and_running(orc):
    from paper_2108_04315_b300 import binding as B
    (P, plan, xt, y) = _cases(orc)[0]
    yd = to_dev(y)
    h, w, f, sh, it = GEOMS[0]
    x_alone, st_alone = plan.solve(yd)
    srv = B.Server(max_slots=1, passes_per_tick=2)
    yl = torch.rand((4, 256, 256), dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(11))
    t_long = srv.submit(yl, 256, 256, 2, gen.half_pixel_shifts(), PSF, iters=5000)   # runs, long
    t_queued = srv.submit(yd, h, w, f, sh, PSF, iters=it)                          # waits for the slot
    srv.cancel(t_queued)
    with pytest.raises(B.MisrError) as e:
        srv.wait(t_queued, timeout_s=60.0)
    assert e.value.status == B.MISR_ECANCELED
    srv.cancel(t_long)
    with pytest.raises(B.MisrError) as e:
        srv.wait(t_long, timeout_s=120.0)
    assert e.value.status == B.MISR_ECANCELED
    with pytest.raises(B.MisrError) as e:        # forgotten once reported
        B.misr_poll(srv.handle, t_long)
    assert e.value.status == B.MISR_EINVAL
    # the server keeps serving, and a request after the cancellations gets its own solve's result
    t = srv.submit(yd, h, w, f, sh, PSF, iters=it)
    x, st, _ = srv.wait(t, timeout_s=60.0)
    assert torch.equal(x, x_alone) and st == st_alone
    # cancelling a finished (already reported) or unknown ticket
    with pytest.raises(B.MisrError) as e:
        srv.cancel(t)
    assert e.value.status == B.MISR_EINVAL
    c = srv.counters()
    assert c["queued"] == 0 and c["running"] == 0
    srv.close()


def test_serving_mixes_model_options(orc):
    """Requests with the L1 term, binning D and non-integer shifts served beside a plain one
    (different kernel variants in one tick): each equals its own misr_solve bit for bit."""
    from paper_2108_04315_b300 import binding as B
    h, w, f = 37, 53, 2
    psf3 = gen.gaussian_psf(3, 0.6)
    frac = [(dx, dy) for dy in (0.05, 0.6) for dx in (0.0, 0.55)]
    kinds = [
        (gen.half_pixel_shifts(), PSF, dict()),
        (gen.half_pixel_shifts(), psf3, dict(data_norm=B.MISR_NORM_L1, data_eps=0.02, decimation=B.MISR_DECIM_BIN)),
        (frac, psf3, dict()),
        (frac, psf3, dict(data_norm=B.MISR_NORM_L1, data_eps=0.05, iterate_dtype=B.MISR_BF16)),
    ]
    y = to_dev(gen.random_field((4, h, w), 2100, 0.0, 2.0).astype(np.float32))
    alone = []
    for sh, psf, kw in kinds:
        x, st = B.Plan(h, w, f, sh, psf, lam=0.01, iters=9, **kw).solve(y)
        alone.append((x.clone(), st))
    srv = B.Server(max_slots=8, passes_per_tick=2)
    tickets = [srv.submit(y, h, w, f, sh, psf, lam=0.01, iters=9, **kw) for sh, psf, kw in kinds]
    for t, (xa, sa) in zip(tickets, alone):
        x, st, _ = srv.wait(t, timeout_s=60.0)
        assert torch.equal(x, xa) and st == sa
    srv.close()


def test_serving_streaming_shape_equals_alone(orc):
    """Requests on the row-streaming shape, served alone (a tick of one slot reduces its sums in
    the pass) and in a burst (a tick of several launches reduces in the reduction kernel), with
    the L1 term and bf16 directions among them: each result equals its own misr_solve (which
    reduces in the pass) bit for bit."""
    from paper_2108_04315_b300 import binding as B
    geoms = [(64, 64, 2, gen.half_pixel_shifts(), {}), (40, 120, 2, gen.half_pixel_shifts(), {}),
             (23, 29, 3, gen.third_pixel_shifts(), {}),
             (48, 64, 2, gen.half_pixel_shifts(), dict(data_norm=B.MISR_NORM_L1, data_eps=0.05)),
             (48, 72, 2, gen.half_pixel_shifts(), dict(iterate_dtype=B.MISR_BF16))]
    ys, alone = [], []
    for i, (h, w, f, sh, kw) in enumerate(geoms):
        P, plan, xt, y = make_case(orc, h, w, f, sh, PSF, seed=2600 + i, iters=12, tile_shape=4, **kw)
        yd = to_dev(y)
        x, st = plan.solve(yd)
        ys.append(yd)
        alone.append((x.clone(), st))
        plan.close()
    srv = B.Server(max_slots=8, passes_per_tick=4)

    def submit(i):
        h, w, f, sh, kw = geoms[i]
        return srv.submit(ys[i], h, w, f, sh, PSF, iters=12, tile_shape=4, **kw)

    def check(i, t):
        x, st, _ = srv.wait(t, timeout_s=60.0)
        assert torch.equal(x, alone[i][0]), f"request {i}: served image differs from misr_solve"
        assert st == alone[i][1]

    check(0, submit(0))                                   # alone
    burst = [(i, submit(i)) for i in (1, 2, 3, 4, 0, 3)]  # several slots per tick
    for i, t in burst:
        check(i, t)
    check(4, submit(4))                                   # alone again, a warm slot
    srv.close()


def test_serving_idle_poll_equals_alone_and_stops(orc):
    """A worker that polls for requests when idle (idle_spin_us): results equal the projection's
    own solve, whether a request comes while it polls or after it has gone to sleep, and the
    server stops at once while it polls."""
    from paper_2108_04315_b300 import binding as B
    (P, plan, xt, y) = _cases(orc)[1]
    yd = to_dev(y)
    h, w, f, sh, it = GEOMS[1]
    x_alone, st_alone = plan.solve(yd)
    srv = B.Server(max_slots=2, passes_per_tick=2, idle_spin_us=1000000)
    desc = B.make_desc(h, w, f, sh, PSF, iters=it)
    for pause in (0.0, 0.02, 1.2):   # during the poll, during it, after it
        time.sleep(pause)
        x, st, times = srv.wait(srv.submit_desc(yd, desc), timeout_s=60.0)
        assert torch.equal(x, x_alone) and st == st_alone
    srv.submit_desc(yd, desc)
    time.sleep(0.05)
    t0 = time.monotonic()
    srv.close()
    assert time.monotonic() - t0 < 0.5   # a poll left to run out would hold it about 0.95 s
    with pytest.raises(B.MisrError) as e:
        B.Server(max_slots=2, idle_spin_us=-1)
    assert e.value.status == B.MISR_EINVAL
