"""The precision form: uint16 detector counts log-converted on the device, and r and p (the
gradient and the search direction) stored in bf16 while x stays the float master copy;
stencils accumulate in FP32 and the SCG scalars are FP64.  Both the float and the bf16-direction
solves are held to the same bars against the FP64 oracle (relative L2 of the image, relative
objective), on a 512 x 512 crop of the u16 workload."""
import numpy as np
import pytest

import gen
from tests.gpu_common import RTOL_J, RTOL_X, rel_l2, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

I0 = 40000.0


def _u16_case(orc, h, w, seed):
    f, sh, psf = 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)
    P = orc.Problem(h, w, f, sh, psf, lam=0.01)
    xt = gen.phantom(f * h, f * w, seed)
    counts = gen.poisson_counts(P.forward_all(xt), I0, seed + 1)
    return P, counts, orc.log_convert(counts, I0), (f, sh, psf)


def test_bf16_directions_match_oracle_on_u16_crop(orc):
    from paper_2108_04315_b300 import binding as B
    h = w = 512
    iters = 100
    P, counts, y64, (f, sh, psf) = _u16_case(orc, h, w, gen.CONFIG_SEEDS["precision"])
    xr, _ = P.scg(y64, P.shift_add(y64), iters)
    J_ref = P.objective(xr, y64)
    yd = to_dev(counts.view(np.int16))
    errs = {}
    for name, dt in (("f32", B.MISR_F32), ("bf16", B.MISR_BF16)):
        plan = B.Plan(h, w, f, sh, psf, lam=0.01, iters=iters, in_dtype=B.MISR_U16, flat_field=I0, iterate_dtype=dt)
        x, st = plan.solve(yd)
        xg = x.cpu().numpy().astype(np.float64)
        e_x = rel_l2(xg, xr)
        e_j = abs(P.objective(xg, y64) - J_ref) / J_ref
        errs[name] = (e_x, e_j)
        print(f"{name}: image rel L2 vs FP64 oracle {e_x:.2e}, objective rel {e_j:.2e}, "
              f"accepted {st['accepted']}/{st['iters_done']}")
        assert st["iters_done"] == iters
        assert e_x <= RTOL_X and e_j <= RTOL_J
        plan.close()


def test_bf16_gradient_is_the_float_gradient_rounded(orc):
    """misr_gradient of a bf16-direction plan returns r' as stored, i.e. the float gradient
    rounded to bf16 (relative error at most 2^-8 per value)."""
    from paper_2108_04315_b300 import binding as B
    P, counts, y64, (f, sh, psf) = _u16_case(orc, 64, 80, 811)
    yd = to_dev(counts.view(np.int16))
    x = to_dev(gen.phantom(128, 160, 812).astype(np.float32))
    grads = {}
    for name, dt in (("f32", B.MISR_F32), ("bf16", B.MISR_BF16)):
        plan = B.Plan(64, 80, f, sh, psf, lam=0.01, iters=1, in_dtype=B.MISR_U16, flat_field=I0, iterate_dtype=dt)
        J, g = plan.gradient(yd, x)
        grads[name] = (J, g.cpu().numpy())
        plan.close()
    gf, gb = grads["f32"][1], grads["bf16"][1]
    assert grads["f32"][0] == pytest.approx(grads["bf16"][0], rel=1e-6)
    rounded = torch.from_numpy(gf).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(gb, rounded)
    assert np.max(np.abs(gb - gf) / np.maximum(np.abs(gf), 1e-30)) <= 2.0 ** -8


def test_batch_mixes_float_and_bf16_directions(orc):
    from paper_2108_04315_b300 import binding as B
    cases = []
    for i, dt in enumerate((B.MISR_F32, B.MISR_BF16, B.MISR_BF16)):
        P, counts, y64, (f, sh, psf) = _u16_case(orc, 40 + 8 * i, 56, 900 + i)
        plan = B.Plan(40 + 8 * i, 56, f, sh, psf, lam=0.01, iters=15, in_dtype=B.MISR_U16, flat_field=I0,
                      iterate_dtype=dt)
        cases.append((plan, to_dev(counts.view(np.int16))))
    alone = [p.solve(y)[0].clone() for p, y in cases]
    batch = B.Batch([p for p, _ in cases])
    xs, _ = batch.solve([y for _, y in cases])
    for a, b in zip(alone, xs):
        assert torch.equal(a, b)
    batch.close()


def test_probe_rejects_bf16_plans():
    from paper_2108_04315_b300 import binding as B
    plan = B.Plan(16, 16, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5), iters=1, iterate_dtype=B.MISR_BF16)
    z = torch.zeros((32, 32), dtype=torch.float32, device="cuda")
    y = torch.zeros((4, 16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(B.MisrError) as e:
        plan.pass_probe(y, z, z, z, 0.1, 0.0)
    assert e.value.status == B.MISR_ENOTIMPL
