"""Multi-image interpolation (misr_interpolate, Sec. 4.1.1): the paper's non-iterative
comparator, each LR sample inserted at the HR pixel it was taken at and 0 where no frame
samples.  With one frame per HR phase no pixel gets two samples, so float frames are copied
and the image must equal the FP64 oracle's shift-and-add rounded to float32 bit for bit; u16
counts go through the device's FP32 log conversion (relative error a few FP32 ulps)."""
import numpy as np
import pytest

import gen
from tests.gpu_common import asym_separable_psf, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    # name: (h, w, f, shifts)
    "tiny_f2": (64, 64, 2, gen.half_pixel_shifts()),
    "ragged_f3_k9": (23, 29, 3, gen.third_pixel_shifts()),
    "partial_f2_k3": (30, 41, 2, [(0.0, 0.0), (0.5, 0.0), (0.5, 0.5)]),
    "f1": (45, 70, 1, [(0.0, 0.0)]),
    "f4_k16": (17, 21, 4, gen.phase_shifts(4)),
    "odd_width": (13, 7, 2, gen.half_pixel_shifts()),       # W = 14: scalar stores
    "single_pixel": (1, 1, 2, gen.half_pixel_shifts()),
    "f8_k5": (3, 5, 8, [(0.0, 0.0), (0.125, 0.0), (0.5, 0.25), (0.875, 0.875), (0.25, 0.625)]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_interpolation_equals_oracle_bitwise(orc, name):
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts = CASES[name]
    psf = gen.gaussian_psf(5, 0.5)
    P = orc.Problem(h, w, f, shifts, psf)
    y = gen.random_field((len(shifts), h, w), 40, -1.0, 3.0).astype(np.float32)
    plan = B.Plan(h, w, f, shifts, psf, iters=1)
    x = torch.full((f * h, f * w), float("nan"), device="cuda")
    plan.interpolate(to_dev(y), x)
    ref = P.shift_add(y.astype(np.float64)).astype(np.float32)
    assert np.array_equal(x.cpu().numpy(), ref)
    plan.close()


def test_interpolation_of_u16_counts(orc):
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts = 48, 40, 2, gen.half_pixel_shifts()
    psf = gen.gaussian_psf(5, 0.5)
    P = orc.Problem(h, w, f, shifts, psf)
    counts = gen.poisson_counts(P.forward_all(gen.phantom(f * h, f * w, 41)), 40000.0, 42)
    counts[0, 0, :3] = 0                                    # clamped to 1 before the log
    plan = B.Plan(h, w, f, shifts, psf, iters=1, in_dtype=B.MISR_U16, flat_field=40000.0)
    x = plan.interpolate(to_dev(counts.view(np.int16))).cpu().numpy().astype(np.float64)
    ref = P.shift_add(orc.log_convert(counts, 40000.0))
    np.testing.assert_allclose(x, ref, rtol=4e-7, atol=4e-6)


def test_interpolation_is_the_solve_start_point(orc):
    """A zero-iteration MISR_X0_SHIFT_ADD solve returns the interpolated image, and the call
    leaves a plan's solve state alone (a later resume-free solve is unchanged)."""
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts = CASES["ragged_f3_k9"]
    psf = asym_separable_psf(5)
    y = to_dev(gen.random_field((len(shifts), h, w), 43, 0.0, 2.0).astype(np.float32))
    p0 = B.Plan(h, w, f, shifts, psf, iters=0)
    x0, _ = p0.solve(y)
    assert torch.equal(p0.interpolate(y), x0)
    p5 = B.Plan(h, w, f, shifts, psf, iters=5)
    a, sa = p5.solve(y)
    p5.interpolate(y)
    b, sb = p5.solve(y)
    assert torch.equal(a, b) and sa == sb


def test_interpolation_into_an_unaligned_buffer(orc):
    """An output pointer off the 16-byte grid takes the scalar stores."""
    from paper_2108_04315_b300 import binding as B
    h, w, f, shifts = CASES["tiny_f2"]
    psf = gen.gaussian_psf(5, 0.5)
    P = orc.Problem(h, w, f, shifts, psf)
    y = gen.random_field((len(shifts), h, w), 44, -1.0, 3.0).astype(np.float32)
    plan = B.Plan(h, w, f, shifts, psf, iters=1)
    buf = torch.full((f * h * f * w + 1,), float("nan"), device="cuda")
    x = buf[1:].view(f * h, f * w)                       # 4 bytes past a 256-byte boundary
    plan.interpolate(to_dev(y), x)
    ref = P.shift_add(y.astype(np.float64)).astype(np.float32)
    assert np.array_equal(x.cpu().numpy(), ref)
    assert torch.isnan(buf[0])
