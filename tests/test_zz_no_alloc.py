"""The allocation-free gradient entry point (misr_gradient_noalloc) against the plan-based
misr_gradient, through the C ABI.

misr_gradient_noalloc serves callers that cannot allocate device memory (their memory is
reserved by another allocator, or cudaMalloc's implicit synchronisation is not acceptable in
their acquisition loop): its workspace is a fixed array inside the library.  Two calls in a
row on different problems check that the shared array is set up and cleared correctly.
This file is collected last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes as C

import numpy as np
import pytest

import gen
from tests.gpu_common import RTOL_OP, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _noalloc_fn():
    from paper_2108_04315_b300 import binding as B
    L = B.lib()
    fn = L.misr_gradient_noalloc
    fn.argtypes = [C.POINTER(B.misr_desc), C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]
    fn.restype = C.c_int
    return B, fn


def test_gradient_noalloc_matches_plan_gradient_on_two_calls():
    B, fn = _noalloc_fn()
    cases = [
        (64, 64, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5), 31),   # 128 x 128 HR
        (37, 45, 3, gen.third_pixel_shifts(), gen.gaussian_psf(5, 0.7), 32),  # 111 x 135 HR, ragged
    ]
    stream = torch.cuda.current_stream()
    for h, w, f, shifts, psf, seed in cases:
        K = len(shifts)
        y = torch.from_numpy(gen.random_field((K, h, w), seed, 0.0, 2.0).astype(np.float32)).cuda()
        x = torch.from_numpy((gen.phantom(f * h, f * w, seed + 1) +
                              gen.random_field((f * h, f * w), seed + 2, -0.1, 0.1)).astype(np.float32)).cuda()
        plan = B.Plan(h, w, f, shifts, psf, lam=0.01, iters=1)
        J_ref, g_ref = plan.gradient(y, x)
        desc = B.make_desc(h, w, f, shifts, psf, lam=0.01, iters=1)
        g = torch.full_like(x, float("nan"))
        J = C.c_double()
        rc = fn(C.byref(desc), y.data_ptr(), x.data_ptr(), g.data_ptr(), C.byref(J), stream.cuda_stream)
        assert rc == B.MISR_OK, B.misr_last_error()
        assert rel_l2(g.cpu().numpy(), g_ref.cpu().numpy()) <= RTOL_OP
        assert J.value == pytest.approx(J_ref, rel=RTOL_OP)
        plan.close()


def test_gradient_noalloc_rejects_images_above_its_limit():
    B, fn = _noalloc_fn()
    desc = B.make_desc(300, 200, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5))   # 600 x 400 HR
    x = torch.zeros((600, 400), device="cuda")
    y = torch.zeros((4, 300, 200), device="cuda")
    g = torch.zeros_like(x)
    rc = fn(C.byref(desc), y.data_ptr(), x.data_ptr(), g.data_ptr(), None, 0)
    assert rc == B.MISR_EINVAL
    assert "512" in B.misr_last_error()
