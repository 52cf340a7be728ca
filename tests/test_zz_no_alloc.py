"""The allocation-free gradient entry point (misr_gradient_noalloc) through the C ABI: against
the plan-based misr_gradient and against the FP64 oracle, its size limit and FP32-only
refusal, and its timeout path.

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

CASES = [
    (64, 64, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5), 31),   # 128 x 128 HR
    (37, 45, 3, gen.third_pixel_shifts(), gen.gaussian_psf(5, 0.7), 32),  # 111 x 135 HR, ragged
]


def _noalloc_fn():
    from paper_2108_04315_b300 import binding as B
    L = B.lib()
    fn = L.misr_gradient_noalloc
    fn.argtypes = [C.POINTER(B.misr_desc), C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]
    fn.restype = C.c_int
    return B, fn


def _inputs(h, w, f, shifts, seed):
    K = len(shifts)
    y = gen.random_field((K, h, w), seed, 0.0, 2.0).astype(np.float32)
    x = (gen.phantom(f * h, f * w, seed + 1) + gen.random_field((f * h, f * w), seed + 2, -0.1, 0.1)).astype(np.float32)
    return y, x


def test_gradient_noalloc_matches_plan_gradient_on_two_calls():
    B, fn = _noalloc_fn()
    stream = torch.cuda.current_stream()
    for h, w, f, shifts, psf, seed in CASES:
        y, x = (torch.from_numpy(a).cuda() for a in _inputs(h, w, f, shifts, seed))
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


def test_gradient_noalloc_matches_the_oracle(orc):
    """J(x) (Eq. 9) and grad J(x) of the allocation-free call against the FP64 oracle directly,
    on the same two geometries, two calls in a row."""
    B, fn = _noalloc_fn()
    for h, w, f, shifts, psf, seed in CASES:
        y, x = _inputs(h, w, f, shifts, seed)
        P = orc.Problem(h, w, f, shifts, psf, lam=0.01)
        Jr, gr = P.gradient(x.astype(np.float64), y.astype(np.float64))
        desc = B.make_desc(h, w, f, shifts, psf, lam=0.01, iters=1)
        yd, xd = torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda()
        g = torch.full_like(xd, float("nan"))
        J = B.misr_gradient_noalloc(desc, yd.data_ptr(), xd.data_ptr(), g.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
        assert rel_l2(g.cpu().numpy(), gr) <= RTOL_OP
        assert J == pytest.approx(Jr, rel=RTOL_OP)


def test_gradient_noalloc_rejects_images_above_its_limit():
    B, fn = _noalloc_fn()
    desc = B.make_desc(300, 200, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5))   # 600 x 400 HR
    x = torch.zeros((600, 400), device="cuda")
    y = torch.zeros((4, 300, 200), device="cuda")
    g = torch.zeros_like(x)
    rc = fn(C.byref(desc), y.data_ptr(), x.data_ptr(), g.data_ptr(), None, 0)
    assert rc == B.MISR_EINVAL
    assert "512" in B.misr_last_error()


def test_gradient_noalloc_refuses_bf16_iterates():
    """The call computes in FP32 only: a BF16-iterate descriptor is refused, not silently run
    in FP32."""
    B, fn = _noalloc_fn()
    h, w, f, shifts, psf, seed = CASES[0]
    desc = B.make_desc(h, w, f, shifts, psf, iterate_dtype=B.MISR_BF16)
    y, x = (torch.from_numpy(a).cuda() for a in _inputs(h, w, f, shifts, seed))
    g = torch.zeros_like(x)
    rc = fn(C.byref(desc), y.data_ptr(), x.data_ptr(), g.data_ptr(), None, 0)
    assert rc == B.MISR_EINVAL
    assert "FP32" in B.misr_last_error()


def test_gradient_noalloc_after_a_timed_out_call():
    """With the wait limit at 0 every tile load is reported late and the call returns
    MISR_ETIMEOUT (no fault: the kernel gives up on its bounded waits, drains its copies and
    returns); with the default limit again, the next call gives the healthy gradient bit for
    bit, so a timed-out call leaves nothing behind in the shared array."""
    B, fn = _noalloc_fn()
    h, w, f, shifts, psf, seed = CASES[1]
    desc = B.make_desc(h, w, f, shifts, psf, lam=0.01, iters=1)
    y, x = (torch.from_numpy(a).cuda() for a in _inputs(h, w, f, shifts, seed))
    s = torch.cuda.current_stream().cuda_stream
    g_ok = torch.full_like(x, float("nan"))
    J_ok = B.misr_gradient_noalloc(desc, y.data_ptr(), x.data_ptr(), g_ok.data_ptr(), s)
    try:
        B.misr_noalloc_set_wait_limit(0)
        g = torch.zeros_like(x)
        with pytest.raises(B.MisrError) as e:
            B.misr_gradient_noalloc(desc, y.data_ptr(), x.data_ptr(), g.data_ptr(), s)
        assert e.value.status == B.MISR_ETIMEOUT
    finally:
        B.misr_noalloc_set_wait_limit(B.TMA_WAIT_TRIES_DEFAULT)
    for _ in range(2):
        g2 = torch.full_like(x, float("nan"))
        J2 = B.misr_gradient_noalloc(desc, y.data_ptr(), x.data_ptr(), g2.data_ptr(), s)
        assert torch.equal(g2, g_ok) and J2 == J_ok
