"""C ABI checks that need no GPU: the library builds and loads, exports every entry point
declared in include/*.h, and rejects invalid descriptors on the host (MISR_EINVAL /
MISR_ENOTIMPL) before touching the device."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(misr_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    from paper_2108_04315_b300 import build, binding
    build.build()
    return binding.lib()


def test_header_declares_entry_points():
    names = declared_functions()
    for want in ("misr_plan_create", "misr_plan_destroy", "misr_solve", "misr_solve_host", "misr_solve_host_many",
                 "misr_forward",
                 "misr_gradient", "misr_pass_probe", "misr_get_trace", "misr_last_error", "misr_version"):
        assert want in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, f"not exported: {missing}"


def test_version_string(L):
    from paper_2108_04315_b300 import binding
    assert "sm_103a" in binding.misr_version()


def _desc(**kw):
    import gen
    from paper_2108_04315_b300 import binding
    base = dict(lr_h=16, lr_w=16, factor=2, shifts=gen.half_pixel_shifts(), psf=gen.gaussian_psf(5, 0.5))
    base.update(kw)
    return binding.make_desc(**base)


@pytest.mark.parametrize("kw,status", [
    (dict(factor=0), "EINVAL"),
    (dict(lr_h=0), "EINVAL"),
    (dict(shifts=[(0.0, 0.0)] * 65), "EINVAL"),                   # K > 64
    (dict(shifts=[(0.25, 0.0)], psf=np.ones((3, 3)), tile_shape=1), "ENOTIMPL"),   # per-phase taps: 32x32 only
    (dict(shifts=[(0.0, float("nan"))]), "EINVAL"),
    (dict(shifts=[(0.0, 2.0 ** 20)]), "EINVAL"),                  # shift beyond 2^20 HR px
    (dict(shifts=[(0.0, 0.0), (0.0, 0.0)], iterate_dtype=2), "ENOTIMPL"),   # frame-wise pass: float r and p
    (dict(psf=np.ones((4, 4))), "EINVAL"),                        # even PSF
    (dict(psf=np.ones((7, 7))), "EINVAL"),                        # PSF larger than 5x5
    (dict(psf=np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1.0]])), "EINVAL"),   # not separable
    (dict(eps=0.0), "EINVAL"),
    (dict(eps=1e-20), "EINVAL"),                                  # eps^2 below the FP32 normals
    (dict(btv_w=4), "EINVAL"),
    (dict(lam=-1.0), "EINVAL"),
    (dict(iters=-1), "EINVAL"),
    (dict(in_dtype=7), "EINVAL"),
    (dict(iterate_dtype=1), "EINVAL"),                            # u16 is an input type only
    (dict(data_norm=2), "EINVAL"),
    (dict(data_norm=1, data_eps=0.0), "EINVAL"),                  # the L1 term needs eps_d > 0
    (dict(data_norm=1, data_eps=1e20), "EINVAL"),
    (dict(data_norm=1, data_eps=float("nan")), "EINVAL"),
    (dict(decimation=2), "EINVAL"),
])
def test_invalid_descriptor_rejected_on_host(L, kw, status):
    from paper_2108_04315_b300 import binding
    d = _desc(**kw)
    h = C.c_void_p()
    rc = L.misr_plan_create(C.byref(d), C.byref(h))
    assert rc == getattr(binding, "MISR_" + status), binding.misr_last_error()
    assert h.value is None
    assert binding.misr_last_error()


def test_null_arguments_rejected(L):
    from paper_2108_04315_b300 import binding
    assert L.misr_plan_create(None, None) == binding.MISR_EINVAL
    assert L.misr_solve(None, None, None, None, None) == binding.MISR_EINVAL
    assert L.misr_solve_host_many(None, 1, None, None, None) == binding.MISR_EINVAL
    assert L.misr_plan_set_wait_limit(None, 0) == binding.MISR_EINVAL
    assert L.misr_debug_bounds(None, None) == binding.MISR_EINVAL
    assert L.misr_cancel(None, 1) == binding.MISR_EINVAL
    assert L.misr_interpolate(None, None, None, None) == binding.MISR_EINVAL
    assert L.misr_state_bytes(None, None) == binding.MISR_EINVAL
    assert L.misr_export_state(None, None, 0) == binding.MISR_EINVAL
    assert L.misr_import_state(None, None, 0) == binding.MISR_EINVAL
    assert L.misr_resume(None, None, None, None, None) == binding.MISR_EINVAL
    assert L.misr_plan_destroy(None) == binding.MISR_OK


@pytest.mark.parametrize("cfg", [(0, 0, 0), (4097, 0, 0), (4, -1, 0), (4, 1001, 0), (4, 0, -1), (4, 0, 1000001)])
def test_server_config_rejected_on_host(L, cfg):
    """misr_server_create checks its configuration before it touches the device"""
    from paper_2108_04315_b300 import binding
    slots, tick, spin = cfg
    c = binding.misr_server_cfg(slots, tick, 0, 0, spin, 0)
    h = C.c_void_p()
    assert L.misr_server_create(C.byref(c), C.byref(h)) == binding.MISR_EINVAL
    assert h.value is None


@pytest.mark.parametrize("kw", [
    dict(shifts=[(0.0, 0.0)] * 5),                                # K > f^2
    dict(shifts=[(0.0, 0.0), (0.0, 0.0)]),                        # same phase twice
    dict(shifts=[(0.5, 0.0), (0.0, 0.5), (-0.5, 0.0), (0.0, -0.5)], decimation=1, psf=np.ones((3, 3))),  # the study's
    dict(shifts=[(0.25, 0.0)]),                                   # f*s not an integer, 5x5 PSF: 6 taps
    dict(shifts=[(0.0, 0.0), (0.6, 0.0), (0.0, 0.5), (0.55, 0.5)], psf=np.ones((3, 3))),  # off a product lattice
    dict(shifts=[(1.0, 0.0)]),                                    # shift beyond [0, 1-1/f]
    dict(decimation=1),                                           # 5x5 PSF binned at f=2: 6 taps
    dict(decimation=1, factor=3, shifts=[(0.0, 0.0)], psf=np.ones((3, 3))),
])
def test_frame_wise_geometries_accepted_on_host(L, kw):
    """Frame sets the fused passes cannot interleave go to the frame-wise pass: the descriptor
    checks accept them, and misr_autotune (nothing to choose: one pass kernel) answers
    MISR_TILE_AUTO before any device work."""
    from paper_2108_04315_b300 import binding
    d = _desc(**kw)
    shape, ms = binding.misr_autotune(d, 1)
    assert shape == binding.MISR_TILE_AUTO
    assert not np.any(ms)
