"""ctypes binding of libmisr.so (the C ABI in include/misr.h).

Argument marshalling only: every step of the solve runs in the library's CUDA kernels.  The
functions carry the C names; `Plan` wraps a plan for torch tensors (device memory and streams
come from PyTorch).  Importing this module fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmisr.so")

MISR_OK, MISR_EINVAL, MISR_ENOMEM, MISR_ECUDA, MISR_EAGAIN, MISR_ETIMEOUT, MISR_ENOTIMPL, MISR_ECANCELED = range(8)
MISR_F32, MISR_U16, MISR_BF16 = 0, 1, 2
MISR_X0_ZERO, MISR_X0_SHIFT_ADD, MISR_X0_GIVEN = 0, 1, 2
MISR_TILE_AUTO, MISR_TILE_32x64, MISR_TILE_32x32, MISR_TILE_16x64, MISR_TILE_STREAM = 0, 1, 2, 3, 4
MISR_N_TILE_SHAPES = 4
MISR_NORM_L2, MISR_NORM_L1 = 0, 1
MISR_DECIM_POINT, MISR_DECIM_BIN = 0, 1
MISR_TRACE_COLS = 10
MISR_PASS_SUMS = 10
TRACE_FIELDS = ("E", "J_trial", "alpha", "delta", "mu", "lam", "Delta", "pn2", "rn2", "accept")
PASS_SUM_FIELDS = ("J_data", "dJ_data", "R_btv", "rr", "rr_cross", "pr", "pp", "a", "b", "c")


class misr_desc(C.Structure):
    _fields_ = [
        ("lr_h", C.c_int32), ("lr_w", C.c_int32), ("K", C.c_int32), ("factor", C.c_int32),
        ("shifts", C.POINTER(C.c_float)), ("psf", C.POINTER(C.c_float)), ("psf_size", C.c_int32),
        ("lambda_", C.c_double), ("btv_alpha", C.c_double), ("btv_w", C.c_int32),
        ("eps", C.c_double), ("iters", C.c_int32), ("x0_mode", C.c_int32),
        ("in_dtype", C.c_int32), ("flat_field", C.c_float), ("iterate_dtype", C.c_int32),
        ("tile_shape", C.c_int32), ("data_norm", C.c_int32), ("data_eps", C.c_double),
        ("decimation", C.c_int32),
    ]


class misr_stats(C.Structure):
    _fields_ = [
        ("iters_done", C.c_int32), ("accepted", C.c_int32), ("status", C.c_int32),
        ("reserved", C.c_int32), ("J_final", C.c_double), ("rnorm2", C.c_double),
        ("lambda_scg", C.c_double),
    ]


class misr_server_cfg(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("passes_per_tick", C.c_int32),
                ("hbm_budget_bytes", C.c_uint64), ("hbm_reserve_bytes", C.c_uint64),
                ("idle_spin_us", C.c_int32), ("reserved", C.c_int32)]


class MisrError(RuntimeError):
    def __init__(self, status, where):
        self.status = int(status)
        super().__init__(f"{where} failed with status {status}: {misr_last_error()}")


_lib = None
VP = C.c_void_p
DP = C.POINTER(C.c_double)


def lib():
    """Load libmisr.so (built in-tree by paper_2108_04315_b300/build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2108_04315_b300/build.py` "
                              "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        L.misr_version.restype = C.c_char_p
        L.misr_last_error.restype = C.c_char_p
        L.misr_plan_create.argtypes = [C.POINTER(misr_desc), C.POINTER(VP)]
        L.misr_plan_destroy.argtypes = [VP]
        L.misr_plan_workspace_bytes.argtypes = [VP, C.POINTER(C.c_size_t)]
        L.misr_plan_set_wait_limit.argtypes = [VP, C.c_uint32]
        L.misr_debug_bounds.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_int32)]
        L.misr_forward.argtypes = [VP, VP, VP, VP]
        L.misr_interpolate.argtypes = [VP, VP, VP, VP]
        L.misr_gradient.argtypes = [VP, VP, VP, VP, DP, VP]
        L.misr_gradient_noalloc.argtypes = [C.POINTER(misr_desc), VP, VP, VP, DP, VP]
        L.misr_noalloc_set_wait_limit.argtypes = [C.c_uint32]
        L.misr_pass_probe.argtypes = [VP, VP, VP, VP, VP, C.c_double, C.c_double, VP, VP, VP, DP, VP]
        L.misr_solve.argtypes = [VP, VP, VP, VP, C.POINTER(misr_stats)]
        L.misr_solve_host.argtypes = [VP, VP, VP, C.POINTER(misr_stats)]
        L.misr_solve_host_many.argtypes = [VP, C.c_int32, C.POINTER(VP), C.POINTER(VP), C.POINTER(misr_stats)]
        L.misr_get_trace.argtypes = [VP, DP, C.c_int32, C.POINTER(C.c_int32)]
        L.misr_state_bytes.argtypes = [VP, C.POINTER(C.c_size_t)]
        L.misr_export_state.argtypes = [VP, VP, C.c_size_t]
        L.misr_import_state.argtypes = [VP, VP, C.c_size_t]
        L.misr_resume.argtypes = [VP, VP, VP, VP, C.POINTER(misr_stats)]
        L.misr_batch_create.argtypes = [C.c_int32, C.POINTER(VP), C.POINTER(VP)]
        L.misr_batch_destroy.argtypes = [VP]
        L.misr_batch_solve.argtypes = [VP, C.POINTER(VP), C.POINTER(VP), VP, C.POINTER(misr_stats)]
        L.misr_autotune.argtypes = [C.POINTER(misr_desc), C.c_int32, C.POINTER(C.c_int32), DP]
        L.misr_server_create.argtypes = [C.POINTER(misr_server_cfg), C.POINTER(VP)]
        L.misr_server_destroy.argtypes = [VP]
        L.misr_submit.argtypes = [VP, C.POINTER(misr_desc), VP, VP, C.POINTER(C.c_uint64)]
        L.misr_poll.argtypes = [VP, C.c_uint64, C.POINTER(misr_stats), DP]
        L.misr_server_wait.argtypes = [VP, C.c_uint64, C.c_double]
        L.misr_cancel.argtypes = [VP, C.c_uint64]
        L.misr_server_counters.argtypes = [VP, C.POINTER(C.c_int64)]
        for name in ("misr_plan_create", "misr_plan_destroy", "misr_plan_workspace_bytes", "misr_plan_set_wait_limit",
                     "misr_debug_bounds",
                     "misr_forward", "misr_interpolate",
                     "misr_gradient", "misr_pass_probe", "misr_solve", "misr_solve_host", "misr_solve_host_many",
                     "misr_get_trace", "misr_state_bytes", "misr_export_state", "misr_import_state", "misr_resume",
                     "misr_batch_create", "misr_batch_destroy", "misr_batch_solve", "misr_server_create",
                     "misr_server_destroy", "misr_submit", "misr_poll", "misr_server_wait", "misr_server_counters", "misr_cancel",
                     "misr_autotune", "misr_gradient_noalloc", "misr_noalloc_set_wait_limit"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(status, where):
    if status != MISR_OK:
        raise MisrError(status, where)


# ---------------------------------------------------------------- C names, thin wrappers
def misr_version() -> str:
    return lib().misr_version().decode()


def misr_last_error() -> str:
    return lib().misr_last_error().decode()


def misr_plan_create(desc: misr_desc) -> int:
    h = VP()
    _check(lib().misr_plan_create(C.byref(desc), C.byref(h)), "misr_plan_create")
    return h.value


def misr_plan_destroy(plan: int) -> None:
    _check(lib().misr_plan_destroy(VP(plan)), "misr_plan_destroy")


def misr_plan_workspace_bytes(plan: int) -> int:
    n = C.c_size_t()
    _check(lib().misr_plan_workspace_bytes(VP(plan), C.byref(n)), "misr_plan_workspace_bytes")
    return n.value


def misr_forward(plan: int, x_dev: int, y_dev: int, stream: int = 0) -> None:
    _check(lib().misr_forward(VP(plan), VP(x_dev), VP(y_dev), VP(stream)), "misr_forward")


def misr_interpolate(plan: int, y_dev: int, x_dev: int, stream: int = 0) -> None:
    _check(lib().misr_interpolate(VP(plan), VP(y_dev), VP(x_dev), VP(stream)), "misr_interpolate")


def misr_gradient(plan: int, y_dev: int, x_dev: int, g_dev: int, stream: int = 0) -> float:
    J = C.c_double()
    _check(lib().misr_gradient(VP(plan), VP(y_dev), VP(x_dev), VP(g_dev), C.byref(J), VP(stream)),
           "misr_gradient")
    return J.value


def misr_pass_probe(plan, y_dev, x_dev, r_dev, p_old_dev, alpha, beta, x_out, r_out, p_out, stream=0):
    sums = (C.c_double * MISR_PASS_SUMS)()
    _check(lib().misr_pass_probe(VP(plan), VP(y_dev), VP(x_dev), VP(r_dev), VP(p_old_dev), float(alpha),
                                 float(beta), VP(x_out), VP(r_out), VP(p_out), sums, VP(stream)),
           "misr_pass_probe")
    return dict(zip(PASS_SUM_FIELDS, list(sums)))


def misr_debug_bounds():
    """(bits, first) of the bounds-checked build; raises MisrError(MISR_ENOTIMPL) on the normal one."""
    bits = C.c_uint32()
    first = (C.c_int32 * 4)()
    _check(lib().misr_debug_bounds(C.byref(bits), first), "misr_debug_bounds")
    return int(bits.value), list(first)


TMA_WAIT_TRIES_DEFAULT = 1 << 24


def misr_plan_set_wait_limit(plan: int, tries: int):
    _check(lib().misr_plan_set_wait_limit(VP(plan), int(tries)), "misr_plan_set_wait_limit")


def misr_gradient_noalloc(desc: misr_desc, y_dev: int, x_dev: int, g_dev: int, stream: int = 0) -> float:
    J = C.c_double()
    _check(lib().misr_gradient_noalloc(C.byref(desc), VP(y_dev), VP(x_dev), VP(g_dev), C.byref(J), VP(stream)),
           "misr_gradient_noalloc")
    return J.value


def misr_noalloc_set_wait_limit(tries: int):
    _check(lib().misr_noalloc_set_wait_limit(int(tries)), "misr_noalloc_set_wait_limit")


def misr_solve(plan: int, y_dev: int, x_dev: int, stream: int = 0, want_stats: bool = True):
    st = misr_stats()
    _check(lib().misr_solve(VP(plan), VP(y_dev), VP(x_dev), VP(stream), C.byref(st) if want_stats else None),
           "misr_solve")
    return _stats_dict(st) if want_stats else None


def misr_solve_host(plan: int, y_host: int, x_host: int):
    st = misr_stats()
    _check(lib().misr_solve_host(VP(plan), VP(y_host), VP(x_host), C.byref(st)), "misr_solve_host")
    return _stats_dict(st)


def misr_solve_host_many(plan: int, y_hosts, x_hosts, want_stats: bool = True):
    """Solve len(y_hosts) projections from host buffers (addresses) with overlapped copies."""
    n = len(y_hosts)
    if len(x_hosts) != n:
        raise ValueError("y_hosts and x_hosts differ in length")
    ya = (VP * max(1, n))(*[VP(a) for a in y_hosts])
    xa = (VP * max(1, n))(*[VP(a) for a in x_hosts])
    st = (misr_stats * max(1, n))()
    _check(lib().misr_solve_host_many(VP(plan), n, ya, xa, st if want_stats else None), "misr_solve_host_many")
    return [_stats_dict(st[k]) for k in range(n)] if want_stats else None


def misr_state_bytes(plan: int) -> int:
    n = C.c_size_t()
    _check(lib().misr_state_bytes(VP(plan), C.byref(n)), "misr_state_bytes")
    return int(n.value)


def misr_export_state(plan: int) -> np.ndarray:
    buf = np.zeros(misr_state_bytes(plan), dtype=np.uint8)
    _check(lib().misr_export_state(VP(plan), buf.ctypes.data, buf.nbytes), "misr_export_state")
    return buf


def misr_import_state(plan: int, buf: np.ndarray):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib().misr_import_state(VP(plan), buf.ctypes.data, buf.nbytes), "misr_import_state")


def misr_resume(plan: int, y_dev: int, x_dev: int, stream: int = 0, want_stats: bool = True):
    st = misr_stats()
    _check(lib().misr_resume(VP(plan), VP(y_dev), VP(x_dev), VP(stream), C.byref(st) if want_stats else None),
           "misr_resume")
    return _stats_dict(st) if want_stats else None


def misr_get_trace(plan: int, max_rows: int):
    buf = np.zeros((max(1, max_rows), MISR_TRACE_COLS), dtype=np.float64)
    rows = C.c_int32()
    _check(lib().misr_get_trace(VP(plan), buf.ctypes.data_as(DP), int(max_rows), C.byref(rows)), "misr_get_trace")
    buf = buf[: rows.value]
    return {k: buf[:, i].copy() for i, k in enumerate(TRACE_FIELDS)}


def misr_batch_create(plans) -> int:
    arr = (VP * len(plans))(*[VP(p) for p in plans])
    h = VP()
    _check(lib().misr_batch_create(len(plans), arr, C.byref(h)), "misr_batch_create")
    return h.value


def misr_batch_destroy(batch: int) -> None:
    _check(lib().misr_batch_destroy(VP(batch)), "misr_batch_destroy")


def misr_batch_solve(batch: int, y_devs, x_devs, stream: int = 0, want_stats: bool = True):
    n = len(y_devs)
    ya = (VP * n)(*[VP(v) for v in y_devs])
    xa = (VP * n)(*[VP(v) for v in x_devs])
    st = (misr_stats * n)()
    _check(lib().misr_batch_solve(VP(batch), ya, xa, VP(stream), st if want_stats else None), "misr_batch_solve")
    return [_stats_dict(st[i]) for i in range(n)] if want_stats else None


def misr_server_create(max_slots: int, passes_per_tick: int = 0, hbm_budget_bytes: int = 0,
                       hbm_reserve_bytes: int = 0, idle_spin_us: int = 0) -> int:
    cfg = misr_server_cfg(int(max_slots), int(passes_per_tick), int(hbm_budget_bytes), int(hbm_reserve_bytes),
                          int(idle_spin_us), 0)
    h = VP()
    _check(lib().misr_server_create(C.byref(cfg), C.byref(h)), "misr_server_create")
    return h.value


def misr_server_destroy(server: int) -> None:
    _check(lib().misr_server_destroy(VP(server)), "misr_server_destroy")


def misr_submit(server: int, desc: misr_desc, y_dev: int, x_dev: int) -> int:
    t = C.c_uint64()
    _check(lib().misr_submit(VP(server), C.byref(desc), VP(y_dev), VP(x_dev), C.byref(t)), "misr_submit")
    return t.value


def misr_poll(server: int, ticket: int):
    """None while the request is pending; else (stats dict, (t_submit, t_start, t_end))."""
    st = misr_stats()
    times = np.zeros(3, dtype=np.float64)
    rc = lib().misr_poll(VP(server), C.c_uint64(ticket), C.byref(st), times.ctypes.data_as(DP))
    if rc == MISR_EAGAIN:
        return None
    _check(rc, "misr_poll")
    return _stats_dict(st), tuple(float(v) for v in times)


def misr_server_wait(server: int, ticket: int, timeout_s: float) -> None:
    _check(lib().misr_server_wait(VP(server), C.c_uint64(ticket), float(timeout_s)), "misr_server_wait")


def misr_server_counters(server: int) -> dict:
    out = (C.c_int64 * 5)()
    _check(lib().misr_server_counters(VP(server), out), "misr_server_counters")
    return dict(zip(("queued", "running", "slots", "slot_bytes", "passes_launched"), list(out)))


def misr_autotune(desc: misr_desc, passes: int = 10):
    """Time every tile shape on this geometry; the fastest becomes the default of later plans of
    the same HR size.  Returns (chosen MISR_TILE_*, ms per pass of each shape)."""
    shape = C.c_int32()
    ms = np.zeros(MISR_N_TILE_SHAPES, dtype=np.float64)
    _check(lib().misr_autotune(C.byref(desc), int(passes), C.byref(shape), ms.ctypes.data_as(DP)), "misr_autotune")
    return shape.value, ms


def _stats_dict(st: misr_stats):
    return {"iters_done": st.iters_done, "accepted": st.accepted, "status": st.status,
            "J_final": st.J_final, "rnorm2": st.rnorm2, "lambda_scg": st.lambda_scg}


# ---------------------------------------------------------------- torch convenience layer
def make_desc(lr_h, lr_w, factor, shifts, psf, lam=0.01, btv_alpha=0.4, btv_w=3, eps=1e-3, iters=100,
              x0_mode=MISR_X0_SHIFT_ADD, in_dtype=MISR_F32, flat_field=40000.0, iterate_dtype=MISR_F32,
              tile_shape=MISR_TILE_AUTO, data_norm=MISR_NORM_L2, data_eps=0.0, decimation=MISR_DECIM_POINT):
    sh = np.ascontiguousarray(np.asarray(shifts, dtype=np.float32).reshape(-1))
    ps = np.ascontiguousarray(np.asarray(psf, dtype=np.float32))
    d = misr_desc()
    d.lr_h, d.lr_w, d.K, d.factor = int(lr_h), int(lr_w), len(sh) // 2, int(factor)
    d.shifts = sh.ctypes.data_as(C.POINTER(C.c_float))
    d.psf = ps.ctypes.data_as(C.POINTER(C.c_float))
    d.psf_size = int(ps.shape[0])
    d.lambda_, d.btv_alpha, d.btv_w, d.eps = float(lam), float(btv_alpha), int(btv_w), float(eps)
    d.iters, d.x0_mode, d.in_dtype = int(iters), int(x0_mode), int(in_dtype)
    d.flat_field, d.iterate_dtype = float(flat_field), int(iterate_dtype)
    d.tile_shape = int(tile_shape)
    d.data_norm, d.data_eps = int(data_norm), float(data_eps)
    d.decimation = int(decimation)
    d._keep = (sh, ps)  # keep the host arrays alive while the descriptor is used
    return d


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Plan:
    """A plan plus torch-tensor entry points.  Tensors must be contiguous CUDA tensors on the
    plan's device: y (K, h, w) float32 or uint16-as-int16/uint16, x (H, W) float32."""

    def __init__(self, lr_h, lr_w, factor, shifts, psf, **kw):
        self.desc = make_desc(lr_h, lr_w, factor, shifts, psf, **kw)
        self.h, self.w, self.f = int(lr_h), int(lr_w), int(factor)
        self.K = self.desc.K
        self.H, self.W = self.f * self.h, self.f * self.w
        self.iters = self.desc.iters
        self.handle = misr_plan_create(self.desc)

    def close(self):
        if getattr(self, "handle", None):
            misr_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _ptr(t, dtype=None):
        assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
        if dtype is not None:
            assert t.dtype == dtype, (t.dtype, dtype)
        return int(t.data_ptr())

    def workspace_bytes(self):
        return misr_plan_workspace_bytes(self.handle)

    def forward(self, x, y_out=None, stream=None):
        import torch
        if y_out is None:
            y_out = torch.empty((self.K, self.h, self.w), dtype=torch.float32, device=x.device)
        misr_forward(self.handle, self._ptr(x, torch.float32), self._ptr(y_out, torch.float32), _stream_handle(stream))
        return y_out

    def interpolate(self, y, x_out=None, stream=None):
        """Multi-image interpolation of the frames y (the plan's in_dtype) into an HR image."""
        import torch
        if x_out is None:
            x_out = torch.empty((self.H, self.W), dtype=torch.float32, device=y.device)
        misr_interpolate(self.handle, self._ptr(y), self._ptr(x_out, torch.float32), _stream_handle(stream))
        return x_out

    def gradient(self, y, x, stream=None):
        import torch
        g = torch.empty_like(x)
        J = misr_gradient(self.handle, self._ptr(y), self._ptr(x, torch.float32), self._ptr(g), _stream_handle(stream))
        return J, g

    def pass_probe(self, y, x, r, p_old, alpha, beta, stream=None):
        import torch
        xo, ro, po = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
        sums = misr_pass_probe(self.handle, self._ptr(y), self._ptr(x, torch.float32), self._ptr(r, torch.float32),
                               self._ptr(p_old, torch.float32), alpha, beta, self._ptr(xo), self._ptr(ro),
                               self._ptr(po), _stream_handle(stream))
        return xo, ro, po, sums

    def solve(self, y, x_out=None, stream=None, stats=True):
        import torch
        if x_out is None:
            x_out = torch.empty((self.H, self.W), dtype=torch.float32, device=y.device)
        st = misr_solve(self.handle, self._ptr(y), self._ptr(x_out, torch.float32), _stream_handle(stream), stats)
        return x_out, st

    def solve_host(self, y_host: np.ndarray, x_host: np.ndarray):
        assert y_host.flags.c_contiguous and x_host.flags.c_contiguous and x_host.dtype == np.float32
        return misr_solve_host(self.handle, y_host.ctypes.data, x_host.ctypes.data)

    def solve_host_many(self, y_hosts, x_hosts, stats=True):
        """Projections y_hosts[k] -> x_hosts[k] (C-contiguous host arrays), the copies of one
        overlapped with the solve of another (page-locked arrays overlap; others serialise)."""
        for a in list(y_hosts) + list(x_hosts):
            assert a.flags.c_contiguous
        assert all(x.dtype == np.float32 for x in x_hosts)
        return misr_solve_host_many(self.handle, [a.ctypes.data for a in y_hosts], [a.ctypes.data for a in x_hosts],
                                    stats)

    def export_state(self):
        """Checkpoint of the last completed solve (x_k, r_k, p_{k-1} and the SCG scalars)."""
        return misr_export_state(self.handle)

    def import_state(self, buf):
        misr_import_state(self.handle, buf)

    def resume(self, y, x_out=None, stream=None, stats=True):
        """Continue the imported (or stopped) solve to this plan's iteration count."""
        import torch
        if x_out is None:
            x_out = torch.empty((self.H, self.W), dtype=torch.float32, device=y.device)
        st = misr_resume(self.handle, self._ptr(y), self._ptr(x_out, torch.float32), _stream_handle(stream), stats)
        return x_out, st

    def trace(self):
        return misr_get_trace(self.handle, self.iters)


class Batch:
    """Plans solved together: one fused-pass launch per SCG step over all of their tiles."""

    def __init__(self, plans):
        self.plans = list(plans)
        self.handle = misr_batch_create([p.handle for p in self.plans])

    def close(self):
        if getattr(self, "handle", None):
            misr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, ys, xs=None, stream=None, stats=True):
        import torch
        if xs is None:
            xs = [torch.empty((p.H, p.W), dtype=torch.float32, device=y.device) for p, y in zip(self.plans, ys)]
        st = misr_batch_solve(self.handle, [Plan._ptr(y) for y in ys], [Plan._ptr(x, torch.float32) for x in xs],
                              _stream_handle(stream), stats)
        return xs, st


class Server:
    """Continuous-batching solver: submit projections as they arrive, poll or wait for results.
    Frames and outputs are CUDA tensors that must stay alive until their ticket finishes."""

    def __init__(self, max_slots=64, passes_per_tick=0, hbm_budget_bytes=0, hbm_reserve_bytes=0, idle_spin_us=0):
        self.handle = misr_server_create(max_slots, passes_per_tick, hbm_budget_bytes, hbm_reserve_bytes,
                                         idle_spin_us)
        self._live = {}

    def close(self):
        if getattr(self, "handle", None):
            misr_server_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, y, lr_h, lr_w, factor, shifts, psf, x_out=None, **kw):
        return self.submit_desc(y, make_desc(lr_h, lr_w, factor, shifts, psf, **kw), x_out)

    def submit_desc(self, y, desc, x_out=None):
        """submit with a descriptor made once by make_desc (an acquisition loop's scan class):
        no per-request marshalling of the shifts, the PSF and the options."""
        import torch
        if x_out is None:
            x_out = torch.empty((desc.factor * desc.lr_h, desc.factor * desc.lr_w), dtype=torch.float32,
                                device=y.device)
        # work queued on the caller's stream (e.g. the frames' upload) must be done first
        stream = torch.cuda.current_stream(y.device)
        if not stream.query():
            stream.synchronize()
        t = misr_submit(self.handle, desc, Plan._ptr(y), Plan._ptr(x_out, torch.float32))
        self._live[t] = (y, x_out)
        return t

    def poll(self, ticket):
        try:
            r = misr_poll(self.handle, ticket)
        except MisrError:
            self._live.pop(ticket, None)
            raise
        if r is None:
            return None
        y, x = self._live.pop(ticket)
        return x, r[0], r[1]

    def wait(self, ticket, timeout_s=60.0):
        misr_server_wait(self.handle, ticket, timeout_s)
        return self.poll(ticket)

    def cancel(self, ticket):
        """Drop a queued request, or stop a running one after the current tick (MISR_ECANCELED)."""
        _check(lib().misr_cancel(VP(self.handle), int(ticket)), "misr_cancel")

    def counters(self):
        return misr_server_counters(self.handle)
