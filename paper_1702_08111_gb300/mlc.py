"""Python binding of the C ABI in include/mlc.h (argument marshalling only).

Every step of a solve runs in the CUDA library ``_lib/libmlc_gb300.so``; this
module only checks tensors, passes raw device pointers and turns status codes
into exceptions.  PyTorch provides device memory and streams.  There is no
CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
# MLC_GB300_LIBRARY selects another build of the same library (the checked
# debugging variant, libmlc_gb300_checked.so)
LIB_PATH = os.environ.get("MLC_GB300_LIBRARY") or os.path.join(HERE, "_lib", "libmlc_gb300.so")

MLC_TIER_FP64, MLC_TIER_SPLIT, MLC_TIER_DF, MLC_TIER_SPLIT_DF = 0, 1, 2, 3
F32_CHARGE_TIERS = (MLC_TIER_SPLIT, MLC_TIER_SPLIT_DF)
TIER_NAMES = {MLC_TIER_FP64: "fp64", MLC_TIER_SPLIT: "split", MLC_TIER_DF: "df", MLC_TIER_SPLIT_DF: "split_df"}
MLC_MODE_MLC, MLC_MODE_MLC0 = 0, 1
(MLC_OK, MLC_ERR_INVALID_ARG, MLC_ERR_UNSUPPORTED, MLC_ERR_OOM, MLC_ERR_CUDA, MLC_ERR_ADMISSION,
 MLC_ERR_TIMEOUT, MLC_ERR_INDEX) = range(8)
STAGE_MOMENTS, STAGE_FH, STAGE_PHIH, STAGE_PHIB, STAGE_DGF = 0, 1, 2, 3, 4
STAGE_COARSE_SAMPLES, STAGE_FACE_INDEX, STAGE_COARSE_INDEX = 5, 6, 7
STAGE_PHIB_OUTER = 8  # Q = 10: boundary values one node off the face planes

EXPORTED = [
    "mlc_params_init", "mlc_plan_create", "mlc_plan_create_ex", "mlc_plan_destroy",
    "mlc_plan_workspace_bytes", "mlc_solve", "mlc_solve_host", "mlc_batch_solve",
    "mlc_debug_stage_bytes", "mlc_debug_export", "mlc_plan_info", "mlc_server_create",
    "mlc_server_destroy", "mlc_server_enqueue", "mlc_server_wait", "mlc_status_string",
    "mlc_debug_set_timing", "mlc_debug_timing", "mlc_solve_noalloc", "mlc_plan_status",
    "mlc_debug_batch_choice", "mlc_plan_scratch_bytes", "mlc_plan_set_scratch", "mlc_debug_set_fault",
    "mlc_plan_set_dgf", "mlc_debug_batch_chunk",
]
LAUNCH_NAMES = ["moments", "conv_fwd_x", "conv_slab", "conv_inv_x", "resid", "assemble",
                "coarse_fwd_x", "coarse_fwd_y", "coarse_z_kernel", "coarse_inv_y", "coarse_inv_x",
                "boundary", "dirichlet"]


class MLCError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


class mlc_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in
                ("N", "n", "s", "C", "P", "Q", "g_beta", "b", "tier", "mode", "dgf_nD", "dgf_zeta",
                 "conv_chunk", "levels", "coarse_s")]


class mlc_request(ctypes.Structure):
    _fields_ = [("params", mlc_params), ("f", ctypes.c_void_p), ("phi", ctypes.c_void_p)]


class mlc_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    if os.path.abspath(path) == os.path.abspath(_build.LIB_CHECKED):
        if _build.needs_build(_build.LIB_CHECKED):
            _build.build(checked=True)
    elif _build.needs_build():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"MLC CUDA library not found at {path}")
    lib = ctypes.CDLL(path)
    vp, ip, i = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int
    lib.mlc_params_init.argtypes = [ctypes.POINTER(mlc_params), i, i, i, i, i]
    lib.mlc_plan_create.argtypes = [i, i, i, i, i, i, ctypes.POINTER(vp)]
    lib.mlc_plan_create_ex.argtypes = [ctypes.POINTER(mlc_params), ctypes.POINTER(vp)]
    lib.mlc_plan_destroy.argtypes = [vp]
    lib.mlc_plan_workspace_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.mlc_plan_scratch_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.mlc_plan_set_scratch.argtypes = [vp, vp, ctypes.c_size_t]
    lib.mlc_solve.argtypes = [vp, vp, vp, vp]
    lib.mlc_solve_host.argtypes = [vp, vp, vp, vp]
    lib.mlc_solve_noalloc.argtypes = [vp, vp, vp, vp]
    lib.mlc_plan_status.argtypes = [vp]
    lib.mlc_debug_batch_choice.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)]
    lib.mlc_batch_solve.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    lib.mlc_debug_batch_chunk.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)]
    lib.mlc_debug_stage_bytes.argtypes = [vp, i, ctypes.POINTER(ctypes.c_size_t)]
    lib.mlc_debug_export.argtypes = [vp, i, vp, ctypes.c_size_t]
    lib.mlc_plan_info.argtypes = [vp, ip]
    lib.mlc_server_create.argtypes = [ctypes.c_size_t, i, ctypes.POINTER(vp)]
    lib.mlc_server_destroy.argtypes = [vp]
    lib.mlc_server_enqueue.argtypes = [vp, ctypes.POINTER(mlc_request), ctypes.POINTER(ctypes.c_uint64)]
    lib.mlc_server_wait.argtypes = [vp, ctypes.c_uint64, i, ctypes.POINTER(mlc_result)]
    lib.mlc_debug_set_timing.argtypes = [vp, i]
    lib.mlc_debug_set_fault.argtypes = [vp, i]
    lib.mlc_plan_set_dgf.argtypes = [vp, vp, i]
    lib.mlc_debug_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_float), i]
    lib.mlc_status_string.argtypes = [i]
    lib.mlc_status_string.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name != "mlc_status_string":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def status_string(s: int) -> str:
    try:
        return load_library().mlc_status_string(int(s)).decode()
    except Exception:
        return "unknown"


def _check(rc: int, what: str):
    if rc != 0:
        raise MLCError(rc, what)


def make_params(N, n, s, P=4, Q=4, C=4, g_beta=-1, b=-1, tier=MLC_TIER_FP64, mode=MLC_MODE_MLC,
                dgf_nD=-1, dgf_zeta=-1, conv_chunk=-1, levels=-1, coarse_s=-1) -> mlc_params:
    p = mlc_params()
    load_library().mlc_params_init(ctypes.byref(p), N, n, s, P, Q)
    p.C, p.g_beta, p.b, p.tier, p.mode, p.dgf_nD, p.dgf_zeta = C, g_beta, b, tier, mode, dgf_nD, dgf_zeta
    p.conv_chunk = conv_chunk
    p.levels = levels
    p.coarse_s = coarse_s
    return p


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


@dataclass
class PlanInfo:
    N: int
    n: int
    s: int
    b: int
    g_alpha: int
    g_beta: int
    P: int
    npoly: int
    fh_lo: int
    fh_hi: int
    phih_lo: int
    phih_hi: int
    M: int
    Mc: int
    L: int
    nD: int


class Plan:
    """A solver plan (mlc_plan_create_ex); owns device tables and workspace."""

    def __init__(self, N, n, s, P=4, Q=4, **kw):
        lib = load_library()
        self.params = make_params(N, n, s, P, Q, **kw)
        h = ctypes.c_void_p()
        _check(lib.mlc_plan_create_ex(ctypes.byref(self.params), ctypes.byref(h)), "mlc_plan_create_ex")
        self._h = h
        arr = (ctypes.c_int * 16)()
        _check(lib.mlc_plan_info(self._h, arr), "mlc_plan_info")
        self.info = PlanInfo(*list(arr))
        self.tier = self.params.tier

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load_library().mlc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self):
        """mlc_plan_status: synchronise; raise MLCError(TIMEOUT) if a kernel's bounded wait gave up."""
        _check(load_library().mlc_plan_status(self._h), "mlc_plan_status")

    def workspace_bytes(self) -> int:
        v = ctypes.c_size_t()
        _check(load_library().mlc_plan_workspace_bytes(self._h, ctypes.byref(v)), "workspace")
        return v.value

    def scratch_bytes(self) -> int:
        """Bytes of local-convolution scratch a solve needs (mlc_plan_scratch_bytes)."""
        v = ctypes.c_size_t()
        _check(load_library().mlc_plan_scratch_bytes(self._h, ctypes.byref(v)), "scratch_bytes")
        return v.value

    def set_scratch(self, buf=None):
        """Use caller-owned device memory (a CUDA tensor, kept alive by the caller)
        as the local-convolution scratch; None returns to the plan's own."""
        ptr = None if buf is None else ctypes.c_void_p(buf.data_ptr())
        nb = 0 if buf is None else buf.numel() * buf.element_size()
        _check(load_library().mlc_plan_set_scratch(self._h, ptr, ctypes.c_size_t(nb)), "set_scratch")
        self._scratch = buf

    def _check_tensors(self, f, phi):
        import torch
        N = self.params.N
        want = torch.float32 if self.tier in F32_CHARGE_TIERS else torch.float64
        if not (f.is_cuda and phi.is_cuda):
            raise ValueError("f and phi must be CUDA tensors")
        if f.dtype != want or phi.dtype != torch.float64:
            raise ValueError(f"f must be {want}, phi float64")
        if tuple(f.shape) != (N, N, N) or tuple(phi.shape) != (N, N, N):
            raise ValueError(f"f and phi must have shape ({N},{N},{N})")
        if not (f.is_contiguous() and phi.is_contiguous()):
            raise ValueError("f and phi must be contiguous")

    def solve(self, f, phi=None, stream=None):
        """Enqueue a solve on `stream` (default: torch's current stream)."""
        import torch
        if phi is None:
            phi = torch.empty((self.params.N,) * 3, dtype=torch.float64, device=f.device)
        self._check_tensors(f, phi)
        _check(load_library().mlc_solve(self._h, ctypes.c_void_p(f.data_ptr()),
                                        ctypes.c_void_p(phi.data_ptr()),
                                        ctypes.c_void_p(_stream_handle(stream))), "mlc_solve")
        return phi

    def solve_noalloc(self, f, phi, stream=None):
        """mlc_solve_noalloc: the same solve with the local-convolution scratch in
        the library's static device array (nothing is allocated by the call)."""
        self._check_tensors(f, phi)
        _check(load_library().mlc_solve_noalloc(self._h, ctypes.c_void_p(f.data_ptr()),
                                                ctypes.c_void_p(phi.data_ptr()),
                                                ctypes.c_void_p(_stream_handle(stream))), "mlc_solve_noalloc")
        return phi

    def solve_host(self, f_host, phi_host, stream=None):
        """Host arrays in, host array out (copies inside the call); synchronises."""
        _check(load_library().mlc_solve_host(self._h, ctypes.c_void_p(f_host.data_ptr()),
                                             ctypes.c_void_p(phi_host.data_ptr()),
                                             ctypes.c_void_p(_stream_handle(stream))), "mlc_solve_host")
        return phi_host

    def set_dgf(self, table):
        """mlc_plan_set_dgf: use the DGF octant `table` ((L+1)^3 FP64 array,
        k fastest) and rebuild the tables derived from it."""
        import numpy as np
        t = np.ascontiguousarray(table, dtype=np.float64)
        L = t.shape[0] - 1
        if t.shape != (L + 1,) * 3:
            raise ValueError("table must be a cube (L+1)^3")
        _check(load_library().mlc_plan_set_dgf(self._h, ctypes.c_void_p(t.ctypes.data), L), "set_dgf")
        arr = (ctypes.c_int * 16)()
        _check(load_library().mlc_plan_info(self._h, arr), "mlc_plan_info")
        self.info = PlanInfo(*list(arr))

    def set_fault(self, kind: int):
        """Test hook mlc_debug_set_fault: 1 = the inverse-x bulk copies are not
        issued and their bounded waits run out (status TIMEOUT); 0 = normal."""
        _check(load_library().mlc_debug_set_fault(self._h, int(kind)), "set_fault")

    def set_timing(self, enable: bool = True):
        _check(load_library().mlc_debug_set_timing(self._h, int(enable)), "set_timing")

    def timing(self):
        """Per-launch durations (ms) of the last solve, keyed by LAUNCH_NAMES."""
        arr = (ctypes.c_float * len(LAUNCH_NAMES))()
        _check(load_library().mlc_debug_timing(self._h, arr, len(LAUNCH_NAMES)), "timing")
        return dict(zip(LAUNCH_NAMES, list(arr)))

    def export(self, stage: int):
        import numpy as np
        lib = load_library()
        nb = ctypes.c_size_t()
        _check(lib.mlc_debug_stage_bytes(self._h, stage, ctypes.byref(nb)), "stage bytes")
        if stage in (STAGE_FACE_INDEX, STAGE_COARSE_INDEX):
            out = np.empty(nb.value // 4, dtype=np.int32)
            _check(lib.mlc_debug_export(self._h, stage, ctypes.c_void_p(out.ctypes.data), nb.value), "export")
            i = self.info
            if stage == STAGE_FACE_INDEX:
                nodes = 3 * (i.N // i.n + 1) * (i.N + 1) ** 2
            else:
                nodes = (i.fh_hi - i.fh_lo + 1) ** 3
            return out[:nodes + 1].astype(np.int64), out[nodes + 1:].astype(np.int64)
        out = np.empty(nb.value // 8, dtype=np.float64)
        _check(lib.mlc_debug_export(self._h, stage, ctypes.c_void_p(out.ctypes.data), nb.value), "export")
        i = self.info
        if stage == STAGE_COARSE_SAMPLES:
            nc = (i.n + 2 * i.s) // 4 + 1
            return out.reshape(-1, nc, nc, nc)
        if stage == STAGE_MOMENTS:
            return out.reshape(-1, i.npoly)
        if stage == STAGE_FH:
            m = i.fh_hi - i.fh_lo + 1
            return out.reshape(m, m, m)
        if stage == STAGE_PHIH:
            m = i.phih_hi - i.phih_lo + 1
            return out.reshape(m, m, m)
        if stage == STAGE_PHIB:
            npl = i.N // i.n + 1
            return out.reshape(3, npl, i.N + 1, i.N + 1)
        if stage == STAGE_PHIB_OUTER:
            npl = i.N // i.n + 1
            return out.reshape(3, npl, 2, i.N + 1, i.N + 1)
        if stage == STAGE_DGF:
            m = i.L + 1
            return out.reshape(m, m, m)
        return out


def batch_choice(plans, fs, phis) -> dict:
    """The batch autotuner's choice for these arrays: branches and persistence."""
    k = len(plans)
    H = (ctypes.c_void_p * k)(*[p.handle.value for p in plans])
    F = (ctypes.c_void_p * k)(*[f.data_ptr() for f in fs])
    P = (ctypes.c_void_p * k)(*[p.data_ptr() for p in phis])
    v = load_library().mlc_debug_batch_choice(k, H, F, P)
    ch = load_library().mlc_debug_batch_chunk(k, H, F, P)
    return {"branches": v // 2, "persistent_slab": bool(v & 1), "patches_per_conv_launch": ch}


def batch_solve(plans, fs, phis, stream=None):
    lib = load_library()
    k = len(plans)
    H = (ctypes.c_void_p * k)(*[p.handle.value for p in plans])
    F = (ctypes.c_void_p * k)(*[f.data_ptr() for f in fs])
    P = (ctypes.c_void_p * k)(*[p.data_ptr() for p in phis])
    for p, f, ph in zip(plans, fs, phis):
        p._check_tensors(f, ph)
    _check(lib.mlc_batch_solve(k, H, F, P, ctypes.c_void_p(_stream_handle(stream))), "mlc_batch_solve")
    return phis


class Server:
    """Continuous-batching solve server (mlc_server_*): requests are admitted
    while others run, under a device-memory budget; plans stay resident."""

    def __init__(self, budget_bytes: int, max_batch: int = 8):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.mlc_server_create(ctypes.c_size_t(int(budget_bytes)), int(max_batch), ctypes.byref(h)),
               "mlc_server_create")
        self._h = h
        self._keep = {}

    def enqueue(self, f, phi, N, n, s, P=4, Q=4, **kw) -> int:
        """Queue a solve of f into phi (device tensors kept alive until wait)."""
        req = mlc_request()
        req.params = make_params(N, n, s, P, Q, **kw)
        req.f = f.data_ptr()
        req.phi = phi.data_ptr()
        t = ctypes.c_uint64()
        _check(load_library().mlc_server_enqueue(self._h, ctypes.byref(req), ctypes.byref(t)), "mlc_server_enqueue")
        self._keep[t.value] = (f, phi)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        """(status, latency_ms, queue_ms) of a finished request; raises on TIMEOUT."""
        res = mlc_result()
        _check(load_library().mlc_server_wait(self._h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(res)),
               "mlc_server_wait")
        self._keep.pop(ticket, None)
        return res.status, res.latency_ms, res.queue_ms

    def close(self):
        if getattr(self, "_h", None):
            load_library().mlc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
