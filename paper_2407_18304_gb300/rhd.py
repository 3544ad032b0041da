"""Python binding of the C ABI in ``include/rhd.h`` (argument marshalling only).

Every step of the source-term update runs in the CUDA library; this module
only turns torch tensors into the C structs and calls ``rhd_source_update``.
There is no CPU path: if the library is missing, the call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

FP64, MIXED = 0, 1
M1, EDDINGTON = 0, 1
PPL_FIXED, PC, PPL_FREE = 0, 1, 2
STATUS_OK, STATUS_FALLBACK, STATUS_MAXITER, STATUS_INVALID = 0, 1, 2, 3
GROUP_TEST = 1
FLUX_TEST = 2
CELL_PER_THREAD = 4
LANES_16 = 8
MAX_GROUPS = 256
NOALLOC_BYTES = 64 << 20

_P = ctypes.c_void_p
_D = ctypes.c_double


class State(ctypes.Structure):
    _fields_ = [("rho", _P), ("mom", _P * 3), ("egas", _P), ("kappa0", _P), ("erad", _P),
                ("frad", _P * 3), ("src", _P), ("status", _P), ("iters", _P),
                ("group_stride", ctypes.c_int64), ("c_v", _D), ("theta", _D), ("c", _D),
                ("c_hat", _D), ("a_rad", _D), ("h", _D), ("k_B", _D), ("tol", _D),
                ("tol_outer", _D), ("max_newton", ctypes.c_int32), ("max_outer", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("closure", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class Groups(ctypes.Structure):
    _fields_ = [("n_groups", ctypes.c_int32), ("edges", ctypes.POINTER(_D))]


class OpacityLaw(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("n_seg", ctypes.c_int32),
                ("nu_break", ctypes.POINTER(_D)), ("seg_logk", ctypes.POINTER(_D)),
                ("seg_beta", ctypes.POINTER(_D)), ("nu_ref", _D),
                ("khat_gminus", ctypes.POINTER(_D)), ("alpha_g", ctypes.POINTER(_D)),
                ("temp_exponent", _D), ("T_ref", _D)]


class Grid(ctypes.Structure):
    _fields_ = [("state", State), ("groups", Groups), ("opacity_law", OpacityLaw), ("dt", _D),
                ("n_cells", ctypes.c_int64)]


class RhdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rhd error {code}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load the in-tree CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing "
                               "(run __graft_entry__.build() or python -m paper_2407_18304_gb300.build)")
        _lib = ctypes.CDLL(path)
        _lib.rhd_source_update.restype = ctypes.c_int
        _lib.rhd_source_update.argtypes = [ctypes.POINTER(State), ctypes.POINTER(Groups),
                                           ctypes.POINTER(OpacityLaw), _D, ctypes.c_int64, _P]
        _lib.rhd_source_update_noalloc.restype = ctypes.c_int
        _lib.rhd_source_update_noalloc.argtypes = [ctypes.POINTER(State), ctypes.POINTER(Groups),
                                                   ctypes.POINTER(OpacityLaw), _D, ctypes.c_int64,
                                                   _P]
        _lib.rhd_context_create.restype = ctypes.c_int
        _lib.rhd_context_create.argtypes = [ctypes.POINTER(_P)]
        _lib.rhd_context_destroy.restype = ctypes.c_int
        _lib.rhd_context_destroy.argtypes = [_P]
        _lib.rhd_source_update_batched.restype = ctypes.c_int
        _lib.rhd_source_update_batched.argtypes = [_P, ctypes.POINTER(Grid), ctypes.c_int32, _P]
        _lib.rhd_context_autotune.restype = ctypes.c_int
        _lib.rhd_context_autotune.argtypes = [_P, ctypes.POINTER(Grid), ctypes.c_int32, _P]
        _lib.rhd_context_shape.restype = ctypes.c_int
        _lib.rhd_context_shape.argtypes = [_P, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int32)]
        _lib.rhd_context_mapping.restype = ctypes.c_int
        _lib.rhd_context_mapping.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_int32)]
        _lib.rhd_context_set_mapping.restype = ctypes.c_int
        _lib.rhd_context_set_mapping.argtypes = [_P, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_int32]
        _F = ctypes.c_void_p
        sig = {
            "rhd_surrogate_create": [ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(_P)],
            "rhd_surrogate_destroy": [_P],
            "rhd_surrogate_dims": [_P, ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)],
            "rhd_surrogate_features": [_P, ctypes.POINTER(State), ctypes.POINTER(Groups),
                                       ctypes.POINTER(OpacityLaw), _D, ctypes.c_int64, _F, _P],
            "rhd_surrogate_targets": [_P, ctypes.POINTER(State), ctypes.POINTER(State),
                                      ctypes.POINTER(Groups), ctypes.POINTER(OpacityLaw), _D,
                                      ctypes.c_int64, _F, _P],
            "rhd_surrogate_fit_normalization": [_P, _F, _F, ctypes.c_int64, _P],
            "rhd_surrogate_params": [_P, _F, _F, ctypes.c_int32, _P],
            "rhd_surrogate_loss_grad": [_P, _F, _F, ctypes.c_int64, _F, _F, _P],
            "rhd_surrogate_train_step": [_P, _F, _F, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_float, _F, _P],
            "rhd_surrogate_predict": [_P, _F, ctypes.c_int64, _F, _P],
            "rhd_surrogate_error": [_P, ctypes.POINTER(ctypes.c_int32)],
            "rhd_surrogate_test_wait_timeout": [_P, ctypes.c_int32],
            "rhd_source_update_warm": [_P, ctypes.POINTER(State), ctypes.POINTER(Groups),
                                       ctypes.POINTER(OpacityLaw), _D, ctypes.c_int64, _P],
            "rhd_surrogate_save": [_P, ctypes.c_char_p],
            "rhd_surrogate_checkpoint": [_P, ctypes.c_char_p],
            "rhd_surrogate_load": [ctypes.c_char_p, ctypes.POINTER(_P)],
            "rhd_surrogate_warm_start": [_P, ctypes.POINTER(State), ctypes.POINTER(Groups),
                                         ctypes.POINTER(OpacityLaw), _D, ctypes.c_int64, _F, _F,
                                         _P],
        }
        for name, args in sig.items():
            f = getattr(_lib, name)
            f.restype = ctypes.c_int
            f.argtypes = args
        _lib.rhd_source_update_host.restype = ctypes.c_int
        _lib.rhd_source_update_host.argtypes = [ctypes.POINTER(State), ctypes.POINTER(Groups),
                                                ctypes.POINTER(OpacityLaw), _D, ctypes.c_int64,
                                                _P, ctypes.c_int64]
        _lib.rhd_imex_step.restype = ctypes.c_int
        _lib.rhd_imex_step.argtypes = [ctypes.POINTER(State), ctypes.POINTER(Groups),
                                       ctypes.POINTER(OpacityLaw), _D, ctypes.c_int64, _P]
        _lib.rhd_profile_start.restype = ctypes.c_int
        _lib.rhd_profile_start.argtypes = []
        _lib.rhd_profile_kernel.restype = ctypes.c_int
        _lib.rhd_profile_kernel.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_double)]
        _lib.rhd_events_start.restype = ctypes.c_int
        _lib.rhd_events_start.argtypes = []
        _lib.rhd_events_stop.restype = ctypes.c_int
        _lib.rhd_events_stop.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        _lib.rhd_profile_stop.restype = ctypes.c_int
        _lib.rhd_profile_stop.argtypes = [ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_double)]
        _lib.rhd_strerror.restype = ctypes.c_char_p
        _lib.rhd_strerror.argtypes = [ctypes.c_int]
        _lib.rhd_version.restype = ctypes.c_int
        _lib.rhd_version.argtypes = []
    return _lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(_D))


def _check(t: torch.Tensor, name: str, shape, dtype=torch.float64, device: str = "cuda"):
    if not isinstance(t, torch.Tensor) or t.device.type != device:
        raise ValueError(f"{name} must be a {device.upper()} tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name}: expected contiguous {dtype} {tuple(shape)}, got "
                         f"{t.dtype} {tuple(t.shape)}")
    # the library launches on the current device: another device's pointers would fault
    if device == "cuda" and t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on {t.device} but the current device is "
                         f"cuda:{torch.cuda.current_device()}")


def make_law(law, mode: int = PPL_FIXED, khat_g=None, alpha_g=None, temp_exponent=0.0, T_ref=1.0):
    """Pack an opacity law (nu_break, seg_logk, seg_beta, nu_ref) into the C struct.

    Returns (struct, keep-alive list)."""
    nb = np.ascontiguousarray(law.nu_break, dtype=np.float64)
    lk = np.ascontiguousarray(law.seg_logk, dtype=np.float64)
    be = np.ascontiguousarray(law.seg_beta, dtype=np.float64)
    keep = [nb, lk, be]
    s = OpacityLaw(mode, len(lk), _dp(nb) if len(nb) else None, _dp(lk), _dp(be),
                   float(law.nu_ref), None, None, float(temp_exponent), float(T_ref))
    if khat_g is not None:
        kg = np.ascontiguousarray(khat_g, dtype=np.float64)
        keep.append(kg)
        s.khat_gminus = _dp(kg)
        if alpha_g is not None:
            ag = np.ascontiguousarray(alpha_g, dtype=np.float64)
            keep.append(ag)
            s.alpha_g = _dp(ag)
    return s, keep


def _state(state: dict, G: int, n: int, gs: int, *, c_v: float, consts: dict, theta: float,
           precision: int, closure: int, tol: float, tol_outer: float, max_newton: int,
           max_outer: int, status, iters, flags: int, device: str = "cuda") -> State:
    """Check the tensors of one grid and fill the C state struct."""
    rho = state["rho"]
    d = device
    _check(rho, "rho", (rho.shape[0],), device=d)
    # the per-cell arrays hold rho.shape[0] cells; the library reads n of them
    if not 0 <= n <= rho.shape[0] or gs < n:
        raise ValueError(f"n_cells = {n} with {rho.shape[0]} cells per array and group "
                         f"stride {gs}")
    _check(state["mom"], "mom", (3, rho.shape[0]), device=d)
    _check(state["egas"], "egas", (rho.shape[0],), device=d)
    _check(state["erad"], "erad", (G, gs), device=d)
    _check(state["frad"], "frad", (3, G, gs), device=d)
    if state.get("kappa0") is not None:
        _check(state["kappa0"], "kappa0", (rho.shape[0],), device=d)
    if state.get("src") is not None:
        _check(state["src"], "src", (G, gs), device=d)
    if status is not None:
        _check(status, "status", (rho.shape[0],), torch.uint8, device=d)
    if iters is not None:
        _check(iters, "iters", (rho.shape[0],), torch.uint8, device=d)
    mom, frad = state["mom"], state["frad"]
    st = State()
    st.rho = _ptr(rho)
    for d in range(3):
        st.mom[d] = _ptr(mom[d])
        st.frad[d] = _ptr(frad[d])
    st.egas = _ptr(state["egas"])
    st.kappa0 = _ptr(state.get("kappa0"))
    st.erad = _ptr(state["erad"])
    st.src = _ptr(state.get("src"))
    st.status = _ptr(status)
    st.iters = _ptr(iters)
    st.group_stride = gs
    st.c_v, st.theta = float(c_v), float(theta)
    st.c, st.c_hat, st.a_rad = float(consts["c"]), float(consts.get("c_hat", consts["c"])), float(consts["a_rad"])
    st.h, st.k_B = float(consts["h"]), float(consts["k_B"])
    st.tol, st.tol_outer = float(tol), float(tol_outer)
    st.max_newton, st.max_outer = int(max_newton), int(max_outer)
    st.precision, st.closure, st.flags = int(precision), int(closure), int(flags)
    return st


def source_update(state: dict, edges, law, *, dt: float, c_v: float, consts: dict,
                  theta: float = 1.0, precision: int = FP64, closure: int = M1,
                  tol: float = 0.0, tol_outer: float = 0.0, max_newton: int = 0,
                  max_outer: int = 0, status: torch.Tensor | None = None,
                  iters: torch.Tensor | None = None, mode: int = PPL_FIXED, khat_g=None,
                  alpha_g=None, temp_exponent: float = 0.0, T_ref: float = 1.0,
                  stream: torch.cuda.Stream | None = None, n_cells: int | None = None,
                  group_stride: int = 0, flags: int = 0) -> None:
    """In-place implicit source-term update of one grid (see include/rhd.h).

    ``state`` holds CUDA float64 tensors: rho [n], mom [3, n], egas [n],
    kappa0 [n] or None, erad [G, n], frad [3, G, n], src [G, n] or None.
    ``law`` has nu_break, seg_logk, seg_beta, nu_ref (piecewise powerlaw)."""
    rho = state["rho"]
    n = rho.shape[0] if n_cells is None else n_cells
    e = np.ascontiguousarray(edges, dtype=np.float64)
    G = len(e) - 1
    gs = group_stride or rho.shape[0]
    st = _state(state, G, n, gs, c_v=c_v, consts=consts, theta=theta, precision=precision,
                closure=closure, tol=tol, tol_outer=tol_outer, max_newton=max_newton,
                max_outer=max_outer, status=status, iters=iters, flags=flags)
    gr = Groups(G, _dp(e))
    lw, keep = make_law(law, mode, khat_g, alpha_g, temp_exponent, T_ref)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().rhd_source_update(ctypes.byref(st), ctypes.byref(gr), ctypes.byref(lw), float(dt),
                                 int(n), ctypes.c_void_p(s.cuda_stream))
    del keep
    if rc != 0:
        raise RhdError(rc, lib().rhd_strerror(rc).decode())


def imex_step(state: dict, edges, law, *, dt: float, c_v: float, consts: dict,
              precision: int = FP64, closure: int = M1, tol: float = 0.0,
              tol_outer: float = 0.0, max_newton: int = 0, max_outer: int = 0,
              status: torch.Tensor | None = None, iters: torch.Tensor | None = None,
              mode: int = PPL_FIXED, khat_g=None, alpha_g=None, temp_exponent: float = 0.0,
              T_ref: float = 1.0, stream: torch.cuda.Stream | None = None, flags: int = 0) -> None:
    """``rhd_imex_step``: one step of the two-stage IMEX integrator without
    transport (stage 1 theta = 1, stage 2 theta = 1/2 from the average of the
    start and stage 1); same arguments as ``source_update``; a ``src`` entry is
    refused by the library (RhdError)."""
    rho = state["rho"]
    n = rho.shape[0]
    e = np.ascontiguousarray(edges, dtype=np.float64)
    G = len(e) - 1
    st = _state(state, G, n, n, c_v=c_v, consts=consts, theta=1.0, precision=precision,
                closure=closure, tol=tol, tol_outer=tol_outer, max_newton=max_newton,
                max_outer=max_outer, status=status, iters=iters, flags=flags)
    gr = Groups(G, _dp(e))
    lw, keep = make_law(law, mode, khat_g, alpha_g, temp_exponent, T_ref)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().rhd_imex_step(ctypes.byref(st), ctypes.byref(gr), ctypes.byref(lw), float(dt),
                             int(n), ctypes.c_void_p(s.cuda_stream))
    del keep
    if rc != 0:
        raise RhdError(rc, lib().rhd_strerror(rc).decode())


def source_update_host(state: dict, edges, law, *, dt: float, c_v: float, consts: dict,
                       theta: float = 1.0, precision: int = FP64, closure: int = M1,
                       tol: float = 0.0, tol_outer: float = 0.0, max_newton: int = 0,
                       max_outer: int = 0, status: torch.Tensor | None = None,
                       iters: torch.Tensor | None = None, mode: int = PPL_FIXED, khat_g=None,
                       alpha_g=None, temp_exponent: float = 0.0, T_ref: float = 1.0,
                       flags: int = 0, surrogate: "Surrogate | None" = None,
                       chunk_cells: int = 0) -> None:
    """``rhd_source_update_host``: the update of a grid whose tensors live in
    host memory (CPU float64 tensors, pinned for overlapped copies; same layout
    as ``source_update``), in chunks streamed through the GPU; with a
    ``surrogate`` each chunk starts from its guess.  Synchronous."""
    rho = state["rho"]
    n = rho.shape[0]
    e = np.ascontiguousarray(edges, dtype=np.float64)
    G = len(e) - 1
    st = _state(state, G, n, n, c_v=c_v, consts=consts, theta=theta, precision=precision,
                closure=closure, tol=tol, tol_outer=tol_outer, max_newton=max_newton,
                max_outer=max_outer, status=status, iters=iters, flags=flags, device="cpu")
    gr = Groups(G, _dp(e))
    lw, keep = make_law(law, mode, khat_g, alpha_g, temp_exponent, T_ref)
    h = surrogate._h if surrogate is not None else None
    rc = lib().rhd_source_update_host(ctypes.byref(st), ctypes.byref(gr), ctypes.byref(lw),
                                      float(dt), int(n), h, int(chunk_cells))
    del keep
    if rc != 0:
        raise RhdError(rc, lib().rhd_strerror(rc).decode())


def source_update_noalloc(state: dict, edges, law, *, dt: float, c_v: float, consts: dict,
                          theta: float = 1.0, closure: int = M1, tol: float = 0.0,
                          tol_outer: float = 0.0, max_newton: int = 0, max_outer: int = 0,
                          status: torch.Tensor | None = None, iters: torch.Tensor | None = None,
                          mode: int = PPL_FIXED, khat_g=None, alpha_g=None,
                          temp_exponent: float = 0.0, T_ref: float = 1.0,
                          stream: torch.cuda.Stream | None = None, flags: int = 0) -> None:
    """The mixed form through ``rhd_source_update_noalloc`` (no device
    allocation; the library's fixed 64 MiB device array holds the FP32 warm
    start).  Same arguments and layout as ``source_update``."""
    rho = state["rho"]
    n = rho.shape[0]
    e = np.ascontiguousarray(edges, dtype=np.float64)
    G = len(e) - 1
    _check(rho, "rho", (n,))
    _check(state["mom"], "mom", (3, n))
    _check(state["egas"], "egas", (n,))
    _check(state["erad"], "erad", (G, n))
    _check(state["frad"], "frad", (3, G, n))
    if state.get("kappa0") is not None:
        _check(state["kappa0"], "kappa0", (n,))
    if state.get("src") is not None:
        _check(state["src"], "src", (G, n))
    if status is not None:
        _check(status, "status", (n,), torch.uint8)
    if iters is not None:
        _check(iters, "iters", (n,), torch.uint8)
    st = State()
    st.rho = _ptr(rho)
    for d in range(3):
        st.mom[d] = _ptr(state["mom"][d])
        st.frad[d] = _ptr(state["frad"][d])
    st.egas = _ptr(state["egas"])
    st.kappa0 = _ptr(state.get("kappa0"))
    st.erad = _ptr(state["erad"])
    st.src = _ptr(state.get("src"))
    st.status = _ptr(status)
    st.iters = _ptr(iters)
    st.group_stride = n
    st.c_v, st.theta = float(c_v), float(theta)
    st.c, st.c_hat = float(consts["c"]), float(consts.get("c_hat", consts["c"]))
    st.a_rad, st.h, st.k_B = float(consts["a_rad"]), float(consts["h"]), float(consts["k_B"])
    st.tol, st.tol_outer = float(tol), float(tol_outer)
    st.max_newton, st.max_outer = int(max_newton), int(max_outer)
    st.precision, st.closure, st.flags = MIXED, int(closure), int(flags)
    gr = Groups(G, _dp(e))
    lw, keep = make_law(law, mode, khat_g, alpha_g, temp_exponent, T_ref)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().rhd_source_update_noalloc(ctypes.byref(st), ctypes.byref(gr), ctypes.byref(lw),
                                         float(dt), int(n), ctypes.c_void_p(s.cuda_stream))
    del keep
    if rc != 0:
        raise RhdError(rc, lib().rhd_strerror(rc).decode())


MAX_GROUPS_BATCHED = 64
HOST_CHUNK = 1 << 20  # default cells per chunk of rhd_source_update_host
MAX_GRIDS = 4096


def _raise(rc: int) -> None:
    if rc != 0:
        raise RhdError(rc, lib().rhd_strerror(rc).decode())


class GridSpec:
    """One grid of a batched call: the C descriptor plus the host arrays it
    points to (kept alive here)."""

    def __init__(self, state: dict, edges, law, *, dt: float, c_v: float, consts: dict,
                 theta: float = 1.0, precision: int = MIXED, closure: int = M1, tol: float = 0.0,
                 tol_outer: float = 0.0, max_newton: int = 0, max_outer: int = 0,
                 status: torch.Tensor | None = None, iters: torch.Tensor | None = None,
                 mode: int = PPL_FIXED, khat_g=None, alpha_g=None, temp_exponent: float = 0.0,
                 T_ref: float = 1.0, flags: int = 0):
        n = state["rho"].shape[0]
        e = np.ascontiguousarray(edges, dtype=np.float64)
        G = len(e) - 1
        st = _state(state, G, n, n, c_v=c_v, consts=consts, theta=theta, precision=precision,
                    closure=closure, tol=tol, tol_outer=tol_outer, max_newton=max_newton,
                    max_outer=max_outer, status=status, iters=iters, flags=flags)
        lw, keep = make_law(law, mode, khat_g, alpha_g, temp_exponent, T_ref)
        self.keep = keep + [e]
        self.state = state
        self.c = Grid(st, Groups(G, _dp(e)), lw, float(dt), int(n))


BATCH_BUCKETS = 3  # RHD_BATCH_BUCKETS: group counts 1..16, 17..32, 33..64
# the mappings each bucket offers, as lanes per cell (1: one cell per thread;
# passes 0: the one-grid call's mapping for the call's precision)
PASS_MAPPINGS = ((0, 1, 8), (0, 1, 8, 16, 32), (0, 1, 16, 32))
CORRECTION_MAPPINGS = ((8,), (8, 16), (16, 32))


class Context:
    """A batched-update context (``rhd_context_t``): staging buffers, the
    captured CUDA graph, the per-bucket mappings and the tuned launch shape,
    reused across calls."""

    def __init__(self):
        h = _P()
        _raise(lib().rhd_context_create(ctypes.byref(h)))
        self._h = h

    def close(self) -> None:
        if self._h is not None and self._h.value:
            _raise(lib().rhd_context_destroy(self._h))
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _array(grids):
        arr = (Grid * len(grids))()
        for k, g in enumerate(grids):
            arr[k] = g.c
        return arr

    def update(self, grids: list, stream: torch.cuda.Stream | None = None) -> None:
        """In-place update of every grid in one persistent launch."""
        s = stream if stream is not None else torch.cuda.current_stream()
        arr = self._array(grids)
        _raise(lib().rhd_source_update_batched(self._h, arr, len(grids),
                                               ctypes.c_void_p(s.cuda_stream)))

    def autotune(self, grids: list, stream: torch.cuda.Stream | None = None) -> tuple[int, int]:
        """Time each bucket's mappings and the CTA shape on these grids (their
        state is left as it was) and keep the fastest; returns (threads,
        cells_per_item); ``mappings`` has the picked mappings."""
        s = stream if stream is not None else torch.cuda.current_stream()
        arr = self._array(grids)
        _raise(lib().rhd_context_autotune(self._h, arr, len(grids),
                                          ctypes.c_void_p(s.cuda_stream)))
        return self.shape

    @property
    def shape(self) -> tuple[int, int]:
        t, c = ctypes.c_int32(), ctypes.c_int32()
        _raise(lib().rhd_context_shape(self._h, ctypes.byref(t), ctypes.byref(c)))
        return t.value, c.value

    def mapping(self, bucket: int) -> tuple[int, int]:
        """(passes, correction) lanes per cell of bucket ``bucket``."""
        p, c = ctypes.c_int32(), ctypes.c_int32()
        _raise(lib().rhd_context_mapping(self._h, bucket, ctypes.byref(p), ctypes.byref(c)))
        return p.value, c.value

    def set_mapping(self, bucket: int, passes: int, correction: int) -> None:
        _raise(lib().rhd_context_set_mapping(self._h, bucket, passes, correction))

    @property
    def mappings(self) -> list[tuple[int, int]]:
        return [self.mapping(b) for b in range(BATCH_BUCKETS)]


class Surrogate:
    """The learned warm start (``rhd_surrogate_t``): a BF16 MLP on the tensor
    cores mapping a cell's state to a guess of its updated temperature and
    group energies.  All arrays are CUDA float32 tensors, row-major."""

    def __init__(self, n_groups: int, seed: int = 0, _handle=None):
        h = _handle
        if h is None:
            h = _P()
            _raise(lib().rhd_surrogate_create(int(n_groups), int(seed), ctypes.byref(h)))
        self._h = h
        self.n_groups = int(n_groups)
        nf, no, npar = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _raise(lib().rhd_surrogate_dims(h, ctypes.byref(nf), ctypes.byref(no), ctypes.byref(npar)))
        self.n_features, self.n_outputs, self.n_params = nf.value, no.value, npar.value

    def save(self, path: str) -> None:
        """``rhd_surrogate_save``: parameters and standardisation to a file."""
        _raise(lib().rhd_surrogate_save(self._h, os.fsencode(path)))

    def checkpoint(self, path: str) -> None:
        """``rhd_surrogate_checkpoint``: the network and its Adam state, so that
        a surrogate loaded from the file resumes training bit for bit."""
        _raise(lib().rhd_surrogate_checkpoint(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str) -> "Surrogate":
        """``rhd_surrogate_load``: a surrogate on the current device from a saved file."""
        h = _P()
        _raise(lib().rhd_surrogate_load(os.fsencode(path), ctypes.byref(h)))
        nf, no, npar = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _raise(lib().rhd_surrogate_dims(h, ctypes.byref(nf), ctypes.byref(no), ctypes.byref(npar)))
        return cls(no.value - 1, _handle=h)

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _raise(lib().rhd_surrogate_destroy(self._h))
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _s(stream):
        s = stream if stream is not None else torch.cuda.current_stream()
        return ctypes.c_void_p(s.cuda_stream)

    def _grid(self, state, edges, law, dt, c_v, consts, mode=PPL_FIXED):
        n = state["rho"].shape[0]
        e = np.ascontiguousarray(edges, dtype=np.float64)
        st = _state(state, len(e) - 1, n, n, c_v=c_v, consts=consts, theta=1.0, precision=FP64,
                    closure=M1, tol=0.0, tol_outer=0.0, max_newton=0, max_outer=0, status=None,
                    iters=None, flags=0)
        lw, keep = make_law(law, mode)
        return st, Groups(len(e) - 1, _dp(e)), lw, keep + [e], n

    def features(self, state, edges, law, *, dt, c_v, consts, stream=None) -> torch.Tensor:
        st, gr, lw, keep, n = self._grid(state, edges, law, dt, c_v, consts)
        x = torch.empty((n, self.n_features), dtype=torch.float32, device=state["rho"].device)
        _raise(lib().rhd_surrogate_features(self._h, ctypes.byref(st), ctypes.byref(gr),
                                            ctypes.byref(lw), float(dt), n, _ptr(x), self._s(stream)))
        del keep
        return x

    def warm_start(self, state, edges, law, *, dt, c_v, consts, stream=None):
        """``rhd_surrogate_warm_start``: the Newton start the warm-started
        update takes -- (E_int,0 [n] float64, R_g,0 / E_tot [G, n] float32)."""
        st, gr, lw, keep, n = self._grid(state, edges, law, dt, c_v, consts)
        dev = state["rho"].device
        eint = torch.empty(n, dtype=torch.float64, device=dev)
        r = torch.empty((len(edges) - 1, n), dtype=torch.float32, device=dev)
        _raise(lib().rhd_surrogate_warm_start(self._h, ctypes.byref(st), ctypes.byref(gr),
                                              ctypes.byref(lw), float(dt), n, _ptr(eint), _ptr(r),
                                              self._s(stream)))
        del keep
        return eint, r

    def targets(self, before, after, edges, law, *, dt, c_v, consts, stream=None) -> torch.Tensor:
        sa, gr, lw, keep, n = self._grid(before, edges, law, dt, c_v, consts)
        sb, _, _, keep2, n_after = self._grid(after, edges, law, dt, c_v, consts)
        if n_after != n:
            raise ValueError(f"before holds {n} cells, after {n_after}")
        y = torch.empty((n, self.n_outputs), dtype=torch.float32, device=before["rho"].device)
        _raise(lib().rhd_surrogate_targets(self._h, ctypes.byref(sa), ctypes.byref(sb),
                                           ctypes.byref(gr), ctypes.byref(lw), float(dt), n,
                                           _ptr(y), self._s(stream)))
        del keep, keep2
        return y

    def fit_normalization(self, x, y, stream=None) -> None:
        _check(x, "x", (x.shape[0], self.n_features), torch.float32)
        _check(y, "y", (x.shape[0], self.n_outputs), torch.float32)
        _raise(lib().rhd_surrogate_fit_normalization(self._h, _ptr(x), _ptr(y), x.shape[0],
                                                     self._s(stream)))

    def get_params(self, stream=None):
        dev = torch.device("cuda", torch.cuda.current_device())
        p = torch.empty(self.n_params, dtype=torch.float32, device=dev)
        nrm = torch.empty(2 * (self.n_features + self.n_outputs), dtype=torch.float32, device=dev)
        _raise(lib().rhd_surrogate_params(self._h, _ptr(p), _ptr(nrm), 0, self._s(stream)))
        return p, nrm

    def set_params(self, params=None, normalization=None, stream=None) -> None:
        if params is not None:
            _check(params, "params", (self.n_params,), torch.float32)
        if normalization is not None:
            _check(normalization, "normalization", (2 * (self.n_features + self.n_outputs),),
                   torch.float32)
        _raise(lib().rhd_surrogate_params(self._h, _ptr(params), _ptr(normalization), 1,
                                          self._s(stream)))

    def loss_grad(self, x, y, stream=None):
        _check(x, "x", (x.shape[0], self.n_features), torch.float32)
        _check(y, "y", (x.shape[0], self.n_outputs), torch.float32)
        loss = torch.zeros(1, dtype=torch.float32, device=x.device)
        grad = torch.empty(self.n_params, dtype=torch.float32, device=x.device)
        _raise(lib().rhd_surrogate_loss_grad(self._h, _ptr(x), _ptr(y), x.shape[0], _ptr(loss),
                                             _ptr(grad), self._s(stream)))
        return loss, grad

    def train_step(self, x, y, first, batch, mult, add, lr, loss=None, stream=None) -> None:
        _check(x, "x", (x.shape[0], self.n_features), torch.float32)
        _check(y, "y", (x.shape[0], self.n_outputs), torch.float32)
        if loss is not None:
            _check(loss, "loss", (1,), torch.float32)
        _raise(lib().rhd_surrogate_train_step(self._h, _ptr(x), _ptr(y), x.shape[0], int(first),
                                              int(batch), int(mult), int(add), float(lr),
                                              _ptr(loss), self._s(stream)))

    def predict(self, x, stream=None) -> torch.Tensor:
        _check(x, "x", (x.shape[0], self.n_features), torch.float32)
        y = torch.empty((x.shape[0], self.n_outputs), dtype=torch.float32, device=x.device)
        _raise(lib().rhd_surrogate_predict(self._h, _ptr(x), x.shape[0], _ptr(y), self._s(stream)))
        return y

    def error_flag(self) -> int:
        f = ctypes.c_int32()
        _raise(lib().rhd_surrogate_error(self._h, ctypes.byref(f)))
        return f.value

    def test_wait_timeout(self, on: bool) -> None:
        """Test support: make the tensor-core waits give up (see include/rhd.h)."""
        _raise(lib().rhd_surrogate_test_wait_timeout(self._h, 1 if on else 0))

    def source_update(self, state: dict, edges, law, *, dt: float, c_v: float, consts: dict,
                      theta: float = 1.0, precision: int = MIXED, closure: int = M1,
                      tol: float = 0.0, tol_outer: float = 0.0, max_newton: int = 0,
                      max_outer: int = 0, status=None, iters=None, mode: int = PPL_FIXED,
                      khat_g=None, alpha_g=None, temp_exponent: float = 0.0, T_ref: float = 1.0,
                      stream=None, flags: int = 0) -> None:
        """``rhd_source_update_warm``: the update of one grid started from this
        surrogate's guess (same arguments as ``source_update``)."""
        n = state["rho"].shape[0]
        e = np.ascontiguousarray(edges, dtype=np.float64)
        st = _state(state, len(e) - 1, n, n, c_v=c_v, consts=consts, theta=theta,
                    precision=precision, closure=closure, tol=tol, tol_outer=tol_outer,
                    max_newton=max_newton, max_outer=max_outer, status=status, iters=iters,
                    flags=flags)
        gr = Groups(len(e) - 1, _dp(e))
        lw, keep = make_law(law, mode, khat_g, alpha_g, temp_exponent, T_ref)
        _raise(lib().rhd_source_update_warm(self._h, ctypes.byref(st), ctypes.byref(gr),
                                            ctypes.byref(lw), float(dt), n, self._s(stream)))
        del keep


KERNEL_FP32, KERNEL_CORRECTION, KERNEL_FP64, KERNEL_INFERENCE, KERNEL_REFINE = 0, 1, 2, 3, 4
KERNEL_NAMES = ("fp32_passes", "correction", "fp64_passes", "inference", "refine")
EVENT_NAMES = ("cells32", "eval32", "outer32", "cellsc", "resid64", "step32", "finish64",
               "cells64", "eval64", "cached64", "outer64", "fluxnewton", "infer", "residdf",
               "stepdf")


def profile_start() -> None:
    """Start timing the solver launches of this thread's update calls."""
    _raise(lib().rhd_profile_start())


def profile_stop() -> tuple[int, float]:
    """(launches timed, their summed duration in ms) since profile_start."""
    n, ms = ctypes.c_int32(), ctypes.c_double()
    _raise(lib().rhd_profile_stop(ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def profile_kernel(kind: int) -> tuple[int, float]:
    """(launches, summed ms) of one kind of launch (KERNEL_*) at the last profile_stop."""
    n, ms = ctypes.c_int32(), ctypes.c_double()
    _raise(lib().rhd_profile_kernel(int(kind), ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def events_start() -> None:
    """Zero the device's event counters and count this thread's update calls."""
    _raise(lib().rhd_events_start())


def events_stop() -> dict:
    """Stop counting; {event name: count} (include/rhd.h, RHD_EV_*)."""
    buf = (ctypes.c_uint64 * len(EVENT_NAMES))()
    _raise(lib().rhd_events_stop(buf))
    return dict(zip(EVENT_NAMES, (int(x) for x in buf)))


def strerror(code: int) -> str:
    return lib().rhd_strerror(int(code)).decode()
