"""FP64 CPU oracle for the multigroup implicit source-term update.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It wraps the plain C
library built from ``oracle/rhd_oracle.c`` (see its header for what it
computes and which equations of He, Wibking & Krumholz 2024 each part follows).
It shares no code with the CUDA library and never imports it.

Parity status of each function (what pins it; the pins live in
``tests/test_oracle_pins.py``):

* ``planck_P`` / ``planck_Q`` / ``planck_band`` -- arbitrary-precision
  quadrature, the total-band sum rule, the switch-point continuity.
* ``ppl_mean_opacity`` -- quadrature of eq. chiQ for powerlaw opacity and
  spectrum; the PC reduction at alpha_chi = 0.
* ``group_table`` -- hand-evaluated laws; PC/PPL limits.
* ``ppl_free_slopes`` -- a hand-worked minmod example, the exact index of a
  binned powerlaw spectrum, the edge groups and undefined slopes.
* ``group_terms`` -- the analytic Planck mean of the pulse opacity (Sec. 4.2.3,
  the value printed there, and its printed T^-3.5 law at 2e7 K), chi_F = chi_0 in the PC case (after eq. chiDiff),
  the diffusion-limit invariant of eq. Fdiff; with free slopes, chi_E and chi_B
  of a binned powerlaw spectrum against quadrature of eq. chiQ, and chi_E =
  chi_B for E_g = b_g.
* ``closure`` -- the free-streaming and isotropic limits, trace = E.
* ``arrowhead_solve`` -- dense LU on random arrowheads.
* ``source_update`` -- conservation, v=0 equilibrium, grey reduction, linear
  relaxation closed form (also with a source term), the source entering only
  as E_g^(t) + S_g (eq. FGFR), the Doppler-test equilibrium temperature
  printed in Sec. 4.2.1, the moving equilibrium at c_hat = c and c/10, and the
  group flux spectrum against the angle integral eq. bbF.

``tests/test_oracle_mutants.py`` plants plausible mistakes in copies of this
package and checks that each one fails a pin.
* ``imex_step`` -- two ``source_update`` calls composed as eqs. imex1/imex2
  prescribe with no transport; pinned by the closed-form amplification
  1/(1 + lambda dt) of a small grey disequilibrium and by conservation.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rhd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "librhd_oracle.so")

CLOSURE_M1 = 0
CLOSURE_EDDINGTON = 1
PPL_FIXED = 0
PC = 1
PPL_FREE = 2


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build`` (plain gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(_SRC[:-2] + ".h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("c_hat", ctypes.c_double), ("a_rad", ctypes.c_double),
                ("h", ctypes.c_double), ("k_B", ctypes.c_double), ("c_v", ctypes.c_double),
                ("theta", ctypes.c_double), ("dt", ctypes.c_double),
                ("temp_exponent", ctypes.c_double), ("T_ref", ctypes.c_double),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("closure", ctypes.c_int32)]


class _Groups(ctypes.Structure):
    _fields_ = [("n_groups", ctypes.c_int32), ("edges", ctypes.POINTER(ctypes.c_double)),
                ("khat_minus", ctypes.POINTER(ctypes.c_double)),
                ("alpha", ctypes.POINTER(ctypes.c_double)),
                ("free_slopes", ctypes.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, dp, i32, i64 = ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_int64
        _lib.orc_planck_P.restype = d
        _lib.orc_planck_P.argtypes = [d]
        _lib.orc_planck_Q.restype = d
        _lib.orc_planck_Q.argtypes = [d]
        _lib.orc_planck_band.restype = d
        _lib.orc_planck_band.argtypes = [d, d]
        _lib.orc_ppl_mean_opacity.restype = d
        _lib.orc_ppl_mean_opacity.argtypes = [d, d, d, d]
        _lib.orc_group_table.restype = ctypes.c_int
        _lib.orc_group_table.argtypes = [i32, dp, i32, i32, dp, dp, dp, d, dp, dp]
        _lib.orc_group_terms.restype = None
        _lib.orc_group_terms.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_Groups), d, d,
                                         dp, dp, dp, dp, dp, dp, dp]
        _lib.orc_ppl_free_slopes.restype = None
        _lib.orc_ppl_free_slopes.argtypes = [i32, dp, dp, dp]
        _lib.orc_closure.restype = None
        _lib.orc_closure.argtypes = [i32, d, d, dp, dp]
        _lib.orc_arrowhead_solve.restype = None
        _lib.orc_arrowhead_solve.argtypes = [i32, d, dp, dp, dp, dp, dp]
        _lib.orc_dense_solve.restype = ctypes.c_int
        _lib.orc_dense_solve.argtypes = [i32, dp, dp, dp]
        _lib.orc_source_update.restype = ctypes.c_int
        _lib.orc_source_update.argtypes = [i64, ctypes.POINTER(_Params), ctypes.POINTER(_Groups),
                                           dp, dp, dp, dp, dp, dp, dp,
                                           ctypes.POINTER(ctypes.c_int32), dp,
                                           ctypes.POINTER(ctypes.c_int32), i32]
        _lib.orc_max_threads.restype = i32
        _lib.orc_max_threads.argtypes = []
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


@dataclass
class Params:
    """Physical constants and solver settings (units are the caller's)."""
    c: float = 2.99792458e10
    c_hat: float | None = None
    a_rad: float = 7.565723e-15
    h: float = 6.62607015e-27
    k_B: float = 1.380649e-16
    c_v: float = 1.0
    theta: float = 1.0
    dt: float = 1.0
    temp_exponent: float = 0.0
    T_ref: float = 1.0
    tol: float = 1e-14
    max_iter: int = 100
    closure: int = CLOSURE_M1

    def _c(self) -> _Params:
        return _Params(self.c, self.c if self.c_hat is None else self.c_hat, self.a_rad, self.h,
                       self.k_B, self.c_v, self.theta, self.dt, self.temp_exponent, self.T_ref,
                       self.tol, int(self.max_iter), int(self.closure))


@dataclass
class Groups:
    """Group edges and per-group opacity table (khat at the lower edge, slope).
    free_slopes: spectral indices of B_nu and E_nu from Appendix A instead of -1."""
    edges: np.ndarray
    khat_minus: np.ndarray
    alpha: np.ndarray
    free_slopes: bool = False
    _keep: list = field(default_factory=list, repr=False)

    def _c(self) -> _Groups:
        e, k, a = _f64(self.edges), _f64(self.khat_minus), _f64(self.alpha)
        self._keep = [e, k, a]
        return _Groups(len(k), _dp(e), _dp(k), _dp(a), int(bool(self.free_slopes)))


def planck_P(x: float) -> float:
    return lib().orc_planck_P(float(x))


def planck_Q(x: float) -> float:
    return lib().orc_planck_Q(float(x))


def planck_band(x0: float, x1: float) -> float:
    return lib().orc_planck_band(float(x0), float(x1))


def ppl_mean_opacity(chi_minus, alpha_chi, alpha_Q, r) -> float:
    return lib().orc_ppl_mean_opacity(float(chi_minus), float(alpha_chi), float(alpha_Q), float(r))


def ppl_free_slopes(edges, Q) -> np.ndarray:
    """alpha_Q,g of Appendix A (eqs. sg, minmod) from group values Q_g."""
    e, q = _f64(edges), _f64(Q)
    out = np.zeros(len(q))
    lib().orc_ppl_free_slopes(len(q), _dp(e), _dp(q), _dp(out))
    return out


def group_table(edges, mode, nu_break, seg_logk, seg_beta, nu_ref):
    """(khat_minus, alpha) per group from a piecewise-powerlaw opacity law
    (PPL_FREE shares the PPL_FIXED table; the slopes are the Groups' flag)."""
    if mode == PPL_FREE:
        mode = PPL_FIXED
    e = _f64(edges)
    ng = len(e) - 1
    nb, lk, be = _f64(nu_break), _f64(seg_logk), _f64(seg_beta)
    if len(nb) == 0:
        nb = np.zeros(1)
    km, al = np.zeros(ng), np.zeros(ng)
    rc = lib().orc_group_table(ng, _dp(e), int(mode), len(lk), _dp(nb), _dp(lk), _dp(be),
                               float(nu_ref), _dp(km), _dp(al))
    if rc != 0:
        raise ValueError("orc_group_table rejected the law or the edges")
    return km, al


def group_terms(params: Params, groups: Groups, chi0_scale: float, T: float,
                erad0=None) -> dict:
    """b_g, Delta terms and the mean opacities at T; erad0 sets chi_E's slopes
    when groups.free_slopes."""
    ng = len(groups.khat_minus)
    out = {k: np.zeros(ng) for k in ("b", "dnb", "dnxb", "chiB", "chiE", "chiF")}
    pc, gc = params._c(), groups._c()
    e0 = None if erad0 is None else _f64(erad0)
    lib().orc_group_terms(ctypes.byref(pc), ctypes.byref(gc), float(chi0_scale), float(T),
                          None if e0 is None else _dp(e0),
                          _dp(out["b"]), _dp(out["dnb"]), _dp(out["dnxb"]), _dp(out["chiB"]),
                          _dp(out["chiE"]), _dp(out["chiF"]))
    return out


def closure(kind: int, c: float, E: float, F) -> np.ndarray:
    f = _f64(F)
    P = np.zeros(9)
    lib().orc_closure(int(kind), float(c), float(E), _dp(f), _dp(P))
    return P.reshape(3, 3)


def arrowhead_solve(a00, top, left, diag, rhs) -> np.ndarray:
    top, left, diag, rhs = _f64(top), _f64(left), _f64(diag), _f64(rhs)
    x = np.zeros(len(rhs))
    lib().orc_arrowhead_solve(len(top), float(a00), _dp(top), _dp(left), _dp(diag), _dp(rhs),
                              _dp(x))
    return x


def dense_solve(A, b) -> np.ndarray:
    A = _f64(A).copy()
    b = _f64(b).copy()
    x = np.zeros(len(b))
    if lib().orc_dense_solve(len(b), _dp(A), _dp(b), _dp(x)) != 0:
        raise np.linalg.LinAlgError("singular matrix")
    return x


def max_threads() -> int:
    return int(lib().orc_max_threads())


def source_update(state: dict, params: Params, groups: Groups, n_threads: int = 0) -> dict:
    """Solve the coupled implicit system for every cell of ``state``.

    ``state`` holds host arrays in the SoA layout: rho [n], mom [3, n], egas [n],
    kappa0 [n] or None, erad [G, n], frad [3, G, n], src [G, n] or None.
    Returns a new dict with the updated mom, egas, erad, frad and the per-cell
    iters, resid and status (0 converged, 2 not converged, 3 invalid input).
    """
    rho = _f64(state["rho"])
    n = rho.shape[0]
    ng = len(groups.khat_minus)
    mom = _f64(state["mom"]).copy()
    egas = _f64(state["egas"]).copy()
    erad = _f64(state["erad"]).copy()
    frad = _f64(state["frad"]).copy()
    assert mom.shape == (3, n) and erad.shape == (ng, n) and frad.shape == (3, ng, n)
    k0 = state.get("kappa0")
    k0 = None if k0 is None else _f64(k0)
    src = state.get("src")
    src = None if src is None else _f64(src)
    iters = np.zeros(n, dtype=np.int32)
    resid = np.zeros(n)
    status = np.zeros(n, dtype=np.int32)
    pc, gc = params._c(), groups._c()
    null = ctypes.POINTER(ctypes.c_double)()
    rc = lib().orc_source_update(
        n, ctypes.byref(pc), ctypes.byref(gc), _dp(rho), _dp(mom), _dp(egas),
        _dp(k0) if k0 is not None else null, _dp(erad), _dp(frad),
        _dp(src) if src is not None else null,
        iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(resid),
        status.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(n_threads))
    if rc != 0:
        raise ValueError("orc_source_update rejected its arguments")
    return {"mom": mom, "egas": egas, "erad": erad, "frad": frad, "iters": iters,
            "resid": resid, "status": status}


def imex_step(state: dict, p: "Params", g: "Groups", n_threads: int = 0) -> dict:
    """One step of the two-stage IMEX integrator (Sec. 3, eqs. imex1, imex2)
    without transport: stage 1 is the implicit source update over dt with
    theta = 1 from U(n); stage 2 starts from U(n) + (dt/2) S(U(n+1/2)) =
    (U(n) + U(n+1/2))/2 -- with no transport dt S(U(n+1/2)) = U(n+1/2) - U(n)
    by stage 1 -- and makes the implicit update with theta = 1/2.  Returns the
    final state with ``status`` the worse of the two stages."""
    import dataclasses
    if state.get("src") is not None:
        raise ValueError("imex_step takes no source term")
    s1 = source_update(state, dataclasses.replace(p, theta=1.0), g, n_threads=n_threads)
    mid = dict(state)
    for k in ("egas", "mom", "erad", "frad"):
        mid[k] = 0.5 * (np.asarray(state[k], dtype=np.float64) + s1[k])
    s2 = source_update(mid, dataclasses.replace(p, theta=0.5), g, n_threads=n_threads)
    s2["status"] = np.maximum(s1["status"], s2["status"])
    return s2
