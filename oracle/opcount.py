"""Operation counts of the per-cell implicit source-term update.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module; it shares no code
with the CUDA library and never imports it.  ``python -m oracle.opcount``
writes ``tests/golden/opcounts.json``, the per-event counts the benchmark's
roofline reads as data.

What is counted.  The update of one cell is written out plainly, in the
order of He, Wibking & Krumholz (2024), Sec. 3, on a counting number type:
every operation on a ``Num`` adds one to a tally of its kind (add -- sub
included --, mul, fma, div, sqrt, exp -- expm1 included --, cmp -- compares,
min, max) and of its precision.  The events are

* ``eval64``: one full evaluation of the inner system at an iterate -- the
  edge Planck terms (a4), the mean opacities of eqs. chiQg/chiDiff (a5), the
  residual of eq. FGFR with R_g of eq. Rnew (a6), the convergence test (a8)
  and the arrowhead elimination of eq. matrix with the Newton step (a7);
* ``outer64``: one outer pass -- the conservative write-back (a9), the flux
  update of eq. numF1 with the closure (a10), the momentum update of eq.
  vupdate (a11) and the outer test (a12);
* ``eval32`` / ``outer32``: the same two in FP32 (the mixed form's first
  phase);
* ``resid64``: one FP64 evaluation of the residual of the fully coupled
  system (inner rows and the flux rows of eq. fupdate) with the paper's two
  tests on it (the mixed form's correction step);
* ``step32``: one Newton step on the coupled system in FP32 -- the Jacobian
  of every group's four rows, the elimination of each group's block, the
  4 x 4 system of the cell, the step;
* ``finish64``: the end of a converged cell -- each R_g from its own row, the
  flux update, the conservative write-back of E_g, E_gas and the momentum;
* ``residdf`` / ``stepdf``: the first Newton step of the correction with the
  coupled residual evaluated in float-float arithmetic (no tests: that step
  decides nothing) and the same FP32 step as ``step32``.  Its operations are
  the FP64 residual's, tallied under the precision ``df``; ``DF_FP32_OPS``
  gives the FP32 operations each float-float operation takes with the
  error-free transformations it is built from (Knuth's two-sum: 6 additions;
  Dekker's fast two-sum: 3; a product's error by one FMA) in the "sloppy"
  double-double forms of Hida, Li & Bailey (2001).

Each event is counted as a part per group plus a part per cell, so a count
per cell-group follows for any N_g: ``per_cell_group(event, G)``.  Special
functions are charged as the operations a method of stated accuracy takes:
the Planck fraction P(x) (or its complement Q) as a degree-13 polynomial in
the argument on the segment of x plus its prefactors (the accuracy of such a
polynomial, 3e-16, is pinned in ``tests/test_planck_table.py``), x/(e^x - 1)
and e^-x from one expm1 and one division; everything else is counted as
written.

Parity status: the counting model is a working solver -- the paper's
inner/outer iteration and the coupled Newton correction written on ``Num`` --
and is pinned by reaching the oracle's root (``tests/test_oracle_opcount.py``),
by counts that are exactly linear in N_g (the O(N_g) cost of eq. matrix), and
by hand counts of small kernels (an arrowhead of two groups, one Horner step).
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import planck_P, planck_Q

KINDS = ("add", "mul", "fma", "div", "sqrt", "exp", "cmp")
PRECS = ("f64", "f32", "df")

# FP32 operations of one float-float operation (hi + lo, ~48 bits):
#   add  a + b: two-sum of the high words (6), the low words added to its
#        error (2), fast two-sum renormalisation (3);
#   mul  a b: the high product and its error by FMA (1 mul, 1 fma), the cross
#        terms (2 fma), fast two-sum (3 add);
#   fma  a b + c: a mul then an add;
#   div  a / b: FP32 reciprocal of b's high word (1 div), first quotient
#        (1 mul), its exact product with b (1 mul, 1 fma), the remainder
#        (3 add, 1 fma), the correction (1 mul), fast two-sum (3 add);
#   sqrt FP32 square root (1 sqrt), its exact square (1 mul, 1 fma), the
#        remainder (3 add), one Newton correction over 2 s (1 div, 1 mul),
#        fast two-sum (3 add);
#   exp  expm1 with Cody & Waite's reduction s = k ln 2 + r (ln 2 in three
#        parts: 4 mul, 1 fma, 32 add), the Taylor series of expm1(r) to r^13
#        (six terms in FP32: 6 fma; six in float-float: 6 mul + 6 add), its
#        assembly r + r^2 S (2 mul, 1 add) and the scaling by 2^k with
#        e^s = 2^k (expm1(r) + 1) beside it (4 mul, 2 add);
#   cmp  high words, then low words on a tie: 2 compares.
_DF_ADD = {"add": 11}
_DF_MUL = {"mul": 1, "fma": 3, "add": 3}


def _df_sum(*parts):
    out = {k: 0 for k in KINDS}
    for n, p in parts:
        for k, v in p.items():
            out[k] += n * v
    return out


DF_FP32_OPS = {
    "add": _df_sum((1, _DF_ADD)),
    "mul": _df_sum((1, _DF_MUL)),
    "fma": _df_sum((1, _DF_MUL), (1, _DF_ADD)),
    "div": _df_sum((1, {"div": 1, "mul": 3, "fma": 2, "add": 6})),
    "sqrt": _df_sum((1, {"sqrt": 1, "div": 1, "mul": 2, "fma": 1, "add": 6})),
    "exp": _df_sum((1, {"mul": 4, "fma": 1, "add": 32}), (6, {"fma": 1}),
                   (6, _DF_MUL), (6, _DF_ADD), (2, _DF_MUL), (1, _DF_ADD),
                   (4, {"mul": 1}), (2, _DF_ADD)),
    "cmp": _df_sum((1, {"cmp": 2})),
}
K15 = 15.0 / math.pi ** 4
PLANCK_DEGREE = 13


class Tally:
    """Counts of operations by (precision, kind)."""

    def __init__(self):
        self.c = {p: {k: 0 for k in KINDS} for p in PRECS}
        self.remap = {}  # precision -> precision it is tallied under

    def add(self, prec: str, kind: str, n: int = 1):
        self.c[self.remap.get(prec, prec)][kind] += n

    def snapshot(self) -> dict:
        return {p: dict(v) for p, v in self.c.items()}

    @staticmethod
    def diff(a: dict, b: dict) -> dict:
        return {p: {k: b[p][k] - a[p][k] for k in KINDS} for p in a}


TALLY = Tally()


def _v(x):
    return x.v if isinstance(x, Num) else float(x)


class Num:
    """A float whose operations are tallied; ``p`` is its precision tag."""
    __slots__ = ("v", "p")

    def __init__(self, v, p="f64"):
        self.v = float(v)
        self.p = p

    def _op(self, kind, v):
        TALLY.add(self.p, kind)
        return Num(v, self.p)

    def __add__(self, o):
        return self._op("add", self.v + _v(o))

    __radd__ = __add__

    def __sub__(self, o):
        return self._op("add", self.v - _v(o))

    def __rsub__(self, o):
        return self._op("add", _v(o) - self.v)

    def __mul__(self, o):
        return self._op("mul", self.v * _v(o))

    __rmul__ = __mul__

    def __truediv__(self, o):
        return self._op("div", self.v / _v(o))

    def __rtruediv__(self, o):
        return self._op("div", _v(o) / self.v)

    def __neg__(self):
        return Num(-self.v, self.p)  # a sign flip folds into the next operation

    def __abs__(self):
        return Num(abs(self.v), self.p)  # folds likewise

    def __lt__(self, o):
        TALLY.add(self.p, "cmp")
        return self.v < _v(o)

    def __le__(self, o):
        TALLY.add(self.p, "cmp")
        return self.v <= _v(o)

    def __gt__(self, o):
        TALLY.add(self.p, "cmp")
        return self.v > _v(o)

    def __ge__(self, o):
        TALLY.add(self.p, "cmp")
        return self.v >= _v(o)

    def __float__(self):
        return self.v


def N(x, p="f64"):
    return x if isinstance(x, Num) else Num(x, p)


def fma(a, b, c):
    a = N(a)
    TALLY.add(a.p, "fma")
    return Num(_v(a) * _v(b) + _v(c), a.p)


def sqrt(a):
    TALLY.add(a.p, "sqrt")
    return Num(math.sqrt(a.v), a.p)


def expm1(a):
    TALLY.add(a.p, "exp")
    return Num(math.expm1(a.v) if a.v < 700 else math.inf, a.p)


def vmin(a, b):
    TALLY.add(a.p, "cmp")
    return a if a.v <= _v(b) else N(b, a.p)


def vmax(a, b):
    TALLY.add(a.p, "cmp")
    return a if a.v >= _v(b) else N(b, a.p)


def dot3(a, b):
    return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]))


# ---------------------------------------------------------------------------
# a4: edge Planck terms
# ---------------------------------------------------------------------------
def edge_terms(xe: float, invT: Num):
    """P or Q, D = (15/pi^4) x^4/(e^x-1) and x D'(x) at one edge x = xe / T.
    x < 2 gives P (low), else Q = 1 - P (no 1 - 1 cancellation in the
    Wien tail).  Values from the oracle's series; the operations charged are
    those of the polynomial method (see the module docstring)."""
    p = invT.p
    x = invT * xe
    if not (x.v > 0.0) or math.isinf(x.v):
        return Num(0.0, p), x.v < 2.0, Num(0.0, p), Num(0.0, p)
    em = expm1(x)
    ep = em + 1.0
    r = 1.0 / (em * ep)               # one reciprocal serves x/(e^x-1) and e^-x
    xr = x * ep * r
    emx = em * r
    x3 = x * x * x
    d = x3 * xr * K15
    ed = d * (4.0 - xr - x)
    low = x < 2.0
    # the polynomial: the argument on its segment, Horner, the prefactors
    u = (x - 1.0) * 1.0
    acc = N(0.0, p)
    for _ in range(PLANCK_DEGREE):
        acc = fma(acc, u, 1.0)
    pq = x3 * acc * K15 * (1.0 if low else emx)
    pq = Num(planck_P(x.v) if low else planck_Q(x.v), p)
    return pq, low, d, ed


def band(pqL, lowL, pqU, lowU):
    if not lowL:
        return pqL - pqU
    if lowU:
        return pqU - pqL
    return (1.0 - pqU) - pqL


# ---------------------------------------------------------------------------
# one cell
# ---------------------------------------------------------------------------
@dataclass
class Cell:
    """Inputs of one cell (host floats) and its iterate (Num)."""
    rho: float
    mom0: np.ndarray
    egas0: float
    kappa0: float
    E0: np.ndarray          # E_g^t + S_g
    Ft: np.ndarray          # [3][G]
    edges: np.ndarray
    kbar: np.ndarray        # chi_E / (rho kappa0), eq. chiQg with alpha_Q = -1
    alpha: np.ndarray
    rm: np.ndarray          # chi_0 at the lower edge / chi_E
    rp: np.ndarray          # chi_0 at the upper edge / chi_E
    c: float
    c_hat: float
    a_rad: float
    h_over_k: float
    c_v: float
    theta: float
    dt: float
    p: str = "f64"
    Eint: Num = None
    R: list = field(default_factory=list)
    F: list = field(default_factory=list)   # [G][3]
    m: list = field(default_factory=list)
    w: list = field(default_factory=list)   # v.F_g / c^2, frozen for an outer pass (a3)
    tau: list = field(default_factory=list)  # c_hat theta dt chi_E,g, 1/tau, tau/(1+tau)
    itau: list = field(default_factory=list)
    qe: list = field(default_factory=list)
    KE: Num = None
    newton: int = 0
    outer: int = 0

    @property
    def G(self):
        return len(self.E0)


def make_cell(state: dict, i: int, params, groups, p="f64") -> Cell:
    """Cell i of a host SoA state (the oracle's input layout)."""
    e = np.asarray(groups.edges, float)
    lr = np.log(e[1:] / e[:-1])
    al = np.asarray(groups.alpha, float)
    z = al * lr
    mf = np.where(np.abs(z) < 1e-6, 1.0 + 0.5 * z, np.expm1(z) / np.where(z == 0.0, 1.0, z))
    src = 0.0 if state.get("src") is None else state["src"][:, i]
    cell = Cell(rho=float(state["rho"][i]), mom0=state["mom"][:, i].copy(),
                egas0=float(state["egas"][i]),
                kappa0=1.0 if state.get("kappa0") is None else float(state["kappa0"][i]),
                E0=state["erad"][:, i] + src, Ft=state["frad"][:, :, i].copy(), edges=e,
                kbar=np.asarray(groups.khat_minus) * mf, alpha=al, rm=1.0 / mf,
                rp=np.exp(z) / mf, c=params.c, c_hat=params.c if params.c_hat is None else params.c_hat,
                a_rad=params.a_rad, h_over_k=params.h / params.k_B, c_v=params.c_v,
                theta=params.theta, dt=params.dt, p=p)
    G = cell.G
    ke = 0.5 * float(cell.mom0 @ cell.mom0) / cell.rho
    cell.Eint = Num(cell.egas0 - ke, p)
    cell.R = [Num(0.0, p) for _ in range(G)]
    cell.F = [[Num(cell.Ft[d, g], p) for d in range(3)] for g in range(G)]
    cell.m = [Num(cell.mom0[d], p) for d in range(3)]
    return cell


def setup(cell: Cell):
    """Per update: tau_g = c_hat theta dt chi_E,g with its reciprocal and
    tau/(1 + tau) = -1/e_g of eq. matrix (a2 with the cell's rho kappa0)."""
    tdt, cs, _ = _consts(cell)
    tcs = N(tdt * cs, cell.p)
    cell.tau = [tcs * cell.kbar[g] for g in range(cell.G)]
    cell.itau = [1.0 / t for t in cell.tau]
    cell.qe = [t / (t + 1.0) for t in cell.tau]


def _consts(cell: Cell):
    tdt = cell.c_hat * cell.theta * cell.dt
    cs = cell.rho * cell.kappa0
    etot = cell.egas0 + cell.c / cell.c_hat * float(np.sum(cell.E0))
    return tdt, cs, etot


def chi_f_ratio(b, aT4, dD, a, rm, rp, dL, dU):
    """eq. chiDiff as chi_F / chi_E, held to the group's range of chi_0."""
    X = rp * dU - rm * dL
    den = b * (4.0 / 3.0) - aT4 * dD * (1.0 / 3.0)
    q = N(1.0, b.p)
    if den > 0.0:
        q = (b * (4.0 / 3.0) + (a * b - aT4 * X) * (1.0 / 3.0)) / den
    return vmin(vmax(q, min(rm, rp)), max(rm, rp)), X


def inner_eval(cell: Cell, tol: float):
    """One evaluation of the inner system at (E_int, R_g) with v, F frozen
    (a4-a8).  Returns 1 when the convergence test holds (then each R_g is set
    from its own row), 0 after a Newton step."""
    tdt, cs, etot = _consts(cell)
    G, p = cell.G, cell.p
    cr = cell.c / cell.c_hat
    rcv = cell.rho * cell.c_v
    T = cell.Eint * (1.0 / rcv)
    aT3 = T * T * T * cell.a_rad
    aT4 = aT3 * T
    invT = 1.0 / T
    eg = [edge_terms(cell.h_over_k * cell.edges[e], invT) for e in range(G + 1)]
    sumR = N(0.0, p)
    sFRe = N(0.0, p)
    sde = N(0.0, p)
    sabs = N(0.0, p)
    FR, dg, qe = [], [], []
    for g in range(G):
        pqL, lowL, dL, _ = eg[g]
        pqU, lowU, dU, _ = eg[g + 1]
        dP = band(pqL, lowL, pqU, lowU)
        dD = dU - dL
        b = aT4 * dP
        db = aT3 * (dP * 4.0 - dD)
        q, _ = chi_f_ratio(b, aT4, dD, cell.alpha[g], cell.rm[g], cell.rp[g], dL, dU)
        Eg = b + q * (1.0 + cell.alpha[g]) * cell.w[g] - cell.R[g] * cell.itau[g]  # eq. Rnew
        fr = Eg - cell.E0[g] - cell.R[g]                                     # eq. FGFR
        d = db * (1.0 / rcv)                                                 # dF_R,g / dE_gas
        ie = cell.qe[g]                                                      # -1 / e_g
        FR.append(fr)
        dg.append(d)
        qe.append(ie)
        sumR = sumR + cell.R[g]
        sFRe = sFRe - fr * ie
        sde = sde - d * ie
        sabs = sabs + abs(fr)
    FG = cell.Eint + cell.KE - cell.egas0 + sumR * cr
    if abs(FG) < tol * etot and sabs * cr < tol * etot:
        for g in range(G):
            cell.R[g] = fma(FR[g], qe[g], cell.R[g])
        return 1
    dE = (sFRe * cr - FG) / (1.0 - sde * cr)                                 # eq. matrix, first row
    lam = 1.0
    while not (cell.Eint + dE * lam > 0.0):                                  # damped while E_int <= 0
        lam *= 0.5
    cell.Eint = cell.Eint + dE * lam
    for g in range(G):
        cell.R[g] = cell.R[g] + fma(dg[g], dE, FR[g]) * qe[g] * lam          # its own row
    cell.newton += 1
    return 0


def pass_begin(cell: Cell):
    """a3: v, E_kin and w_g = v.F_g / c^2 frozen for an outer pass."""
    v = [cell.m[d] * (1.0 / cell.rho) for d in range(3)]
    cell.KE = dot3(cell.m, cell.m) * (0.5 / cell.rho)
    cell.w = [dot3(v, cell.F[g]) * (1.0 / cell.c ** 2) for g in range(cell.G)]


def cached_iteration(cell: Cell, FR: list, dg: list, tol: float):
    """cached64: an inner iteration from group terms kept from the last full
    evaluation (the pass after a converged inner solve starts at the same T
    and R_g, where each row's residual is its v.F term): the sums of eq.
    matrix, the convergence test and the Newton step, no group evaluation."""
    _, _, etot = _consts(cell)
    cr = cell.c / cell.c_hat
    sumR, sFRe, sde, sabs = N(0.0), N(0.0), N(0.0), N(0.0)
    for g in range(cell.G):
        sumR = sumR + cell.R[g]
        sFRe = sFRe - FR[g] * cell.qe[g]
        sde = sde - dg[g] * cell.qe[g]
        sabs = sabs + abs(FR[g])
    FG = cell.Eint + cell.KE - cell.egas0 + sumR * cr
    if abs(FG) < tol * etot and sabs * cr < tol * etot:
        return 1
    dE = (sFRe * cr - FG) / (1.0 - sde * cr)
    cell.Eint = cell.Eint + dE
    for g in range(cell.G):
        cell.R[g] = cell.R[g] + fma(dg[g], dE, FR[g]) * cell.qe[g]
    return 0


def closure_vP(cell: Cell, E, F, v):
    """v.P_g for the M1 closure (Levermore's chi in its rationalised form)."""
    c = cell.c
    fn2 = dot3(F, F)
    if not (E > 0.0 and fn2 > 0.0):   # no direction (or no energy): P = E/3 I
        return [E * v[d] * (1.0 / 3.0) for d in range(3)]
    cE = E * c
    cE2 = cE * cE
    vF = dot3(v, F)
    if fn2 < cE2:
        S = sqrt(cE2 * 4.0 - fn2 * 3.0)
        a = (S - cE) * (1.0 / (3.0 * c))
        k = vF * (3.0 / c) / (cE * 2.0 + S)
        return [fma(a, v[d], k * F[d]) for d in range(3)]
    k = E * vF / fn2
    return [k * F[d] for d in range(3)]


def outer_pass(cell: Cell, tol_outer: float, T: Num, terms: list):
    """a9-a12 after a converged inner solve; terms[g] = (b, q, dnx) at T.
    Returns True when the outer test holds."""
    tdt, cs, etot = _consts(cell)
    G, p = cell.G, cell.p
    cr = cell.c / cell.c_hat
    icc = 1.0 / (cell.c * cell.c_hat)
    v = [cell.m[d] * (1.0 / cell.rho) for d in range(3)]
    KE = cell.KE
    sumR = N(0.0, p)
    for g in range(G):
        sumR = sumR + cell.R[g]
    egas = cell.egas0 - sumR * cr                                            # a9
    dF = [N(0.0, p) for _ in range(3)]
    Fn_all = []
    for g in range(G):
        b, q, dnx = terms[g]
        chiB = cs * cell.kbar[g]
        E = cell.R[g] + cell.E0[g]
        vp = closure_vP(cell, E, cell.F[g], v)
        srcg = (b - dnx * (1.0 / 3.0)) * chiB
        inv = 1.0 / (q * (tdt * chiB) + 1.0)
        kap = inv * (tdt * (1.0 + cell.alpha[g]) * chiB)
        Fn = [fma(kap, vp[d], (srcg * v[d] * tdt + cell.Ft[d, g]) * inv) for d in range(3)]  # eq. numF1
        for d in range(3):
            dF[d] = dF[d] + Fn[d] - cell.Ft[d, g]
        Fn_all.append(Fn)
    mn = [cell.mom0[d] - dF[d] * icc for d in range(3)]                      # eq. vupdate
    vn = [mn[d] * (1.0 / cell.rho) for d in range(3)]
    KEn = dot3(mn, mn) * (0.5 / cell.rho)
    chg = abs(KEn - KE)
    for g in range(G):
        _, q, _ = terms[g]
        wn = dot3(vn, Fn_all[g]) * (1.0 / cell.c ** 2)
        chg = chg + abs((wn - cell.w[g]) * q * (1.0 + cell.alpha[g])) * cell.qe[g]
    cell.F = Fn_all
    cell.m = mn
    cell.outer += 1
    done = chg <= tol_outer * etot
    cell.Eint = egas - KEn
    if not done:
        pass_begin(cell)
    return done, egas


def group_terms_at(cell: Cell, T: Num):
    """(b_g, chi_F/chi_E, (4pi/c) Delta_g(nu chi_0 B)/chi_E) at T, uncounted
    helper of the outer pass (the inner evaluation at the same T computed them)."""
    saved = TALLY.snapshot()
    aT4 = T * T * T * T * cell.a_rad
    invT = 1.0 / T
    eg = [edge_terms(cell.h_over_k * cell.edges[e], invT) for e in range(cell.G + 1)]
    out = []
    for g in range(cell.G):
        pqL, lowL, dL, _ = eg[g]
        pqU, lowU, dU, _ = eg[g + 1]
        b = aT4 * band(pqL, lowL, pqU, lowU)
        q, X = chi_f_ratio(b, aT4, dU - dL, cell.alpha[g], cell.rm[g], cell.rp[g], dL, dU)
        out.append((b, q, aT4 * X))
    TALLY.c = {p: dict(v) for p, v in saved.items()}
    return out


def solve_paper(cell: Cell, tol=1e-11, tol_outer=1e-13, max_newton=64, max_outer=16):
    """The paper's inner/outer iteration for one cell (FP64 form); returns
    (converged, per-event tallies)."""
    ev = {"eval64": [], "outer64": []}
    t0 = TALLY.snapshot()
    setup(cell)
    pass_begin(cell)
    ev["outer64"].append(Tally.diff(t0, TALLY.snapshot()))
    for _ in range(max_outer):
        for _ in range(max_newton + 1):
            t0 = TALLY.snapshot()
            r = inner_eval(cell, tol)
            ev["eval64"].append(Tally.diff(t0, TALLY.snapshot()))
            if r == 1:
                break
        T = cell.Eint * (1.0 / (cell.rho * cell.c_v))
        terms = group_terms_at(cell, T)
        t0 = TALLY.snapshot()
        done, egas = outer_pass(cell, tol_outer, T, terms)
        ev["outer64"].append(Tally.diff(t0, TALLY.snapshot()))
        if done:
            cell.egas_final = egas
            return True, ev
    cell.egas_final = egas
    return False, ev


def result(cell: Cell) -> dict:
    """The cell's final state (host floats) in the oracle's output layout."""
    return {"egas": float(cell.egas_final), "mom": np.array([float(x) for x in cell.m]),
            "erad": np.array([cell.E0[g] + float(cell.R[g]) for g in range(cell.G)]),
            "frad": np.array([[float(cell.F[g][d]) for g in range(cell.G)] for d in range(3)])}


# ---------------------------------------------------------------------------
# per-event counts at a given N_g
# ---------------------------------------------------------------------------
def per_event_counts(state: dict, i: int, params, groups) -> dict:
    """Counts of one eval64 and one outer64 event of cell i (its first inner
    evaluation and first outer pass), split as kind -> count."""
    cell = make_cell(state, i, params, groups)
    setup(cell)
    pass_begin(cell)
    t0 = TALLY.snapshot()
    inner_eval(cell, 0.0)  # tol 0: always the full path (test failed, Newton step)
    e64 = Tally.diff(t0, TALLY.snapshot())["f64"]
    T = cell.Eint * (1.0 / (cell.rho * cell.c_v))
    terms = group_terms_at(cell, T)
    t0 = TALLY.snapshot()
    outer_pass(cell, 0.0, T, terms)
    o64 = Tally.diff(t0, TALLY.snapshot())["f64"]
    return {"eval64": e64, "outer64": o64}


def linear_fit(counts_by_G: dict) -> dict:
    """kind -> (per group, per cell) from counts at two or more N_g."""
    Gs = sorted(counts_by_G)
    out = {}
    for k in KINDS:
        y = np.array([counts_by_G[g][k] for g in Gs], float)
        A = np.vstack([np.array(Gs, float), np.ones(len(Gs))]).T
        sol, *_ = np.linalg.lstsq(A, y, rcond=None)
        out[k] = (float(sol[0]), float(sol[1]))
    return out


# ---------------------------------------------------------------------------
# the mixed form's correction: the fully coupled system (Sec. 3's fixed
# point) -- FP64 residual, FP32 Newton step, FP64 finish
# ---------------------------------------------------------------------------
def to_prec(x, p):
    return Num(_v(x), p)


def momentum_of(cell: Cell):
    """eq. vupdate for the current fluxes: m = m^t - (c c_hat)^-1 sum_g (F_g - F_g^t)."""
    icc = 1.0 / (cell.c * cell.c_hat)
    s = [N(0.0, "f64") for _ in range(3)]
    for g in range(cell.G):
        for d in range(3):
            s[d] = s[d] + (cell.F[g][d] - cell.Ft[d, g])
    return [fma(s[d], -icc, cell.mom0[d]) for d in range(3)]


def coupled_residual(cell: Cell, tol: float, tol_outer: float, m=None):
    """resid64: F_G, F_R,g (eqs. FGFR, Rnew) and F_F,g = F_g - (eq. numF1 at
    the iterate) in FP64, with v from the iterate's momentum, and the
    paper's two tests on them: the inner test, and the outer test on the
    change one more outer pass would make (to first order in it; its sums in
    FP32).  ``m``: the momentum when it is carried (else it is summed)."""
    tdt, cs, etot = _consts(cell)
    G = cell.G
    cr = cell.c / cell.c_hat
    c2 = cell.c ** 2
    m = momentum_of(cell) if m is None else m
    v = [m[d] * (1.0 / cell.rho) for d in range(3)]
    KE = dot3(m, m) * (0.5 / cell.rho)
    T = cell.Eint * (1.0 / (cell.rho * cell.c_v))
    aT3 = T * T * T * cell.a_rad
    aT4 = aT3 * T
    invT = 1.0 / T
    eg = [edge_terms(cell.h_over_k * cell.edges[e], invT) for e in range(G + 1)]
    sumR = N(0.0)
    FR, FF, terms = [], [], []
    for g in range(G):
        pqL, lowL, dL, _ = eg[g]
        pqU, lowU, dU, _ = eg[g + 1]
        b = aT4 * band(pqL, lowL, pqU, lowU)
        q, X = chi_f_ratio(b, aT4, dU - dL, cell.alpha[g], cell.rm[g], cell.rp[g], dL, dU)
        dnx = aT4 * X
        w = dot3(v, cell.F[g]) * (1.0 / c2)
        E = cell.E0[g] + cell.R[g]
        FR.append(b + q * (1.0 + cell.alpha[g]) * w - cell.R[g] * cell.itau[g] - E)
        chiB = cs * cell.kbar[g]
        vp = closure_vP(cell, E, cell.F[g], v)
        srcg = (b - dnx * (1.0 / 3.0)) * chiB
        inv = 1.0 / (q * (tdt * chiB) + 1.0)
        kap = inv * (tdt * (1.0 + cell.alpha[g]) * chiB)
        FF.append([cell.F[g][d] - fma(kap, vp[d], (srcg * v[d] * tdt + cell.Ft[d, g]) * inv)
                   for d in range(3)])
        sumR = sumR + cell.R[g]
        terms.append((q, dnx))
    FG = cell.Eint + KE - cell.egas0 + sumR * cr
    # the tests: FP32 sums of the scaled residuals
    sE = 1.0 / etot
    sabs = N(0.0, "f32")
    dm = [N(0.0, "f32") for _ in range(3)]
    for g in range(G):
        sabs = sabs + abs(to_prec(FR[g], "f32") * sE)
        for d in range(3):
            dm[d] = dm[d] + to_prec(FF[g][d], "f32") * sE
    icc = 1.0 / (cell.c * cell.c_hat)
    dv = [dm[d] * (etot * icc / cell.rho) for d in range(3)]    # the change of v
    vf = [to_prec(v[d], "f32") for d in range(3)]
    chg = abs(dot3([to_prec(m[d], "f32") for d in range(3)], dv) * sE)
    for g in range(G):
        dw = N(0.0, "f32")
        for d in range(3):
            Ff = to_prec(cell.F[g][d], "f32") * sE
            dF = to_prec(FF[g][d], "f32") * sE
            dw = dw + fma(dv[d], Ff - dF, -(vf[d] * dF))
        q32 = to_prec(terms[g][0], "f32")
        chg = chg + abs(q32 * (1.0 + cell.alpha[g]) * dw * (1.0 / c2)) * to_prec(cell.qe[g], "f32")
    passed = abs(FG) < tol * etot and sabs * cr < tol and chg <= tol_outer
    return passed, {"FG": FG, "FR": FR, "FF": FF, "m": m, "v": v, "T": T, "sumR": sumR}


def closure_jac(cell: Cell, E, F, v):
    """v.P, d(v.P)/dF (3x3), d(v.P)/dE and P (3x3), M1 closure (f held at 1)."""
    c = cell.c
    fn = sqrt(dot3(F, F))
    if not (fn.v > 0.0 and E.v > 0.0):
        e3 = E * (1.0 / 3.0)
        Pm = [[e3 if r == q else N(0.0, E.p) for q in range(3)] for r in range(3)]
        return [e3 * v[d] for d in range(3)], [[N(0.0, E.p)] * 3 for _ in range(3)], \
            [v[d] * (1.0 / 3.0) for d in range(3)], Pm
    f = fn / (E * c)
    held = f > 1.0
    if held:
        f = N(1.0, E.p)
    f2 = f * f
    sq = sqrt(4.0 - f2 * 3.0)
    num = f2 * 4.0 + 3.0
    den = sq * 2.0 + 5.0
    chi = num / den
    dchi = N(0.0, E.p) if held else (f * den * 8.0 + f * num * 6.0 / sq) / (den * den)
    iso = (1.0 - chi) * 0.5
    dr = chi * 1.5 - 0.5
    n = [F[d] / fn for d in range(3)]
    vn = dot3(v, n)
    a = dchi * (-0.5 / c)
    bb = dchi * vn * (1.5 / c)
    ee = E * dr / fn
    vp = [E * fma(dr * vn, n[r], iso * v[r]) for r in range(3)]
    M = [[fma(a, v[r] * n[q], fma(bb, n[r] * n[q], ee * (n[r] * (v[q] - vn * n[q])
                                                         + vn * ((1.0 if r == q else 0.0) - n[r] * n[q]))))
          for q in range(3)] for r in range(3)]
    ie = iso + f * dchi * 0.5
    de = dr - f * dchi * 1.5
    dE = [fma(ie, v[r], de * vn * n[r]) for r in range(3)]
    Pm = [[E * ((iso if r == q else 0.0) + dr * n[r] * n[q]) for q in range(3)] for r in range(3)]
    return vp, M, dE, Pm


def solve3(K, rhs):
    """K^-1 rhs for a 3x3 K by its adjugate (rhs: list of 3-vectors)."""
    a = [[K[r][q] for q in range(3)] for r in range(3)]
    co = [[a[(r + 1) % 3][(q + 1) % 3] * a[(r + 2) % 3][(q + 2) % 3]
           - a[(r + 1) % 3][(q + 2) % 3] * a[(r + 2) % 3][(q + 1) % 3] for q in range(3)]
          for r in range(3)]
    det = dot3(a[0], co[0])
    idet = 1.0 / det
    out = []
    for y in rhs:
        out.append([dot3([co[0][r], co[1][r], co[2][r]], y) * idet for r in range(3)])
    return out


def coupled_step(cell: Cell, res: dict):
    """step32: one Newton step on the coupled system, its Jacobian built and
    eliminated in FP32.  Each group's block (R_g, F_g) is eliminated through
    its R_g row and a 3x3 Schur complement with five right-hand sides (the
    residual, the E_int column, the three v columns); the group sums give a
    4x4 system in (dE_int, dv) -- the momentum relation dv = -(rho c
    c_hat)^-1 sum_g dF_g closes it -- then each group's step follows.  The
    step is added to the FP64 iterate."""
    tdt, cs, etot = _consts(cell)
    G, c = cell.G, cell.c
    cr = cell.c / cell.c_hat
    p = "f32"
    sE = 1.0 / etot
    sF = 1.0 / (c * etot)
    T = to_prec(res["T"], p)
    aT3 = T * T * T * cell.a_rad
    aT4 = aT3 * T
    invT = 1.0 / T
    rcv = cell.rho * cell.c_v
    eg = [edge_terms(cell.h_over_k * cell.edges[e], invT) for e in range(G + 1)]
    v = [to_prec(res["v"][d], p) for d in range(3)]
    blocks = []
    for g in range(G):
        pqL, lowL, dL, eL = eg[g]
        pqU, lowU, dU, eU = eg[g + 1]
        dP = band(pqL, lowL, pqU, lowU)
        dD = dU - dL
        b = aT4 * dP
        db = aT3 * (dP * 4.0 - dD)                      # d b_g / dT
        a, rm, rp = cell.alpha[g], cell.rm[g], cell.rp[g]
        X = rp * dU - rm * dL
        den = b * (4.0 / 3.0) - aT4 * dD * (1.0 / 3.0)
        dX = aT3 * (X * 4.0 - (rp * eU - rm * eL))
        q, dq = N(1.0, p), N(0.0, p)
        if den > 0.0:
            q = (b * (4.0 / 3.0) + (a * b - aT4 * X) * (1.0 / 3.0)) / den
            dq = ((db * (4.0 / 3.0) + (db * a - dX) * (1.0 / 3.0))
                  - q * (db * (4.0 / 3.0) - aT3 * (dD * 4.0 - (eU - eL)) * (1.0 / 3.0))) / den
        lo, hi = min(rm, rp), max(rm, rp)
        if q < lo or q > hi:
            dq = N(0.0, p)
            q = vmin(vmax(q, lo), hi)
        tau = to_prec(cell.tau[g], p)
        chiB = cs * cell.kbar[g]
        inv = 1.0 / (q * tau + 1.0)
        kap = inv * tau * (1.0 + a)
        srcs = b - aT4 * X * (1.0 / 3.0)                 # (chi_B b - delta chi / 3) / chi_B
        dsrc = db - dX * (1.0 / 3.0)
        E = to_prec(cell.E0[g] + cell.R[g].v, p)
        F = [to_prec(cell.F[g][d], p) for d in range(3)]
        vp, M, dE, Pm = closure_jac(cell, E, F, v)
        a1 = q * (1.0 + a)
        w = dot3(v, F) * (1.0 / c ** 2)
        # rows scaled: F_R by E_tot, F_F by c E_tot; unknowns r = dR/E_tot,
        # f = dF/(c E_tot), x = dE_int/E_tot, beta = dv/c
        A00 = -(to_prec(cell.itau[g], p) + 1.0)
        A0 = [a1 * v[d] * (1.0 / c) for d in range(3)]
        Af0 = [kap * dE[d] * (-1.0 / c) for d in range(3)]
        Aff = [[(1.0 if r == q2 else 0.0) - kap * M[r][q2] for q2 in range(3)] for r in range(3)]
        c0 = (db + dq * (1.0 + a) * w) * (etot / rcv) * sE
        # d F_F,g / dE_int through chi_F (q) in 1/(1 + tau q) and kap, and
        # through the source term; base + kap v.P is F_g at the root
        cF = [inv * tau * (dq * F[d] - v[d] * dsrc) * (1.0 / (rcv * c)) for d in range(3)]
        B0 = [a1 * F[d] * (c / c ** 2) * sE for d in range(3)]
        BF = [[-(inv * tau * srcs * (1.0 if r == q2 else 0.0) + kap * Pm[r][q2]) * (c * sF)
               for q2 in range(3)] for r in range(3)]
        rhs0 = to_prec(res["FR"][g], p) * (-sE)
        rhsF = [to_prec(res["FF"][g][d], p) * (-sF) for d in range(3)]
        # eliminate through the R_g row: K = Aff - Af0 A0^T / A00
        ia = 1.0 / A00
        K = [[Aff[r][q2] - Af0[r] * A0[q2] * ia for q2 in range(3)] for r in range(3)]
        cols = [(rhs0, rhsF), (-c0, [-cF[d] for d in range(3)])] + \
               [(-B0[l], [-BF[d][l] for d in range(3)]) for l in range(3)]
        sol = solve3(K, [[t[1][d] - Af0[d] * t[0] * ia for d in range(3)] for t in cols])
        us = [((t[0] - dot3(A0, y)) * ia, y) for t, y in zip(cols, sol)]
        blocks.append(us)   # [p, q, S_0, S_1, S_2], each (r, f[3])
    # the cell's 4x4 system in (x, beta)
    sums = [[N(0.0, p), [N(0.0, p)] * 3] for _ in range(5)]
    for us in blocks:
        for k in range(5):
            sums[k][0] = sums[k][0] + us[k][0]
            sums[k][1] = [sums[k][1][d] + us[k][1][d] for d in range(3)]
    mu = etot / (cell.rho * c * cell.c_hat)
    m = res["m"]
    A = [[N(0.0, p)] * 5 for _ in range(4)]
    A[0] = [sums[1][0] * cr + 1.0] + [to_prec(m[d], p) * (c * sE) + sums[2 + d][0] * cr
                                      for d in range(3)] + \
           [to_prec(res["FG"], p) * (-sE) - sums[0][0] * cr]
    for r in range(3):
        A[1 + r] = [sums[1][1][r] * mu] + [sums[2 + d][1][r] * mu + (1.0 if r == d else 0.0)
                                           for d in range(3)] + [sums[0][1][r] * (-mu)]
    # Gaussian elimination (partial pivoting is a choice of rows: not counted)
    for col in range(4):
        piv = max(range(col, 4), key=lambda r: abs(A[r][col].v))
        A[col], A[piv] = A[piv], A[col]
        ip = 1.0 / A[col][col]
        for r in range(col + 1, 4):
            fct = A[r][col] * ip
            A[r] = [A[r][k] - fct * A[col][k] if k >= col else A[r][k] for k in range(5)]
    y = [None] * 4
    for r in range(3, -1, -1):
        t = A[r][4]
        for k in range(r + 1, 4):
            t = t - A[r][k] * y[k]
        y[r] = t / A[r][r]
    x, beta = y[0], y[1:]
    # the step, added to the FP64 iterate
    cell.Eint = fma(to_prec(x, "f64"), etot, cell.Eint)
    for g, us in enumerate(blocks):
        r = us[0][0] + us[1][0] * x + dot3([us[2 + d][0] for d in range(3)], beta)
        cell.R[g] = fma(to_prec(r, "f64"), etot, cell.R[g])
        for d in range(3):
            f = us[0][1][d] + us[1][1][d] * x + dot3([us[2 + k][1][d] for k in range(3)], beta)
            cell.F[g][d] = fma(to_prec(f, "f64"), c * etot, cell.F[g][d])


def finish(cell: Cell, res: dict):
    """finish64: each R_g from its own row, the flux update F_g - F_F,g, the
    conservative write-back E_g = E_g^t + S_g + R_g, E_gas = E_gas^t -
    (c/c_hat) sum_g R_g and the momentum of eq. vupdate, in FP64."""
    cr = cell.c / cell.c_hat
    sumR = N(0.0)
    for g in range(cell.G):
        cell.R[g] = fma(res["FR"][g], cell.qe[g], cell.R[g])
        sumR = sumR + cell.R[g]
        cell.F[g] = [cell.F[g][d] - res["FF"][g][d] for d in range(3)]
    cell.m = momentum_of(cell)
    cell.egas_final = cell.egas0 - sumR * cr


# ---------------------------------------------------------------------------
# the table the benchmark reads
# ---------------------------------------------------------------------------
EVENTS = ("setup64", "eval64", "cached64", "outer64", "eval32", "outer32", "resid64", "step32",
          "finish64", "residdf", "stepdf")


def _event_counts(state, i, params, groups):
    """One of each event on cell i: tallies by precision and kind."""
    out = {}
    for prec, tag in (("f64", "64"), ("f32", "32")):
        cell = make_cell(state, i, params, groups, p=prec)
        t0 = TALLY.snapshot()
        setup(cell)
        if prec == "f64":
            out["setup64"] = Tally.diff(t0, TALLY.snapshot())
        pass_begin(cell)
        t0 = TALLY.snapshot()
        inner_eval(cell, 0.0)
        out["eval" + tag] = Tally.diff(t0, TALLY.snapshot())
        if prec == "f64":
            c2 = make_cell(state, i, params, groups, p=prec)
            setup(c2)
            pass_begin(c2)
            FR = [c2.R[g] * 1e-3 + 1.0 for g in range(c2.G)]
            dg = [N(1e-3) for _ in range(c2.G)]
            t0 = TALLY.snapshot()
            cached_iteration(c2, FR, dg, 0.0)
            out["cached64"] = Tally.diff(t0, TALLY.snapshot())
        T = cell.Eint * (1.0 / (cell.rho * cell.c_v))
        terms = group_terms_at(cell, T)
        t0 = TALLY.snapshot()
        outer_pass(cell, 0.0, T, terms)
        out["outer" + tag] = Tally.diff(t0, TALLY.snapshot())
    cell = make_cell(state, i, params, groups)
    setup(cell)
    t0 = TALLY.snapshot()
    _, res = coupled_residual(cell, 0.0, 0.0)
    out["resid64"] = Tally.diff(t0, TALLY.snapshot())
    t0 = TALLY.snapshot()
    coupled_step(cell, res)
    out["step32"] = Tally.diff(t0, TALLY.snapshot())
    _, res = coupled_residual(cell, 0.0, 0.0)
    t0 = TALLY.snapshot()
    finish(cell, res)
    out["finish64"] = Tally.diff(t0, TALLY.snapshot())
    # the first step with the residual in float-float: the FP64 residual's
    # operations under "df"; its tests (FP32) are not part of that step
    cell = make_cell(state, i, params, groups)
    setup(cell)
    TALLY.remap = {"f64": "df"}
    t0 = TALLY.snapshot()
    coupled_residual(cell, 0.0, 0.0)
    d = Tally.diff(t0, TALLY.snapshot())
    TALLY.remap = {}
    d["f32"] = {k: 0 for k in KINDS}
    out["residdf"] = d
    out["stepdf"] = {p: dict(v) for p, v in out["step32"].items()}
    return out


def table(presets=("full_256cube_ng64", "surrogate_256cube_ng32", "mixed_128cube_ng16"),
          n_cells: int = 32) -> dict:
    """Mean counts per cell-group of each event on the first n_cells cells of
    each workload (their states decide the branches: the M1 closure's held
    flux, the chi_F bound, the Wien-side Planck form)."""
    from paper_2407_18304_gb300 import synth
    from . import Params, Groups, group_table, PPL_FIXED
    out = {"kinds": list(KINDS), "events": {}}
    for name in presets:
        w = synth.preset(name, n_cells=n_cells)
        st = synth.to_numpy(w.state)
        p = Params(c=w.consts["c"], c_hat=w.consts["c_hat"], a_rad=w.consts["a_rad"],
                   h=w.consts["h"], k_B=w.consts["k_B"], c_v=w.c_v, dt=w.dt)
        km, al = group_table(w.edges, PPL_FIXED, w.law.nu_break, w.law.seg_logk,
                             w.law.seg_beta, w.law.nu_ref)
        g = Groups(w.edges, km, al)
        acc = {e: {pr: {k: 0.0 for k in KINDS} for pr in PRECS} for e in EVENTS}
        for i in range(n_cells):
            ev = _event_counts(st, i, p, g)
            for e in EVENTS:
                for pr in PRECS:
                    for k in KINDS:
                        acc[e][pr][k] += ev[e][pr][k] / (n_cells * w.n_groups)
        out["events"][name] = {e: {pr: {k: round(v, 4) for k, v in acc[e][pr].items()}
                                   for pr in PRECS} for e in EVENTS}
    out["df_fp32_ops"] = DF_FP32_OPS
    return out


GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests",
                      "golden", "opcounts.json")


def write(path: str = GOLDEN) -> str:
    text = json.dumps(table(), indent=1, sort_keys=True) + "\n"
    with open(path, "w") as f:
        f.write(text)
    return text


if __name__ == "__main__":
    write()
