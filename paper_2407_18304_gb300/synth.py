"""Seeded synthetic cell states for the multigroup source-term update.

This module only draws inputs; it holds none of the solver's arithmetic.  It
serves the tests, the oracle comparisons and the benchmark alike, so that both
sides of a parity check always receive the very same tensors.

Recipe (cgs units, one preset per workload):

* group edges: N_g + 1 log-spaced edges with h nu / (k_B T_ref) in [1e-2, 1e2],
  T_ref = 1e7 K;
* rho = exp(N(0, 1)) g cm^-3;  T_gas = U[0.5, 2] T_ref;
* radiation: E_g is a blackbody at T_rad = T_gas * U[0.5, 2] integrated over the
  group (Gauss-Legendre quadrature of the Planck spectrum in ln(nu), 24 nodes per
  group -- an input-side integral, independent of the solver's series);
  |F_g| = U[0, 0.9] c E_g along an isotropic random direction per group;
* velocity: |v|/c = U[0, v_max] along an isotropic random direction;
* gas: mu = 2.33 m_p, c_v = 1.5 k_B / mu, E_gas = rho c_v T + rho |v|^2 / 2;
* opacity: chi_0 = rho kappa0 khat(nu) with khat(nu0) = 1 at h nu0 = k_B T_ref;
  khat is (nu/nu0)^-1 for the smallest preset, otherwise a piecewise powerlaw
  with 8 breakpoints on randomly chosen interior group edges (fewer if the grid
  has fewer), slopes U[-3, 3] and jump factors 10^U[-2, 2] at the breakpoints
  (``random_law_interior`` puts them anywhere instead); kappa0 per cell is set so that
  c rho kappa0 dt is log-uniform in [1e-2, tau_max], dt = 1e-11 s.

Random numbers come from ``torch.Generator`` seeded with ``seed`` (on the
device the tensors are made on), so a given (preset, seed, device type) always
gives the same state.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

C_LIGHT = 2.99792458e10
H_PLANCK = 6.62607015e-27
K_BOLTZ = 1.380649e-16
A_RAD = 8.0 * math.pi ** 5 * K_BOLTZ ** 4 / (15.0 * H_PLANCK ** 3 * C_LIGHT ** 3)
M_PROTON = 1.67262192369e-24
T_REF = 1.0e7
MU = 2.33 * M_PROTON
C_V = 1.5 * K_BOLTZ / MU
DT = 1.0e-11
NU0 = K_BOLTZ * T_REF / H_PLANCK  # h nu0 = k_B T_ref


@dataclass
class OpacityLaw:
    """khat(nu) = exp(seg_logk[s] + seg_beta[s] ln(nu/nu_ref)) in segment s."""
    nu_break: np.ndarray
    seg_logk: np.ndarray
    seg_beta: np.ndarray
    nu_ref: float = NU0


@dataclass
class Workload:
    """A synthetic problem: state tensors plus the grid-wide parameters."""
    name: str
    state: dict
    edges: np.ndarray
    law: OpacityLaw
    dt: float = DT
    c_v: float = C_V
    consts: dict = field(default_factory=lambda: dict(c=C_LIGHT, c_hat=C_LIGHT, a_rad=A_RAD,
                                                      h=H_PLANCK, k_B=K_BOLTZ))

    @property
    def n_cells(self) -> int:
        return int(self.state["rho"].shape[0])

    @property
    def n_groups(self) -> int:
        return len(self.edges) - 1


# name -> (side, n_groups, v_max/c, tau_max, law kind)
PRESETS = {
    "tiny": (8, 4, 1e-3, 1e4, "powerlaw"),
    "fp64_32cube_ng4": (32, 4, 1e-3, 1e4, "powerlaw"),
    "mixed_128cube_ng16": (128, 16, 1e-2, 1e4, "piecewise"),
    "surrogate_256cube_ng32": (256, 32, 1e-2, 1e4, "piecewise"),
    "full_256cube_ng64": (256, 64, 0.1, 1e6, "piecewise"),
}
PRESET_SEED = {"tiny": 18303, "fp64_32cube_ng4": 18304, "mixed_128cube_ng16": 18305,
               "surrogate_256cube_ng32": 18307, "full_256cube_ng64": 18308}


def log_edges(n_groups: int, lo: float = 1e-2, hi: float = 1e2) -> np.ndarray:
    """N_g + 1 log-spaced edges (Hz) with h nu / (k_B T_ref) in [lo, hi]."""
    return NU0 * np.logspace(math.log10(lo), math.log10(hi), n_groups + 1)


def _law_from_breaks(nb: np.ndarray, rng: np.random.Generator) -> OpacityLaw:
    k = len(nb)
    beta = rng.uniform(-3.0, 3.0, k + 1)
    jump = rng.uniform(-2.0, 2.0, k) * math.log(10.0)
    logk = np.zeros(k + 1)
    for s in range(k):
        lb = math.log(nb[s] / NU0)
        logk[s + 1] = logk[s] + (beta[s] - beta[s + 1]) * lb + jump[s]
    s0 = int(np.searchsorted(nb, NU0, side="right"))
    logk -= logk[s0]
    return OpacityLaw(nb, logk, beta, NU0)


def random_law(edges: np.ndarray, rng: np.random.Generator, n_break: int = 8) -> OpacityLaw:
    """Piecewise powerlaw with jumps, normalised to khat(nu0) = 1.

    The breakpoints are distinct interior group edges drawn at random (all of
    them when there are fewer than ``n_break``), so each group sees one powerlaw
    segment and the jumps (factors 10^U[-2, 2]) sit on group boundaries."""
    inner = edges[1:-1]
    k = min(n_break, len(inner))
    nb = np.sort(rng.choice(inner, size=k, replace=False)) if k > 0 else np.zeros(0)
    return _law_from_breaks(nb, rng)


def random_law_interior(edges: np.ndarray, rng: np.random.Generator,
                        n_break: int = 8) -> OpacityLaw:
    """Stress variant: breakpoints log-uniform anywhere in the group range, so a
    jump can fall inside a group and the fitted in-group slope becomes steep."""
    lo, hi = math.log(edges[0]), math.log(edges[-1])
    nb = np.sort(np.exp(rng.uniform(lo, hi, n_break)))
    return _law_from_breaks(nb, rng)


def powerlaw_law(beta: float = -1.0) -> OpacityLaw:
    return OpacityLaw(np.zeros(0), np.zeros(1), np.array([beta]), NU0)


def law_value(law: OpacityLaw, nu: float) -> float:
    """khat at nu (right-continuous at a breakpoint)."""
    s = int(np.searchsorted(law.nu_break, nu, side="right"))
    return math.exp(law.seg_logk[s] + law.seg_beta[s] * math.log(nu / law.nu_ref))


_GL = np.polynomial.legendre.leggauss(24)


def blackbody_group_energy(T_rad: torch.Tensor, edges: np.ndarray) -> torch.Tensor:
    """[G, n] group energies of a blackbody at T_rad (the input spectrum)."""
    xg, wg = (torch.tensor(a, dtype=torch.float64, device=T_rad.device) for a in _GL)
    out = torch.empty((len(edges) - 1, T_rad.shape[0]), dtype=torch.float64, device=T_rad.device)
    norm = 15.0 / math.pi ** 4
    for g in range(len(edges) - 1):
        # integrate t^3/(e^t-1) dt = t^4/(e^t-1) d(ln t) over [x-, x+]
        x0 = H_PLANCK * edges[g] / (K_BOLTZ * T_rad)
        x1 = H_PLANCK * edges[g + 1] / (K_BOLTZ * T_rad)
        l0, l1 = torch.log(x0), torch.log(x1)
        half = 0.5 * (l1 - l0)
        u = (0.5 * (l1 + l0)).unsqueeze(1) + half.unsqueeze(1) * xg.unsqueeze(0)
        t = torch.exp(u)
        f = t ** 4 / torch.expm1(t)
        out[g] = norm * A_RAD * T_rad ** 4 * half * (f * wg.unsqueeze(0)).sum(dim=1)
    return out


def _isotropic(n: int, gen: torch.Generator, device) -> torch.Tensor:
    z = 2.0 * torch.rand(n, generator=gen, dtype=torch.float64, device=device) - 1.0
    phi = 2.0 * math.pi * torch.rand(n, generator=gen, dtype=torch.float64, device=device)
    s = torch.sqrt(torch.clamp(1.0 - z * z, min=0.0))
    return torch.stack([s * torch.cos(phi), s * torch.sin(phi), z])


def make_state(n_cells: int, edges: np.ndarray, law: OpacityLaw, *, v_max: float,
               tau_max: float, seed: int, device="cpu", tau_min: float = 1e-2,
               dtype=torch.float64, chunk: int = 1 << 22) -> dict:
    """Draw one grid's SoA state (see the module docstring for the recipe)."""
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    G = len(edges) - 1
    rand = lambda *s: torch.rand(*s, generator=gen, dtype=torch.float64, device=dev)
    rho = torch.exp(torch.randn(n_cells, generator=gen, dtype=torch.float64, device=dev))
    T = T_REF * (0.5 + 1.5 * rand(n_cells))
    T_rad = T * (0.5 + 1.5 * rand(n_cells))
    vmag = v_max * C_LIGHT * rand(n_cells)
    vdir = _isotropic(n_cells, gen, dev)
    mom = rho * vmag * vdir
    egas = rho * C_V * T + 0.5 * rho * vmag * vmag
    tau = torch.exp(math.log(tau_min) + (math.log(tau_max) - math.log(tau_min)) * rand(n_cells))
    kappa0 = tau / (C_LIGHT * rho * DT)  # khat(nu0) = 1
    erad = torch.empty((G, n_cells), dtype=torch.float64, device=dev)
    for s in range(0, n_cells, chunk):
        e = min(n_cells, s + chunk)
        erad[:, s:e] = blackbody_group_energy(T_rad[s:e], edges)
    fmag = 0.9 * rand(G, n_cells) * C_LIGHT * erad
    frad = torch.empty((3, G, n_cells), dtype=torch.float64, device=dev)
    for g in range(G):
        frad[:, g, :] = fmag[g] * _isotropic(n_cells, gen, dev)
    st = {"rho": rho, "mom": mom.contiguous(), "egas": egas, "kappa0": kappa0,
          "erad": erad, "frad": frad, "src": None}
    if dtype != torch.float64:
        st = {k: (v.to(dtype) if isinstance(v, torch.Tensor) else v) for k, v in st.items()}
    return st


def preset(name: str, device="cpu", n_cells: int | None = None, seed: int | None = None,
           n_groups: int | None = None) -> Workload:
    """One of the named workloads; ``n_cells`` overrides the size (a sample)."""
    side, G, vmax, taumax, kind = PRESETS[name]
    if n_groups is not None:
        G = n_groups
    seed = PRESET_SEED[name] if seed is None else seed
    n = side ** 3 if n_cells is None else n_cells
    edges = log_edges(G)
    rng = np.random.default_rng(seed)
    law = powerlaw_law(-1.0) if kind == "powerlaw" else random_law(edges, rng)
    st = make_state(n, edges, law, v_max=vmax, tau_max=taumax, seed=seed, device=device)
    return Workload(name, st, edges, law)


def batched_grids(n_grids: int = 64, seed: int = 1000 * (18304 + 2), side_lo: int = 16,
                  side_hi: int = 96, groups=(4, 8, 16, 32, 64), device="cpu",
                  max_side: int | None = None) -> list:
    """Uneven grids: side U{side_lo..side_hi}, N_g from ``groups``, own law each."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(n_grids):
        side = int(rng.integers(side_lo, side_hi + 1))
        if max_side is not None:
            side = min(side, max_side)
        G = int(rng.choice(groups))
        edges = log_edges(G)
        law = random_law(edges, np.random.default_rng(seed + j))
        st = make_state(side ** 3, edges, law, v_max=1e-2, tau_max=1e6, seed=seed + j,
                        device=device)
        out.append(Workload(f"grid{j}", st, edges, law))
    return out


def clone_state(st: dict) -> dict:
    return {k: (v.clone() if isinstance(v, torch.Tensor) else v) for k, v in st.items()}


def to_numpy(st: dict) -> dict:
    return {k: (v.detach().cpu().numpy() if isinstance(v, torch.Tensor) else v)
            for k, v in st.items()}


def take_cells(st: dict, idx) -> dict:
    """A sub-state of the cells ``idx`` (same layout)."""
    out = {}
    for k, v in st.items():
        if v is None:
            out[k] = None
        elif v.dim() == 1:
            out[k] = v[idx].contiguous()
        else:
            out[k] = v[..., idx].contiguous()
    return out
