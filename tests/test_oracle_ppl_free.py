"""Pins of the oracle's free-slope mean opacities (Appendix A, eqs. sg and
minmod, fed into eq. chiQg): spectral indices fitted to the group values of
B_nu (at the current temperature) and of E_nu (the radiation energy the update
starts from) instead of the fixed slope -1.

Expected values come from hand-worked examples, from spectra whose index is
known exactly, from quadrature of the definition eq. chiQ, or from invariants
(the reductions to the fixed-slope and PC updates, equilibrium, conservation).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2407_18304_gb300 import synth

mp = pytest.importorskip("mpmath")
mp.mp.dps = 30


# ---------------------------------------------------------------- slopes
def test_minmod_worked_example_log_uniform():
    """Edges e^0, e^2, ..., e^10: every bin centre sqrt(nu- nu+) is e^2 times
    the previous one.  With ln Qbar = 0, 2, 6, 4, 4 the edge slopes are
    2/2, 4/2, -2/2, 0/2 = 1, 2, -1, 0; the interior indices are minmod(1, 2) =
    1, minmod(2, -1) = 0 (signs differ), minmod(-1, 0) = 0; the two end groups
    take -1."""
    edges = np.exp(2.0 * np.arange(6))
    Q = np.exp([0.0, 2.0, 6.0, 4.0, 4.0]) * np.diff(edges)
    np.testing.assert_allclose(O.ppl_free_slopes(edges, Q), [-1, 1, 0, 0, -1], rtol=0, atol=1e-14)


def test_minmod_picks_the_smaller_magnitude_of_negative_slopes():
    """ln Qbar = 0, -2, -6, -10, -12 gives slopes -1, -2, -2, -1: interior
    indices minmod(-1, -2) = -1, minmod(-2, -2) = -2, minmod(-2, -1) = -1."""
    edges = np.exp(2.0 * np.arange(6))
    Q = np.exp([0.0, -2.0, -6.0, -10.0, -12.0]) * np.diff(edges)
    np.testing.assert_allclose(O.ppl_free_slopes(edges, Q), [-1, -1, -2, -1, -1], rtol=0,
                               atol=1e-14)


def test_slopes_use_geometric_centres_and_widths_of_uneven_bins():
    """Uneven edges 1, 2, 8, 16, 50, 51: group averages Qbar_g = nubar_g^k with
    nubar_g = sqrt(nu- nu+) have every edge slope equal to k, so the three
    interior groups take k exactly; Q_g = Qbar_g (nu+ - nu-).  Arithmetic
    centres, or Q_g in place of Qbar_g, would not give k."""
    edges = np.array([1.0, 2.0, 8.0, 16.0, 50.0, 51.0])
    nubar = np.sqrt(edges[:-1] * edges[1:])
    for k in (1.7, -2.3, 0.0):
        Q = nubar ** k * np.diff(edges)
        np.testing.assert_allclose(O.ppl_free_slopes(edges, Q), [-1, k, k, k, -1], rtol=0,
                                   atol=1e-13)


@pytest.mark.parametrize("k", [2.0, -1.0, -3.5, 0.0, 0.6])
def test_binned_powerlaw_spectrum_gives_its_index(k):
    """Q_nu = nu^k integrated over log-uniform bins of ratio r: Qbar_(g+1)/Qbar_g
    = r^k and nubar_(g+1)/nubar_g = r, so every interior index is k."""
    edges = np.logspace(0.0, 3.0, 9)
    if k == -1.0:
        Q = np.log(edges[1:] / edges[:-1])
    else:
        Q = (edges[1:] ** (k + 1) - edges[:-1] ** (k + 1)) / (k + 1)
    a = O.ppl_free_slopes(edges, Q)
    assert a[0] == -1.0 and a[-1] == -1.0
    np.testing.assert_allclose(a[1:-1], k, rtol=0, atol=1e-12)


def test_undefined_slopes_fall_back_to_minus_one():
    """A group next to a non-positive value has an undefined edge slope and
    takes -1, like the end groups; groups two away are unaffected."""
    edges = np.logspace(0.0, 3.0, 8)
    Q = (edges[1:] ** 2 - edges[:-1] ** 2) / 2.0  # index 1
    Q[3] = 0.0
    a = O.ppl_free_slopes(edges, Q)
    np.testing.assert_allclose(a, [-1, 1, -1, -1, -1, 1, -1], rtol=0, atol=1e-12)
    Q[3] = -1.0
    np.testing.assert_allclose(O.ppl_free_slopes(edges, Q), a, rtol=0, atol=0)


@pytest.mark.parametrize("G", [1, 2])
def test_one_or_two_groups_are_all_end_groups(G):
    edges = np.array([1.0, 3.0, 7.0])[: G + 1]
    np.testing.assert_array_equal(O.ppl_free_slopes(edges, np.arange(1.0, G + 1.0)), -np.ones(G))


# ---------------------------------------------------------------- mean opacities
def _params():
    return O.Params(a_rad=synth.A_RAD, h=synth.H_PLANCK, k_B=synth.K_BOLTZ)


@pytest.mark.parametrize("k", [2.0, -2.5])
def test_chi_E_of_a_powerlaw_spectrum_matches_quadrature_of_eq_chiQ(k):
    """E_g^t from E_nu = nu^k: the interior groups' chi_E must be the E_nu-
    weighted mean of chi_0 over the group (eq. chiQ, by quadrature); the end
    groups take the fixed-slope mean (E_nu ~ nu^-1)."""
    G = 7
    edges = synth.log_edges(G)
    alpha = np.array([-2.0, 1.3, -0.7, 2.5, -3.0, 0.4, -1.2])
    khat = np.array([1.2, 0.3, 2.2, 0.9, 5.0, 0.7, 1.1])
    E = np.array([float(mp.quad(lambda n: n ** k, [edges[g], edges[g + 1]])) for g in range(G)])
    grp = O.Groups(edges, khat, alpha, free_slopes=True)
    t = O.group_terms(_params(), grp, 2.0, 1.1e7, erad0=E)
    for g in range(G):
        kq = k if 0 < g < G - 1 else -1.0
        r = edges[g + 1] / edges[g]
        num = mp.quad(lambda u: 2.0 * khat[g] * u ** (alpha[g] + kq), [1, r])
        den = mp.quad(lambda u: u ** kq, [1, r])
        assert t["chiE"][g] == pytest.approx(float(num / den), rel=1e-12)


def test_chi_B_approaches_the_planck_mean_where_the_fixed_slope_does_not():
    """Deep in the Rayleigh-Jeans part (h nu / k T <= 0.03) B_nu ~ nu^2, far
    from the fixed slope -1.  The free-slope chi_B of the interior groups is the
    Planck-weighted mean of chi_0 over the group (quadrature of eq. chiQ with
    the exact Planck function) to the small curvature of B_nu there; the
    fixed-slope value is off by tens of per cent."""
    G = 8
    T = 1.0e7
    nu_T = synth.K_BOLTZ * T / synth.H_PLANCK
    edges = nu_T * np.logspace(-4.0, math.log10(0.03), G + 1)
    alpha = np.full(G, -2.0)
    khat = np.ones(G)
    free = O.group_terms(_params(), O.Groups(edges, khat, alpha, free_slopes=True), 1.0, T)
    fixed = O.group_terms(_params(), O.Groups(edges, khat, alpha), 1.0, T)
    for g in range(1, G - 1):
        x0, x1 = edges[g] / nu_T, edges[g + 1] / nu_T
        B = lambda x: x ** 3 / mp.expm1(x)
        exact = float(mp.quad(lambda x: (x / x0) ** -2.0 * B(x), [x0, x1]) / mp.quad(B, [x0, x1]))
        assert abs(free["chiB"][g] / exact - 1) < 2e-3
        assert abs(fixed["chiB"][g] / exact - 1) > 0.2


def test_chi_E_equals_chi_B_when_E_g_equals_b_g():
    """The same slope method for B and E makes chi_E = chi_B when the radiation
    spectrum is the Planck one (the condition for G^0 to vanish at high optical
    depth, Sec. 2.2.2)."""
    G = 12
    edges = synth.log_edges(G)
    rng = np.random.default_rng(9)
    grp = O.Groups(edges, np.exp(rng.uniform(-1, 1, G)), rng.uniform(-3, 3, G), free_slopes=True)
    t0 = O.group_terms(_params(), grp, 1.5, 9e6)
    t = O.group_terms(_params(), grp, 1.5, 9e6, erad0=t0["b"])
    np.testing.assert_array_equal(t["chiE"], t["chiB"])
    # and they differ from the fixed-slope means
    tf = O.group_terms(_params(), O.Groups(edges, grp.khat_minus, grp.alpha), 1.5, 9e6)
    assert np.max(np.abs(t["chiB"][1:-1] / tf["chiB"][1:-1] - 1)) > 1e-2


# ---------------------------------------------------------------- whole update
def _oracle_params(w, **kw):
    d = dict(c=w.consts["c"], c_hat=w.consts["c_hat"], a_rad=w.consts["a_rad"], h=w.consts["h"],
             k_B=w.consts["k_B"], c_v=w.c_v, dt=w.dt, max_iter=200)
    d.update(kw)
    return O.Params(**d)


def _groups(w, free, mode=O.PPL_FIXED):
    km, al = O.group_table(w.edges, mode, w.law.nu_break, w.law.seg_logk, w.law.seg_beta,
                           w.law.nu_ref)
    return O.Groups(w.edges, km, al, free_slopes=free)


def test_first_order_limit_is_the_four_force_with_free_slopes():
    """For a tiny step the update is the explicit four-force of eqs. G0_3 and
    G1_3 (Eddington pressure, so P_g = E_g/3 I and chi_P = chi_E): chi_B from
    the indices of b_g(T), chi_E from those of E_g^t, chi_F from eq. chiDiff
    with both.  Indices from ppl_free_slopes (pinned above), means by
    quadrature of eq. chiQ; E_g^t zig-zags about b_g so the two index sets
    differ."""
    G = 6
    edges = synth.log_edges(G)
    alpha = np.array([-1.7, -0.8, -2.4, 1.4, -1.1, 0.6])
    khat = np.array([1.5, 0.7, 2.0, 0.4, 1.2, 0.9])
    T, rho, kappa0 = 1.2e7, 0.9, 3.0
    c = synth.C_LIGHT
    x = synth.H_PLANCK * edges / (synth.K_BOLTZ * T)
    aT4 = synth.A_RAD * T ** 4
    B = lambda t: t ** 3 / mp.expm1(t)
    NORM = 15 / mp.pi ** 4
    b = np.array([float(aT4 * NORM * mp.quad(B, [x[g], x[g + 1]])) for g in range(G)])
    E = b * np.array([1.3, 0.8, 1.25, 0.7, 1.2, 0.9])
    aB, aE = O.ppl_free_slopes(edges, b), O.ppl_free_slopes(edges, E)
    assert np.max(np.abs(aB - aE)) > 0.3
    rng = np.random.default_rng(4)
    v = np.array([0.004, -0.002, 0.003]) * c
    F = np.array([0.9 * c * E[g] * d / np.linalg.norm(d) for g, d in enumerate(rng.normal(size=(G, 3)))])
    st = {"rho": np.array([rho]), "mom": (rho * v)[:, None].copy(),
          "egas": np.array([rho * synth.C_V * T + 0.5 * rho * v @ v]), "kappa0": np.array([kappa0]),
          "erad": E[:, None].copy(), "frad": F.T[:, :, None].copy(), "src": None}
    dt = 1e-19
    p = O.Params(a_rad=synth.A_RAD, c_v=synth.C_V, dt=dt, closure=O.CLOSURE_EDDINGTON)
    out = O.source_update(st, p, O.Groups(edges, khat, alpha, free_slopes=True))
    assert out["status"][0] == 0
    nuB = lambda t: NORM * t ** 4 / mp.expm1(t)
    for g in range(G):
        r = edges[g + 1] / edges[g]
        chim = rho * kappa0 * khat[g]

        def mean(aq):
            return float(chim * mp.quad(lambda u: u ** (alpha[g] + aq), [1, r])
                         / mp.quad(lambda u: u ** aq, [1, r]))

        chiB, chiE = mean(aB[g]), mean(aE[g])
        d0, d1 = nuB(x[g]), nuB(x[g + 1])
        dnb = float(aT4 * (d1 - d0))
        dnxb = float(aT4 * chim * (r ** alpha[g] * d1 - d0))
        chiF = ((chiB + chiE / 3) * b[g] + (alpha[g] * chiE * b[g] - dnxb) / 3) / (4 * b[g] / 3 - dnb / 3)
        assert min(1, r ** alpha[g]) < chiF / chim < max(1, r ** alpha[g])  # not held
        G0 = chiB * b[g] - chiE * E[g] + (1 + alpha[g]) * chiF * (v @ F[g]) / c ** 2
        dE = (out["erad"][g, 0] - E[g]) / (c * dt)
        assert dE == pytest.approx(G0, rel=1e-5)
        Gi = -chiF * F[g] + v * (chiB * b[g] - dnxb / 3) + (1 + alpha[g]) * chiE * v * E[g] / 3
        dF = (out["frad"][:, g, 0] - F[g]) / (c * dt)
        np.testing.assert_allclose(dF, Gi, rtol=1e-5, atol=1e-5 * np.abs(Gi).max())


@pytest.mark.parametrize("tau", [1e-2, 1.0, 1e6])
def test_v0_planck_equilibrium_is_unchanged_with_free_slopes(tau):
    w = synth.preset("mixed_128cube_ng16", n_cells=4, seed=5)
    T, rho = 1.37e7, 0.8
    x = w.consts["h"] * w.edges / (w.consts["k_B"] * T)
    aT4 = w.consts["a_rad"] * T ** 4
    NORM = 15 / mp.pi ** 4
    E = np.array([float(aT4 * NORM * mp.quad(lambda t: t ** 3 / mp.expm1(t), [x[g], x[g + 1]]))
                  for g in range(len(x) - 1)])
    G = len(E)
    st = {"rho": np.array([rho]), "mom": np.zeros((3, 1)), "egas": np.array([rho * w.c_v * T]),
          "kappa0": np.array([tau / (synth.C_LIGHT * rho * w.dt)]), "erad": E[:, None].copy(),
          "frad": np.zeros((3, G, 1)), "src": None}
    out = O.source_update(st, _oracle_params(w), _groups(w, True))
    assert out["status"][0] == 0
    np.testing.assert_allclose(out["erad"], st["erad"], rtol=1e-12, atol=0)
    assert out["egas"][0] / (rho * w.c_v) == pytest.approx(T, rel=1e-14)
    assert np.all(out["frad"] == 0.0) and np.all(out["mom"] == 0.0)


def test_reductions_to_the_fixed_slope_and_pc_updates():
    """One or two groups are all end groups (alpha_Q = -1): the free-slope
    update is the fixed-slope one, bit for bit.  PC opacities are flat in
    every group, so the spectrum's index does not enter: free = PC."""
    for G in (1, 2):
        w = synth.preset("mixed_128cube_ng16", n_cells=24, seed=3, n_groups=G)
        st = synth.to_numpy(w.state)
        a = O.source_update(st, _oracle_params(w), _groups(w, True))
        b = O.source_update(st, _oracle_params(w), _groups(w, False))
        assert np.all(a["status"] == 0)
        for k in ("erad", "frad", "mom", "egas"):
            np.testing.assert_array_equal(a[k], b[k])
    w = synth.preset("mixed_128cube_ng16", n_cells=24, seed=3)
    st = synth.to_numpy(w.state)
    a = O.source_update(st, _oracle_params(w), _groups(w, True, O.PC))
    b = O.source_update(st, _oracle_params(w), _groups(w, False, O.PC))
    for k in ("erad", "frad", "mom", "egas"):
        np.testing.assert_array_equal(a[k], b[k])


def test_free_slope_update_conserves_and_differs_from_fixed():
    w = synth.preset("mixed_128cube_ng16", n_cells=48, seed=21)
    st = synth.to_numpy(w.state)
    p = _oracle_params(w)
    a = O.source_update(st, p, _groups(w, True))
    b = O.source_update(st, p, _groups(w, False))
    assert np.all(a["status"] == 0)
    cr = p.c / p.c_hat
    e0 = st["egas"] + cr * st["erad"].sum(0)
    e1 = a["egas"] + cr * a["erad"].sum(0)
    assert np.max(np.abs(e1 - e0) / e0) < 1e-14
    m0 = st["mom"] + st["frad"].sum(1) / (p.c * p.c_hat)
    m1 = a["mom"] + a["frad"].sum(1) / (p.c * p.c_hat)
    mscale = np.abs(st["mom"]) + (np.abs(st["frad"]).sum(1) + np.abs(a["frad"]).sum(1)) / (p.c * p.c_hat)
    assert np.max(np.abs(m1 - m0) / mscale) < 40 * 2.0 ** -52
    rel = np.abs(a["erad"] - b["erad"]) / (np.abs(b["erad"]) + 1e-300)
    assert np.max(rel) > 1e-6
