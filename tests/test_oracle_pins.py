"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value comes from
arbitrary-precision quadrature or root finding (mpmath), a closed form, a value
the paper prints (``tests/golden``), or an invariant of the equations.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2407_18304_gb300 import synth

mp = pytest.importorskip("mpmath")
mp.mp.dps = 40
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def mp_planck_integral(a, b):
    f = lambda t: t ** 3 / mp.expm1(t)
    if b == math.inf:
        return mp.quad(f, [a, a + 10, a + 60, mp.inf])
    pts = [a] + [a + k * (b - a) / 8 for k in range(1, 8)] + [b]
    return mp.quad(f, pts)


NORM = 15 / mp.pi ** 4


def mp_band(x0, x1):
    return NORM * mp_planck_integral(mp.mpf(x0), x1 if x1 == math.inf else mp.mpf(x1))


def mp_nuB(x):
    """(15/pi^4) x^4/(e^x-1): nu * 4 pi B_nu / c per a_R T^4."""
    if x == 0 or x == math.inf:
        return mp.mpf(0)
    x = mp.mpf(x)
    return NORM * x ** 4 / mp.expm1(x)


DIMLESS = dict(c=1.0, c_hat=1.0, a_rad=1.0, h=1.0, k_B=1.0)


# ---------------------------------------------------------------- Planck integrals
@pytest.mark.parametrize("x", [1e-3, 0.01, 0.3, 1.0, 1.9999, 2.0, 2.5, 5.0, 10.0, 30.0, 100.0,
                               400.0])
def test_planck_fraction_matches_quadrature(x):
    P = NORM * mp_planck_integral(mp.mpf(0), mp.mpf(x))
    Q = NORM * mp_planck_integral(mp.mpf(x), math.inf)
    assert abs(P + Q - 1) < mp.mpf(10) ** -30
    assert O.planck_P(x) == pytest.approx(float(P), rel=3e-15, abs=1e-17)
    assert O.planck_Q(x) == pytest.approx(float(Q), rel=3e-14)


def test_planck_band_sum_rule_and_limits():
    rng = np.random.default_rng(1)
    for _ in range(20):
        inner = np.sort(np.exp(rng.uniform(math.log(1e-3), math.log(300.0), 7)))
        edges = np.concatenate([[0.0], inner, [math.inf]])
        s = sum(O.planck_band(edges[i], edges[i + 1]) for i in range(len(edges) - 1))
        assert s == pytest.approx(1.0, abs=2e-15)
    assert O.planck_P(0.0) == 0.0 and O.planck_P(math.inf) == 1.0
    # narrow band in the Wien tail keeps full relative precision
    band = O.planck_band(50.0, 50.5)
    assert band == pytest.approx(float(mp_band(50.0, 50.5)), rel=1e-13)


# ---------------------------------------------------------------- PPL mean opacity
@pytest.mark.parametrize("alpha_chi,alpha_Q,r", [
    (0.0, -1.0, 1.78), (1.3, -1.0, 1.78), (-2.7, -1.0, 10.0), (2.9, -1.0, 1.155),
    (1.0, -2.0, 3.0),   # alpha_chi + alpha_Q = -1: second bracket is ln r
    (-0.4, 0.7, 5.0), (2.2, 1.5, 1.01), (1e-7, -1.0, 2.0)])
def test_ppl_mean_opacity_matches_quadrature(alpha_chi, alpha_Q, r):
    chi_minus = 2.5
    num = mp.quad(lambda u: chi_minus * u ** (alpha_chi + alpha_Q), [1, r])
    den = mp.quad(lambda u: u ** alpha_Q, [1, r])
    expect = float(num / den)
    assert O.ppl_mean_opacity(chi_minus, alpha_chi, alpha_Q, r) == pytest.approx(expect, rel=1e-13)


def test_ppl_mean_opacity_pc_limit():
    for aQ in (-1.0, 0.5, -2.5):
        assert O.ppl_mean_opacity(3.0, 0.0, aQ, 7.0) == pytest.approx(3.0, rel=1e-15)


# ---------------------------------------------------------------- group table
def test_group_table_from_law_edges_and_centres():
    edges = np.array([1.0, 2.0, 4.0, 8.0, 16.0])
    nb = np.array([2.0, 5.0])          # first breakpoint exactly on an edge
    logk = np.array([0.0, 1.0, -2.0])
    beta = np.array([-1.0, 2.0, 0.5])
    khat = lambda s, nu: math.exp(logk[s] + beta[s] * math.log(nu / 3.0))
    km, al = O.group_table(edges, O.PPL_FIXED, nb, logk, beta, 3.0)
    # group 0 = [1,2): lower value seg 0; upper value is the LEFT limit at 2 (seg 0)
    assert km[0] == pytest.approx(khat(0, 1.0), rel=1e-15)
    assert al[0] == pytest.approx(-1.0, rel=1e-14)
    # group 1 = [2,4): lower value is the RIGHT-continuous one at 2 (seg 1)
    assert km[1] == pytest.approx(khat(1, 2.0), rel=1e-15)
    assert al[1] == pytest.approx(2.0, rel=1e-14)
    # group 2 = [4,8) contains the jump at 5: secant slope between edge values
    a2 = math.log(khat(2, 8.0) / khat(1, 4.0)) / math.log(2.0)
    assert al[2] == pytest.approx(a2, rel=1e-14)
    kpc, apc = O.group_table(edges, O.PC, nb, logk, beta, 3.0)
    assert np.all(apc == 0.0)
    assert kpc[3] == pytest.approx(khat(2, math.sqrt(8.0 * 16.0)), rel=1e-15)


# ---------------------------------------------------------------- group terms
def test_pulse_opacity_planck_mean_converges_to_printed_value():
    """Sec. 4.2.3: the PPL group machinery reproduces the analytic Planck mean
    3063.96 cm^-1 of the pulse opacity at T = 1e7 K as the groups narrow.  The
    PPL fixed-slope error is second order in the group width, so four times
    more groups cut it about sixteen-fold, and the Richardson extrapolation of
    the last two refinements lands on the printed value.  (Below 1e11 Hz the
    Planck-mean integrand, proportional to exp(-h nu/k T), adds only 5e-7.)"""
    g = golden("pulse_planck_mean.txt")["chi_P_at_1e7K"]
    h, k, T = synth.H_PLANCK, synth.K_BOLTZ, 1e7
    chi0 = lambda nu: 180.0 * (nu / 1e18) ** -3 * (-math.expm1(-h * nu / (k * T)))
    means = []
    for ng in (128, 512, 2048):
        edges = np.logspace(11, 21, ng + 1)
        km = np.array([chi0(edges[i]) for i in range(ng)])
        al = np.array([math.log(chi0(edges[i + 1]) / chi0(edges[i])) / math.log(edges[i + 1] / edges[i])
                       for i in range(ng)])
        p = O.Params(a_rad=synth.A_RAD, h=h, k_B=k)
        t = O.group_terms(p, O.Groups(edges, km, al), 1.0, T)
        means.append((t["chiB"] * t["b"]).sum() / t["b"].sum())
    e = [abs(m / g - 1.0) for m in means]
    assert e[0] / e[1] > 10 and e[1] / e[2] > 10
    extrap = means[2] + (means[2] - means[1]) / 15.0
    assert extrap == pytest.approx(g, rel=3e-6)


def test_pulse_opacity_planck_mean_follows_printed_temperature_law():
    """The same Planck mean at the pulse's peak temperature T_1 = 2e7 K
    (Sec. 4.2.3), where the printed law gives 3063.96 (T/1e7 K)^-3.5.  The
    opacity's own T^-0.5 factor comes from the group table's (T/T_ref)^p
    factor (T_ref = 1e7 K, p = -0.5), the stimulated-emission factor from the
    per-group values built at T_1; the rest of the -3.5 is the Planck
    spectrum's shift, which the group integrals carry."""
    gd = golden("pulse_planck_mean.txt")
    h, k, T0, T1 = synth.H_PLANCK, synth.K_BOLTZ, 1e7, 2e7
    chi0 = lambda nu: 180.0 * (nu / 1e18) ** -3 * (-math.expm1(-h * nu / (k * T1)))
    means = []
    for ng in (512, 2048):
        edges = np.logspace(11, 21, ng + 1)
        km = np.array([chi0(edges[i]) for i in range(ng)])
        al = np.array([math.log(chi0(edges[i + 1]) / chi0(edges[i])) / math.log(edges[i + 1] / edges[i])
                       for i in range(ng)])
        p = O.Params(a_rad=synth.A_RAD, h=h, k_B=k, temp_exponent=-0.5, T_ref=T0)
        t = O.group_terms(p, O.Groups(edges, km, al), 1.0, T1)
        means.append((t["chiB"] * t["b"]).sum() / t["b"].sum())
    extrap = means[1] + (means[1] - means[0]) / 15.0
    assert extrap == pytest.approx(gd["chi_P_at_1e7K"] * (T1 / T0) ** gd["chi_T_exponent"], rel=3e-6)


def test_chiF_equals_chi_in_pc_limit():
    edges = synth.log_edges(8)
    km = np.linspace(0.5, 3.0, 8)
    p = O.Params(a_rad=synth.A_RAD)
    for T in (5e6, 1e7, 3e7):
        t = O.group_terms(p, O.Groups(edges, km, np.zeros(8)), 4.0, T)
        np.testing.assert_allclose(t["chiF"], 4.0 * km, rtol=2e-15)
        np.testing.assert_allclose(t["chiB"], 4.0 * km, rtol=2e-15)


def test_group_planck_terms_match_quadrature():
    edges = synth.log_edges(6)
    km = np.full(6, 1.0)
    al = np.array([-1.0, 0.5, 2.0, -2.0, 0.0, 1.0])
    T = 1.3e7
    t = O.group_terms(O.Params(a_rad=synth.A_RAD), O.Groups(edges, km, al), 2.0, T)
    x = synth.H_PLANCK * edges / (synth.K_BOLTZ * T)
    aT4 = synth.A_RAD * T ** 4
    for g in range(6):
        assert t["b"][g] == pytest.approx(float(aT4 * mp_band(x[g], x[g + 1])), rel=1e-13)
        dnb = aT4 * (mp_nuB(x[g + 1]) - mp_nuB(x[g]))
        assert t["dnb"][g] == pytest.approx(float(dnb), rel=1e-12)
        r = edges[g + 1] / edges[g]
        dnxb = aT4 * 2.0 * (r ** al[g] * mp_nuB(x[g + 1]) - mp_nuB(x[g]))
        assert t["dnxb"][g] == pytest.approx(float(dnxb), rel=1e-12)


# ---------------------------------------------------------------- closure / linear algebra
def test_closure_limits():
    c, E = 3.0, 2.0
    np.testing.assert_allclose(O.closure(O.CLOSURE_M1, c, E, [0, 0, 0]), np.eye(3) * E / 3, rtol=1e-15)
    np.testing.assert_allclose(O.closure(O.CLOSURE_EDDINGTON, c, E, [1, 2, 3]), np.eye(3) * E / 3,
                               rtol=1e-15)
    n = np.array([1.0, -2.0, 2.0]) / 3.0
    np.testing.assert_allclose(O.closure(O.CLOSURE_M1, c, E, c * E * n), E * np.outer(n, n),
                               rtol=1e-14, atol=1e-15)
    rng = np.random.default_rng(3)
    for f in rng.uniform(0, 1, 10):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        P = O.closure(O.CLOSURE_M1, c, E, f * c * E * d)
        assert np.trace(P) == pytest.approx(E, rel=1e-14)
        np.testing.assert_allclose(P, P.T, rtol=0, atol=1e-15)
        chi = (3 + 4 * f * f) / (5 + 2 * math.sqrt(4 - 3 * f * f))
        assert d @ P @ d == pytest.approx(chi * E, rel=1e-13)


@pytest.mark.parametrize("n", [1, 2, 5, 16, 64])
def test_arrowhead_elimination_matches_dense_lu(n):
    rng = np.random.default_rng(n)
    for _ in range(5):
        top = rng.normal(size=n)
        left = rng.normal(size=n)
        diag = -1.0 - rng.uniform(0.1, 10, size=n)
        a00 = 1.0 + np.abs(top * left / diag).sum()
        A = np.zeros((n + 1, n + 1))
        A[0, 0], A[0, 1:], A[1:, 0] = a00, top, left
        A[np.arange(1, n + 1), np.arange(1, n + 1)] = diag
        rhs = rng.normal(size=n + 1)
        x = O.arrowhead_solve(a00, top, left, diag, rhs)
        x_lu = O.dense_solve(A, rhs)
        x_np = np.linalg.solve(A, rhs)
        cond = np.linalg.cond(A)
        np.testing.assert_allclose(x, x_np, rtol=0, atol=1e-14 * cond * np.abs(x_np).max())
        np.testing.assert_allclose(x_lu, x_np, rtol=0, atol=1e-14 * cond * np.abs(x_np).max())


# ---------------------------------------------------------------- whole update
def oracle_params(w, **kw):
    d = dict(c=w.consts["c"], c_hat=w.consts["c_hat"], a_rad=w.consts["a_rad"], h=w.consts["h"],
             k_B=w.consts["k_B"], c_v=w.c_v, dt=w.dt, max_iter=200)
    d.update(kw)
    return O.Params(**d)


def oracle_groups(w, mode=O.PPL_FIXED):
    km, al = O.group_table(w.edges, mode, w.law.nu_break, w.law.seg_logk, w.law.seg_beta,
                           w.law.nu_ref)
    return O.Groups(w.edges, km, al)


def gas_T(st, c_v):
    ke = 0.5 * (st["mom"] ** 2).sum(0) / st["rho"]
    return (st["egas"] - ke) / (st["rho"] * c_v)


@pytest.mark.parametrize("c_hat_frac,with_src,theta", [(1.0, False, 1.0), (0.1, False, 0.5),
                                                       (1.0, True, 1.0)])
def test_conservation_to_roundoff(c_hat_frac, with_src, theta):
    w = synth.preset("mixed_128cube_ng16", n_cells=96, seed=77)
    st = synth.to_numpy(w.state)
    if with_src:
        st["src"] = 0.3 * st["erad"][:, ::-1].copy()
    p = oracle_params(w, c_hat=w.consts["c"] * c_hat_frac, theta=theta)
    out = O.source_update(st, p, oracle_groups(w))
    assert np.all(out["status"] == 0)
    r = p.c / p.c_hat
    src = st["src"].sum(0) if with_src else 0.0
    e0 = st["egas"] + r * (st["erad"].sum(0) + src)
    e1 = out["egas"] + r * out["erad"].sum(0)
    scale = st["egas"] + r * (st["erad"].sum(0) + src + out["erad"].sum(0))
    assert np.max(np.abs(e1 - e0) / scale) < 40 * 2.0 ** -52
    m0 = st["mom"] + st["frad"].sum(1) / (p.c * p.c_hat)
    m1 = out["mom"] + out["frad"].sum(1) / (p.c * p.c_hat)
    mscale = np.abs(st["mom"]) + (np.abs(st["frad"]).sum(1) + np.abs(out["frad"]).sum(1)) / (p.c * p.c_hat)
    assert np.max(np.abs(m1 - m0) / mscale) < 40 * 2.0 ** -52


@pytest.mark.parametrize("free", [False, True])
def test_source_enters_only_with_the_starting_energy(free):
    """Eq. FGFR: E_g^(t) and S_g appear only as E_g^(t) + S_g (in F_R,g and in
    E_tot), so an update with a source equals the update without one started
    from E_g^(t) + S_g -- moving cells, M1, c_hat = 0.3 c, fixed or App. A
    slopes (whose E_nu index is taken from E_g^(t) + S_g)."""
    w = synth.preset("mixed_128cube_ng16", n_cells=24, seed=91)
    st = synth.to_numpy(w.state)
    rng = np.random.default_rng(4)
    st["src"] = st["erad"] * rng.uniform(-0.4, 0.8, size=st["erad"].shape)
    p = oracle_params(w, c_hat=0.3 * w.consts["c"])
    g = oracle_groups(w)
    g.free_slopes = free
    a = O.source_update(st, p, g)
    b = O.source_update(dict(st, erad=st["erad"] + st["src"], src=None), p, g)
    assert np.all(a["status"] == 0) and np.all(b["status"] == 0)
    for key in ("egas", "mom", "erad", "frad"):
        scale = np.abs(a[key]).max(axis=-1, keepdims=True) + 1e-300
        np.testing.assert_allclose(a[key] / scale, b[key] / scale, rtol=0, atol=1e-12, err_msg=key)


def _equilibrium_state(edges, T, rho, kappa0, consts, c_v):
    x = consts["h"] * edges / (consts["k_B"] * T)
    aT4 = consts["a_rad"] * T ** 4
    G = len(edges) - 1
    E = np.array([float(aT4 * mp_band(x[g], x[g + 1])) for g in range(G)])
    return {"rho": np.array([rho]), "mom": np.zeros((3, 1)), "egas": np.array([rho * c_v * T]),
            "kappa0": np.array([kappa0]), "erad": E[:, None].copy(), "frad": np.zeros((3, G, 1)),
            "src": None}


@pytest.mark.parametrize("tau", [1e-2, 1.0, 1e6])
def test_v0_planck_equilibrium_is_unchanged(tau):
    w = synth.preset("full_256cube_ng64", n_cells=4, seed=5)
    T = 1.37e7
    st = _equilibrium_state(w.edges, T, 0.8, tau / (synth.C_LIGHT * 0.8 * synth.DT), w.consts, w.c_v)
    out = O.source_update(st, oracle_params(w), oracle_groups(w))
    assert out["status"][0] == 0
    np.testing.assert_allclose(out["erad"], st["erad"], rtol=1e-12, atol=0)
    assert gas_T(out | {"rho": st["rho"]}, w.c_v)[0] == pytest.approx(T, rel=1e-14)
    assert np.all(out["frad"] == 0.0) and np.all(out["mom"] == 0.0)


def _grey_T(egas0, E0, rho, c_v, tau, a):
    f = lambda T: rho * c_v * T + (E0 + tau * a * T ** 4) / (1 + tau) - (egas0 + E0)
    return mp.findroot(f, mp.mpf(egas0 / (rho * c_v)), tol=mp.mpf(10) ** -35)


@pytest.mark.parametrize("ng", [1, 8])
def test_grey_reduction_for_frequency_independent_opacity(ng):
    """N_g = 1 over [0, inf), or N_g groups with one constant opacity, at v = 0:
    the gas temperature is the root of the grey backward-Euler balance."""
    if ng == 1:
        edges = np.array([0.0, math.inf])
    else:
        edges = np.concatenate([[0.0], synth.log_edges(ng - 2), [math.inf]])
    assert len(edges) == ng + 1
    law = synth.powerlaw_law(0.0)
    km, al = O.group_table(edges, O.PC, law.nu_break, law.seg_logk, law.seg_beta, law.nu_ref)
    rho, T0, Trad = 1.7, 1.2e7, 0.6e7
    x = synth.H_PLANCK * edges / (synth.K_BOLTZ * Trad)
    E0 = np.array([float(synth.A_RAD * Trad ** 4 * mp_band(x[g], x[g + 1])) for g in range(ng)])
    for tau in (0.3, 30.0, 3e5):
        kappa0 = tau / (synth.C_LIGHT * rho * synth.DT)
        st = {"rho": np.array([rho]), "mom": np.zeros((3, 1)),
              "egas": np.array([rho * synth.C_V * T0]), "kappa0": np.array([kappa0]),
              "erad": E0[:, None].copy(), "frad": np.zeros((3, ng, 1)), "src": None}
        p = O.Params(a_rad=synth.A_RAD, c_v=synth.C_V, dt=synth.DT)
        out = O.source_update(st, p, O.Groups(edges, km, al))
        T = gas_T(out | {"rho": st["rho"]}, synth.C_V)[0]
        Tg = _grey_T(st["egas"][0], E0.sum(), rho, synth.C_V, tau, synth.A_RAD)
        assert T == pytest.approx(float(Tg), rel=1e-13)


@pytest.mark.parametrize("c_hat_frac,theta,tau,src", [(1.0, 1.0, 0.5, 0.0), (1.0, 0.5, 40.0, 0.0),
                                                      (0.1, 1.0, 7.0, 0.0), (0.1, 0.5, 3.0, 3.0),
                                                      (1.0, 1.0, 0.5, -2.0)])
def test_linear_grey_relaxation_matches_closed_form(c_hat_frac, theta, tau, src):
    """Grey, v = 0, small perturbation about equilibrium: one implicit step
    scales the disequilibrium D = kappa u - e by 1/(1 + theta dt chi (c_hat + c kappa)),
    kappa = 4 a T^3 / (rho c_v).  In eq. FGFR the explicit source S_g enters
    only with E_g^(t), as E_g^(t) + S_g, so a perturbation carried partly by
    S (src: S = src delta E, E^(t) = E (1 + delta) - S) relaxes the same way."""
    rho, T0, delta = 1.0, 1.0e7, 1e-7
    c, a, cv = synth.C_LIGHT, synth.A_RAD, synth.C_V
    chat = c * c_hat_frac
    chi = tau / (chat * theta * synth.DT)
    E0 = a * T0 ** 4
    S = src * delta * E0
    st = {"rho": np.array([rho]), "mom": np.zeros((3, 1)), "egas": np.array([rho * cv * T0]),
          "kappa0": np.array([chi / rho]), "erad": np.array([[E0 * (1 + delta) - S]]),
          "frad": np.zeros((3, 1, 1)), "src": np.array([[S]]) if src else None}
    p = O.Params(c=c, c_hat=chat, a_rad=a, c_v=cv, dt=synth.DT, theta=theta)
    edges = np.array([0.0, math.inf])
    out = O.source_update(st, p, O.Groups(edges, np.ones(1), np.zeros(1)))
    kap = 4 * a * T0 ** 3 / (rho * cv)
    D0 = -delta * E0
    T1 = gas_T(out | {"rho": st["rho"]}, cv)[0]
    D1 = kap * rho * cv * (T1 - T0) - (out["erad"][0, 0] - E0)
    expect = 1.0 / (1.0 + theta * synth.DT * chi * (chat + c * kap))
    assert D1 / D0 == pytest.approx(expect, rel=2e-6)


def _doppler_run(edges, v, steps=5, closure=O.CLOSURE_M1, c_hat=1.0):
    """Sec. 4.2.1 set-up, source term only (a uniform periodic medium has no
    transport divergence): a_R = k_B = h = c = 1, rho = 1, C_V = 3/2, T_gas = 1,
    chi_0 = 1e5, no radiation at the start (c_hat < 1: the reduced speed of
    light of Sec. 3)."""
    G = len(edges) - 1
    st = {"rho": np.array([1.0]), "mom": np.array([[v], [0.0], [0.0]]),
          "egas": np.array([1.5 + 0.5 * v * v]), "kappa0": np.array([1e5]),
          "erad": np.full((G, 1), 0.0), "frad": np.zeros((3, G, 1)), "src": None}
    p = O.Params(**dict(DIMLESS, c_hat=c_hat), c_v=1.5, dt=1e3, closure=closure)
    grp = O.Groups(edges, np.ones(G), np.zeros(G))
    for _ in range(steps):
        out = O.source_update(st, p, grp)
        assert out["status"][0] == 0
        st = dict(st, mom=out["mom"], egas=out["egas"], erad=out["erad"], frad=out["frad"])
    return st


def test_doppler_equilibrium_temperature_printed_value():
    gd = golden("doppler_equilibrium.txt")
    root = mp.findroot(lambda T: T ** 4 + 1.5 * T - 1.5, 0.77)
    assert float(root) == pytest.approx(gd["T_exact"], abs=5e-13)
    # groups covering [0, inf): the v = 0 equilibrium is the exact root
    edges = np.concatenate([[0.0], np.logspace(-3, 2, 16), [math.inf]])
    st = _doppler_run(edges, 0.0)
    assert gas_T(st, 1.5)[0] == pytest.approx(gd["T_exact"], abs=1e-12)
    # the paper's 16 groups on [1e-3, 1e2] miss only the far tails
    st = _doppler_run(np.logspace(-3, 2, 17), 0.0)
    assert gas_T(st, 1.5)[0] == pytest.approx(gd["T_exact"], abs=5e-11)


@pytest.mark.parametrize("c_hat,steps", [(1.0, 8), (0.1, 8), (0.1, 1)])
def test_doppler_moving_equilibrium_closed_form(c_hat, steps):
    """v = 1e-3, Eddington pressure, groups covering [0, inf): summed over the
    groups the Doppler terms cancel (Sec. 2.2.1), so the steady state obeys the
    grey relations G^0 = 0: E = b + v.F/c^2 and G^i = 0: F = v (b + E/3), which
    give the E = b (1 + 4v^2/3), F = (4/3) v b equilibrium below eq. Gi_2new to
    second order; with total energy E_gas + (c/c_hat) E and momentum
    rho v + F/(c c_hat) conserved (eqs. egupdate, vupdate) they fix T and v.
    After one step (tau = c_hat dt chi = 1e7 from no radiation) backward Euler
    leaves a disequilibrium of order 1/tau; a step's momentum change is then
    set by the momentum equation itself, which later steps would relax away."""
    v0 = 1e-3
    edges = np.concatenate([[0.0], np.logspace(-3, 2, 16), [math.inf]])
    st = _doppler_run(edges, v0, steps=steps, closure=O.CLOSURE_EDDINGTON, c_hat=c_hat)
    k = 1.0 / c_hat

    def eqs(T, v):
        b = T ** 4
        E = b * (1 + v * v) / (1 - v * v / 3)
        F = v * (b + E / 3)
        return [1.5 * T + 0.5 * v * v + k * E - (1.5 + 0.5 * v0 * v0), v + k * F - v0]
    T_ss, v_ss = mp.findroot(eqs, (mp.mpf("0.6"), mp.mpf(v0)))
    tol = 1e-12 if steps > 1 else 3e-7
    assert gas_T(st, 1.5)[0] == pytest.approx(float(T_ss), rel=tol)
    assert st["mom"][0, 0] == pytest.approx(float(v_ss), rel=10 * tol)
    b = T_ss ** 4
    assert st["erad"].sum() == pytest.approx(float(b * (1 + v_ss ** 2) / (1 - v_ss ** 2 / 3)), rel=tol)
    # the second-order form printed in the paper
    assert st["frad"][0].sum() == pytest.approx(float(4.0 / 3.0 * v_ss * b), rel=1e-6)


def test_doppler_flux_spectrum_against_angle_integral():
    """Group fluxes of the steady state against the angle integral eq. bbF of
    the Doppler-shifted Planck intensity, integrated over each group; the paper
    reports agreement better than 0.1%."""
    bound = golden("doppler_equilibrium.txt")["flux_rel_error_bound"]
    edges = np.logspace(-3, 2, 17)
    st = _doppler_run(edges, 1e-3, steps=8)
    T = gas_T(st, 1.5)[0]
    beta = st["mom"][0, 0]
    # our normalisation: 4 pi B_nu / c integrates to a_R T^4; eq. bbF uses
    # B_nu = 2 nu^3/(e^(nu/T) - 1): factor 15 / (8 pi^5)
    K = 15 / (8 * mp.pi ** 5)

    def Fnu(nu):
        return 2 * mp.pi * mp.quad(lambda mu: mu * 2 * nu ** 3 / mp.expm1(nu / T * (1 - beta * mu)),
                                   [-1, 1])
    errs = []
    for g in range(16):
        Fg = K * mp.quad(Fnu, [edges[g], edges[g + 1]])
        errs.append(abs(st["frad"][0, g, 0] / float(Fg) - 1.0))
    assert max(errs) < bound
    # the first-order treatment errs by O((v/c)(h nu/k T))^2: tiny below the peak
    x_hi = edges[1:] / T
    assert max(e for e, x in zip(errs, x_hi) if x < 10.0) < 1e-6


def test_diffusion_limit_flux_is_stationary():
    """With E_g = b_g, F_g = F_g,diff (eq. Fdiff) and Eddington pressure, the
    flux-mean opacity of eq. chiDiff makes G^i_g vanish: one implicit step leaves
    F_g unchanged up to the O(v^2) energy exchange.  The slopes are chosen so
    that eq. chiDiff stays inside the group's opacity range (checked here)."""
    G = 16
    edges = synth.log_edges(G)
    rng = np.random.default_rng(12)
    alpha = rng.uniform(-2.5, -0.2, G)
    khat = np.exp(rng.uniform(-1.0, 1.0, G))
    T, rho, tau, v = 1.1e7, 1.3, 5e3, 1e-6 * synth.C_LIGHT
    kappa0 = tau / (synth.C_LIGHT * rho * synth.DT)
    consts = dict(a_rad=synth.A_RAD, h=synth.H_PLANCK, k_B=synth.K_BOLTZ)
    st = _equilibrium_state(edges, T, rho, kappa0, consts, synth.C_V)
    x = synth.H_PLANCK * edges / (synth.K_BOLTZ * T)
    aT4 = synth.A_RAD * T ** 4
    b = st["erad"][:, 0]
    dnb = np.array([float(aT4 * (mp_nuB(x[g + 1]) - mp_nuB(x[g]))) for g in range(G)])
    for g in range(G):  # precondition: eq. chiDiff is a proper mean here
        r = edges[g + 1] / edges[g]
        chiB = float(mp.quad(lambda u: u ** (alpha[g] - 1), [1, r]) / mp.log(r))
        dnxb = float(aT4 * (r ** alpha[g] * mp_nuB(x[g + 1]) - mp_nuB(x[g])))
        raw = ((chiB + chiB / 3) * b[g] + (alpha[g] * chiB * b[g] - dnxb) / 3) / (4 * b[g] / 3 - dnb[g] / 3)
        assert r ** alpha[g] < raw < 1.0
    Fdiff = v * (4.0 / 3.0 * b - dnb / 3.0)
    st["frad"][0, :, 0] = Fdiff
    st["mom"][0, 0] = rho * v
    st["egas"][0] += 0.5 * rho * v * v
    p = O.Params(a_rad=synth.A_RAD, c_v=synth.C_V, dt=synth.DT, closure=O.CLOSURE_EDDINGTON)
    grp = O.Groups(edges, khat, alpha)
    out = O.source_update(st, p, grp)
    assert out["status"][0] == 0
    np.testing.assert_allclose(out["frad"][0, :, 0], Fdiff, rtol=1e-8)
    np.testing.assert_allclose(out["frad"][1:], 0.0, atol=0)
    # the same state with the Doppler term of eq. Fdiff dropped is not stationary
    st2 = dict(st, frad=st["frad"].copy())
    st2["frad"][0, :, 0] = v * 4.0 / 3.0 * b
    out2 = O.source_update(st2, p, grp)
    assert np.max(np.abs(out2["frad"][0, :, 0] / st2["frad"][0, :, 0] - 1)) > 1e-3


def test_flux_mean_opacity_is_held_to_the_group_range():
    """Positive in-group slopes in the Rayleigh-Jeans part make eq. chiDiff
    with the alpha_Q = -1 means leave [min chi_0, max chi_0] of the group (even
    turn negative); the oracle holds it to that range (a positively weighted
    mean of chi_0 cannot leave it)."""
    edges = synth.log_edges(16)
    alpha = np.full(16, 2.69)
    t = O.group_terms(O.Params(a_rad=synth.A_RAD), O.Groups(edges, np.ones(16), alpha), 1.0, 1.1e7)
    r = edges[1:] / edges[:-1]
    assert np.all(t["chiF"] >= 1.0 - 1e-15) and np.all(t["chiF"] <= r ** 2.69 * (1 + 1e-15))
    assert t["chiF"][0] == pytest.approx(1.0, rel=1e-15)  # clamped from below


def test_first_order_limit_is_the_four_force():
    """For a tiny step the implicit update is the explicit four-force of eqs.
    G0_3 and G1_3 (PPL fixed slope, Eddington pressure) to first order in dt;
    every ingredient of the expected value comes from quadrature or the
    paper's closed forms, none from the oracle."""
    edges = synth.log_edges(4)
    rng = np.random.default_rng(4)
    alpha = np.array([-1.7, -0.8, -2.4, 1.4])
    khat = np.array([1.5, 0.7, 2.0, 0.4])
    T, rho, kappa0 = 1.2e7, 0.9, 3.0
    c = synth.C_LIGHT
    x = synth.H_PLANCK * edges / (synth.K_BOLTZ * T)
    aT4 = synth.A_RAD * T ** 4
    b = np.array([float(aT4 * mp_band(x[g], x[g + 1])) for g in range(4)])
    E = b * np.array([1.02, 0.97, 1.05, 0.9])
    v = np.array([0.004, -0.002, 0.003]) * c
    F = np.array([0.9 * c * E[g] * d / np.linalg.norm(d) for g, d in enumerate(rng.normal(size=(4, 3)))])
    st = {"rho": np.array([rho]), "mom": (rho * v)[:, None].copy(),
          "egas": np.array([rho * synth.C_V * T + 0.5 * rho * v @ v]), "kappa0": np.array([kappa0]),
          "erad": E[:, None].copy(), "frad": F.T[:, :, None].copy(), "src": None}
    dt = 1e-19
    p = O.Params(a_rad=synth.A_RAD, c_v=synth.C_V, dt=dt, closure=O.CLOSURE_EDDINGTON)
    out = O.source_update(st, p, O.Groups(edges, khat, alpha))
    assert out["status"][0] == 0
    for g in range(4):
        r = edges[g + 1] / edges[g]
        chim = rho * kappa0 * khat[g]
        chiB = float(chim * mp.quad(lambda u: u ** (alpha[g] - 1), [1, r]) / mp.log(r))
        d0, d1 = mp_nuB(x[g]), mp_nuB(x[g + 1])
        dnb = float(aT4 * (d1 - d0))
        dnxb = float(aT4 * chim * (r ** alpha[g] * d1 - d0))
        chiF = ((chiB + chiB / 3) * b[g] + (alpha[g] * chiB * b[g] - dnxb) / 3) / (4 * b[g] / 3 - dnb / 3)
        assert min(1, r ** alpha[g]) < chiF / chim < max(1, r ** alpha[g])  # a proper mean
        G0 = chiB * b[g] - chiB * E[g] + (1 + alpha[g]) * chiF * (v @ F[g]) / c ** 2
        dE = (out["erad"][g, 0] - E[g]) / (c * dt)
        assert dE == pytest.approx(G0, rel=1e-5)
        Gi = -chiF * F[g] + v * (chiB * b[g] - dnxb / 3) + (1 + alpha[g]) * chiB * v * E[g] / 3
        dF = (out["frad"][:, g, 0] - F[g]) / (c * dt)
        np.testing.assert_allclose(dF, Gi, rtol=1e-5, atol=1e-5 * np.abs(Gi).max())


def test_invalid_cells_are_untouched():
    w = synth.preset("tiny", n_cells=6)
    st = synth.to_numpy(w.state)
    st["rho"][1] = -1.0
    st["egas"][2] = np.nan
    st["egas"][3] = 0.25 * (st["mom"][:, 3] ** 2).sum() / st["rho"][3]  # E_int < 0
    out = O.source_update(st, oracle_params(w), oracle_groups(w))
    assert list(out["status"][1:4]) == [3, 3, 3]
    for k in ("erad", "frad", "mom"):
        np.testing.assert_array_equal(out[k][..., 1:4], st[k][..., 1:4])
    assert np.all(out["status"][[0, 4, 5]] == 0)


@pytest.mark.parametrize("tau", [1e-2, 1.0, 10.0])
def test_imex_step_amplification_of_a_small_grey_disequilibrium(tau):
    """The IMEX composition without transport acts on a small grey
    disequilibrium D like y' = -lambda y does under it: stage 1 divides by
    1 + z, stage 2 averages with the start and divides by 1 + z/2, so one
    step multiplies D by ((1 + 1/(1 + z))/2)/(1 + z/2) = 1/(1 + z),
    z = dt chi (c_hat + c kappa).  (z stays small enough that the O(delta z)
    nonlinear part and the solve's tolerance stay below the 2e-6 asked.)"""
    rho, T0, delta = 1.0, 1.0e7, 1e-7
    c, a, cv = synth.C_LIGHT, synth.A_RAD, synth.C_V
    chi = tau / (c * synth.DT)
    E0 = a * T0 ** 4
    st = {"rho": np.array([rho]), "mom": np.zeros((3, 1)), "egas": np.array([rho * cv * T0]),
          "kappa0": np.array([chi / rho]), "erad": np.array([[E0 * (1 + delta)]]),
          "frad": np.zeros((3, 1, 1)), "src": None}
    p = O.Params(c=c, c_hat=c, a_rad=a, c_v=cv, dt=synth.DT)
    edges = np.array([0.0, math.inf])
    out = O.imex_step(st, p, O.Groups(edges, np.ones(1), np.zeros(1)))
    kap = 4 * a * T0 ** 3 / (rho * cv)
    T1 = gas_T(out | {"rho": st["rho"]}, cv)[0]
    D0 = -delta * E0
    D1 = kap * rho * cv * (T1 - T0) - (out["erad"][0, 0] - E0)
    z = synth.DT * chi * (c + c * kap)
    assert D1 / D0 == pytest.approx(1.0 / (1.0 + z), rel=2e-6)
    # total energy kept
    e0 = st["egas"][0] + st["erad"][0, 0]
    assert abs(out["egas"][0] + out["erad"][0, 0] - e0) <= 4e-16 * e0
