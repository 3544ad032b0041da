"""Properties the mathematics fixes for the oracle's building blocks, checked
on many random inputs (hypothesis; CPU only).

* Planck band fractions are additive over adjacent bands in every regime
  (both sides of the series switch at x = 2, the Wien tail), and the band
  over [0, inf) is 1.
* The M1 (Levermore) pressure tensor of any admissible (E, F): symmetric,
  trace E, n.P.n = chi E, eigenvalues in [0, E]; the Eddington factor chi
  rises from 1/3 (isotropic) to 1 (free streaming) with the reduced flux.
* Eq. chiQg is a mean of the in-group powerlaw opacity over a positive
  spectrum, so it lies between the opacity's values at the two group edges,
  whatever the spectral index; a flat opacity gives its own value.
* Appendix A: on any uneven bins, group values of a powerlaw spectrum
  binned as Qbar = nubar^k give every interior group the index k.
* The arrowhead elimination solves the same system as a dense solver.
"""
import math

import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle as O  # noqa: E402

SET = settings(max_examples=300, deadline=None, derandomize=True)
xs = st.floats(min_value=1e-4, max_value=600.0, allow_nan=False, allow_infinity=False)


@SET
@given(xs, xs, xs)
def test_planck_bands_are_additive(a, b, c):
    a, b, c = sorted((a, b, c))
    if not (a < b < c):
        return
    whole = O.planck_band(a, c)
    parts = O.planck_band(a, b) + O.planck_band(b, c)
    assert abs(whole - parts) <= 4e-16 + 4e-15 * whole
    assert 0.0 <= O.planck_band(a, b) <= 1.0
    assert O.planck_band(0.0, math.inf) == pytest.approx(1.0, abs=1e-15)
    assert O.planck_band(0.0, a) + O.planck_band(a, math.inf) == pytest.approx(1.0, abs=2e-15)


@SET
@given(st.floats(1e-30, 1e30), st.floats(0.0, 1.0), st.floats(-1.0, 1.0), st.floats(-1.0, 1.0),
       st.floats(-1.0, 1.0))
def test_m1_pressure_tensor_properties(E, f, u, v, w):
    n = np.array([u, v, w])
    if np.linalg.norm(n) < 1e-3:
        return
    n = n / np.linalg.norm(n)
    c = 3.0e10
    F = f * c * E * n
    P = O.closure(O.CLOSURE_M1, c, E, F)
    scale = E * (1 + 1e-12)
    np.testing.assert_allclose(P, P.T, rtol=0, atol=1e-15 * scale)
    assert np.trace(P) == pytest.approx(E, rel=1e-14)
    ev = np.linalg.eigvalsh(0.5 * (P + P.T))
    assert ev.min() >= -1e-14 * E and ev.max() <= E * (1 + 1e-14)
    if f > 0.0:
        chi = n @ P @ n / E
        assert 1.0 / 3.0 - 1e-14 <= chi <= 1.0 + 1e-14
        # the factor grows with the reduced flux
        P2 = O.closure(O.CLOSURE_M1, c, E, min(1.0, f * 1.1 + 1e-3) * c * E * n)
        assert n @ P2 @ n / E >= chi - 1e-14


@SET
@given(st.floats(0.01, 100.0), st.floats(-6.0, 6.0), st.floats(-6.0, 6.0), st.floats(1.0001, 1e4))
def test_ppl_mean_lies_between_the_edge_opacities(chi_minus, alpha_chi, alpha_Q, r):
    m = O.ppl_mean_opacity(chi_minus, alpha_chi, alpha_Q, r)
    lo, hi = sorted((chi_minus, chi_minus * r ** alpha_chi))
    assert lo * (1 - 1e-12) <= m <= hi * (1 + 1e-12)
    assert O.ppl_mean_opacity(chi_minus, 0.0, alpha_Q, r) == pytest.approx(chi_minus, rel=1e-13)


@SET
@given(st.lists(st.floats(0.05, 2.0), min_size=3, max_size=12), st.floats(-4.0, 4.0))
def test_free_slopes_recover_a_binned_powerlaw(widths, k):
    edges = 1e14 * np.exp(np.concatenate([[0.0], np.cumsum(widths)]))
    nubar = np.sqrt(edges[:-1] * edges[1:])
    Q = nubar ** k * np.diff(edges)
    a = O.ppl_free_slopes(edges, Q)
    assert a[0] == -1.0 and a[-1] == -1.0
    np.testing.assert_allclose(a[1:-1], k, rtol=0, atol=1e-9 * max(1.0, abs(k)))


@SET
@given(st.integers(1, 40), st.integers(0, 2 ** 32 - 1))
def test_arrowhead_matches_a_dense_solve(n, seed):
    rng = np.random.default_rng(seed)
    top, left = rng.normal(size=n), rng.normal(size=n)
    diag = rng.choice([-1.0, 1.0], size=n) * rng.uniform(0.5, 10.0, size=n)
    a00 = rng.choice([-1.0, 1.0]) * (1.0 + np.abs(top * left / diag).sum())
    A = np.zeros((n + 1, n + 1))
    A[0, 0], A[0, 1:], A[1:, 0] = a00, top, left
    A[np.arange(1, n + 1), np.arange(1, n + 1)] = diag
    rhs = rng.normal(size=n + 1)
    x = O.arrowhead_solve(a00, top, left, diag, rhs)
    ref = np.linalg.solve(A, rhs)
    cond = np.linalg.cond(A)
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-14 * cond * max(1.0, np.abs(ref).max()))
