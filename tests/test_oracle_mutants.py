"""The pins hold the oracle: a plausible mistake planted in it fails them.

Each mutant below is one mistake of the kind a restatement of the paper can
make: a dropped term, a wrong sign, a wrong index, a transposed operand, a
wrong constant.  The test copies the oracle (C and Python, the update and the
warm start's network) and the pin tests into a scratch tree, plants the
mistake in the copy, rebuilds the copy's library there and runs the pins
(``test_oracle_properties.py``, ``test_oracle_mlp.py``,
``test_oracle_ppl_free.py``, ``test_oracle_pins.py``) against it.  The
unmodified copy must pass; every mutant must make at least one pin fail.  Nothing is written to the repository: the mistakes exist only
in the scratch copies, on the CPU.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

pytest.importorskip("mpmath")  # the pins that quadrature fixes need it

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C = "oracle/rhd_oracle.c"
PY = "oracle/__init__.py"
MLP = "oracle/mlp.py"

# (name, what the mistake breaks, [(file, exact text, replacement), ...])
MUTANTS = [
    ("wien_series_term", "Planck integral above x = 2: the 6/n^4 term of the series dropped",
     [(C, "6.0 / (dn * dn * dn * dn)", "0.0 / (dn * dn * dn * dn)")]),
    ("bernoulli_sign", "Planck integral below x = 2: alternating sign of the Bernoulli terms",
     [(C, "(j % 2 == 1) ? 1.0 : -1.0", "(j % 2 == 1) ? -1.0 : 1.0")]),
    ("bernoulli_b1", "Planck integral below x = 2: the B_1 term x^4/8 written x^4/6",
     [(C, "x3 * x / 8.0", "x3 * x / 6.0")]),
    ("planck_norm", "normalisation 15/pi^4 of the Planck function written 15/pi^3",
     [(C, "return 15.0 / (ORC_PI * ORC_PI * ORC_PI * ORC_PI);",
       "return 15.0 / (ORC_PI * ORC_PI * ORC_PI);")]),
    ("nuB_power", "edge term nu B_nu: x^4/(e^x - 1) written x^3/(e^x - 1)",
     [(C, "return orc_norm15() * x * x * x * x / expm1(x);",
       "return orc_norm15() * x * x * x / expm1(x);")]),
    ("a_T4", "a_R T^4 written a_R T^3",
     [(C, "double fac = p->a_rad * T * T * T * T;", "double fac = p->a_rad * T * T * T;")]),
    ("chiQg_exponent", "eq. chiQg: numerator exponent alpha_chi + alpha_Q + 1 without the 1",
     [(C, "orc_pow_bracket(alpha_chi + alpha_Q + 1.0, r)", "orc_pow_bracket(alpha_chi + alpha_Q, r)")]),
    ("chiQg_denominator", "eq. chiQg: denominator exponent alpha_Q + 1 written alpha_Q",
     [(C, "orc_pow_bracket(alpha_Q + 1.0, r);", "orc_pow_bracket(alpha_Q, r);")]),
    ("break_on_edge", "group table: a breakpoint on an edge given to the group below",
     [(C, "right ? (nu_break[b] <= nu) : (nu_break[b] < nu)",
       "right ? (nu_break[b] < nu) : (nu_break[b] <= nu)")]),
    ("ppl_slope_sign", "group table: in-group slope divided by ln(nu_-/nu_+)",
     [(C, "(lk1 - lk0) / log(n1 / n0);", "(lk1 - lk0) / log(n0 / n1);")]),
    ("pc_centre", "PC: opacity at the arithmetic instead of the logarithmic centre",
     [(C, "else centre = sqrt(n0 * n1);", "else centre = 0.5 * (n0 + n1);")]),
    ("free_nubar", "App. A: arithmetic instead of geometric group frequency",
     [(C, "double nua = sqrt(edges[g] * edges[g + 1]);", "double nua = 0.5 * (edges[g] + edges[g + 1]);"),
      (C, "double nub = sqrt(edges[g + 1] * edges[g + 2]);",
       "double nub = 0.5 * (edges[g + 1] + edges[g + 2]);")]),
    ("free_qbar", "App. A: group values not divided by the group width",
     [(C, "double qa = Q[g] / (edges[g + 1] - edges[g]);", "double qa = Q[g];"),
      (C, "double qb = Q[g + 1] / (edges[g + 2] - edges[g + 1]);", "double qb = Q[g + 1];")]),
    ("free_maxmod", "App. A: the larger of two positive slopes instead of the smaller",
     [(C, "if (a > 0.0 && b > 0.0) return a < b ? a : b;", "if (a > 0.0 && b > 0.0) return a > b ? a : b;")]),
    ("free_opposite", "App. A: slopes of opposite sign averaged instead of giving 0",
     [(C, "  return 0.0;\n}\n\nvoid orc_ppl_free_slopes", "  return 0.5 * (a + b);\n}\n\nvoid orc_ppl_free_slopes")]),
    ("free_end_groups", "App. A: first and last group alpha = 0 instead of -1",
     [(C, "alpha_out[g] = -1.0; /* eq. minmod", "alpha_out[g] = 0.0; /* eq. minmod")]),
    ("free_left_index", "App. A: the left slope taken at the right edge",
     [(C, "double sl = orc_edge_slope(edges, Q, g - 1);", "double sl = orc_edge_slope(edges, Q, g);")]),
    ("free_alphaE_from_b", "App. A: the E_nu slope fitted to b_g instead of E_g",
     [(C, "if (erad0) orc_ppl_free_slopes(G, gt->edges, erad0, aE);",
       "if (erad0) orc_ppl_free_slopes(G, gt->edges, bg, aE);")]),
    ("chiE_with_aB", "chi_E averaged with the spectral index of B_nu",
     [(C, "orc_ppl_mean_opacity(chim, alpha, aE[g], n1 / n0)",
       "orc_ppl_mean_opacity(chim, alpha, aB[g], n1 / n0)")]),
    ("dnb_sign", "Delta_g(nu B_nu) with the edges swapped",
     [(C, "double dnbg = fac * (d1 - d0);", "double dnbg = fac * (d0 - d1);")]),
    ("chi_upper_edge", "chi_0 at the upper edge: r^-alpha instead of r^alpha",
     [(C, "chim * pow(n1 / n0, alpha)", "chim * pow(n0 / n1, alpha)")]),
    ("dnxb_transposed", "Delta_g(nu chi_0 B_nu): the two edge opacities transposed",
     [(C, "fac * (chip * d1 - chim * d0)", "fac * (chim * d1 - chip * d0)")]),
    ("chiDiff_third", "eq. chiDiff: chi_E/3 written chi_E",
     [(C, "((chiBg + chiEg / 3.0) * bg[g]", "((chiBg + chiEg) * bg[g]")]),
    ("chiDiff_sign", "eq. chiDiff: sign of Delta_g(nu chi_0 B_nu)",
     [(C, "(alpha * chiEg * bg[g] - dnxbg) / 3.0", "(alpha * chiEg * bg[g] + dnxbg) / 3.0")]),
    ("chiDiff_denominator", "eq. chiDiff: sign of Delta_g(nu B_nu) in the denominator",
     [(C, "double den = (4.0 / 3.0) * bg[g] - dnbg / 3.0;", "double den = (4.0 / 3.0) * bg[g] + dnbg / 3.0;")]),
    ("levermore_root", "Levermore closure: sqrt(4 - 3 f^2) written sqrt(4 - 4 f^2)",
     [(C, "sqrt(4.0 - 3.0 * f * f)", "sqrt(4.0 - 4.0 * f * f)")]),
    ("closure_iso", "closure: isotropic part (1 + chi)/2 instead of (1 - chi)/2",
     [(C, "double iso = 0.5 * (1.0 - chi)", "double iso = 0.5 * (1.0 + chi)")]),
    ("closure_index", "closure: n_i n_i instead of n_i n_j",
     [(C, "dir * n[i] * n[j]", "dir * n[i] * n[i]")]),
    ("arrowhead_operand", "arrowhead elimination: top row used for the left column",
     [(C, "a -= top[g] * left[g] / diag[g];", "a -= top[g] * top[g] / diag[g];")]),
    ("lu_rhs", "dense LU: right-hand side not eliminated",
     [(C, "      b[i] -= l * b[k];", "      b[i] -= 0.0 * b[k];")]),
    ("T_without_rho", "T = E_int/(rho c_v) written E_int/c_v",
     [(C, "double T = Eint / (c->rho * p->c_v);", "double T = Eint / p->c_v;")]),
    ("kinetic_half", "kinetic energy without the 1/2",
     [(C, "double KE = 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / c->rho;",
       "double KE = (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / c->rho;")]),
    ("work_1_plus_alpha", "eq. Rnew: (1 + alpha) of the work term written alpha",
     [(C, "(1.0 + alpha) * c->chiF[g] * w", "alpha * c->chiF[g] * w")]),
    ("work_dropped", "eq. Rnew: the v.F work term dropped",
     [(C, "tdt * (c->chiB[g] * c->b[g] + (1.0 + alpha) * c->chiF[g] * w)", "tdt * (c->chiB[g] * c->b[g])")]),
    ("emission_chiE", "eq. Rnew: emission with chi_E instead of chi_B",
     [(C, "tdt * (c->chiB[g] * c->b[g] + (1.0 + alpha)", "tdt * (c->chiE[g] * c->b[g] + (1.0 + alpha)")]),
    ("source_dropped", "eq. eupdate: the explicit source S_g dropped",
     [(C, "r[4 + g] = E - (c->E0[g] + S + A) / (1.0 + tdt * chiE);",
       "r[4 + g] = E - (c->E0[g] + A) / (1.0 + tdt * chiE);")]),
    ("flux_dnxb_sign", "eq. fupdate: sign of Delta_g(nu chi_0 B_nu)/3",
     [(C, "double src = c->chiB[g] * c->b[g] - c->dnxb[g] / 3.0;",
       "double src = c->chiB[g] * c->b[g] + c->dnxb[g] / 3.0;")]),
    ("flux_vP_dropped", "eq. fupdate: the (1 + alpha) chi_E v.P term dropped",
     [(C, "tdt * (v[i] * src + (1.0 + alpha) * chiE * vP)", "tdt * (v[i] * src)")]),
    ("flux_denominator", "eq. fupdate: chi_E instead of chi_F in the implicit denominator",
     [(C, "F[i] - num / (1.0 + tdt * c->chiF[g]);", "F[i] - num / (1.0 + tdt * c->chiE[g]);")]),
    ("gas_speed_ratio", "eq. egupdate: c_hat/c instead of c/c_hat",
     [(C, "r[0] = Eint + KE - c->egas0 + (p->c / p->c_hat) * sumR;",
       "r[0] = Eint + KE - c->egas0 + (p->c_hat / p->c) * sumR;")]),
    ("momentum_speeds", "eq. vupdate: 1/c^2 instead of 1/(c c_hat)",
     [(C, "r[1 + i] = m[i] - c->m0[i] + dF[i] / (p->c * p->c_hat);",
       "r[1 + i] = m[i] - c->m0[i] + dF[i] / (p->c * p->c);")]),
    ("writeback_gas", "write-back: E_gas without the c/c_hat factor",
     [(C, "egas[i] = eg0 - (p->c / p->c_hat) * sumR;", "egas[i] = eg0 - sumR;")]),
    ("writeback_mom_sign", "write-back: momentum change with the wrong sign",
     [(C, "mom[(size_t)d * n_cells + i] = m0[d] - dF[d] / (p->c * p->c_hat);",
       "mom[(size_t)d * n_cells + i] = m0[d] + dF[d] / (p->c * p->c_hat);")]),
    ("opacity_T_factor", "temperature factor (T_ref/T)^p instead of (T/T_ref)^p",
     [(C, "pow(T / p->T_ref, p->temp_exponent)", "pow(p->T_ref / T, p->temp_exponent)")]),
    ("imex_theta", "IMEX stage 2 with theta = 1 instead of 1/2",
     [(PY, "dataclasses.replace(p, theta=0.5)", "dataclasses.replace(p, theta=1.0)")]),
    ("imex_average", "IMEX stage 2 started from U(n+1/2) instead of (U(n) + U(n+1/2))/2",
     [(PY, "mid[k] = 0.5 * (np.asarray(state[k], dtype=np.float64) + s1[k])", "mid[k] = s1[k]")]),
    # the learned warm start's reference network
    ("mlp_x_standardise", "network: features multiplied by their sd instead of divided",
     [(MLP, "xn = (np.asarray(x, dtype=np.float64) - xm) / xs", "xn = (np.asarray(x, dtype=np.float64) - xm) * xs")]),
    ("mlp_y_standardise", "network: targets multiplied by their sd instead of divided",
     [(MLP, "(np.asarray(y, dtype=np.float64) - ym) / ys", "(np.asarray(y, dtype=np.float64) - ym) * ys")]),
    ("mlp_destandardise", "network: raw output divided by the target sd",
     [(MLP, "return out * ys + ym", "return out / ys + ym")]),
    ("mlp_layout", "network: weight matrices read [in][out] instead of [out][in]",
     [(MLP, "dtype=np.float64).reshape(o, i))", "dtype=np.float64).reshape(i, o).T)")]),
    ("mlp_loss_sum", "network: loss summed instead of averaged (forward and backward alike)",
     [(MLP, "return float(np.mean((out - yn) ** 2))", "return float(np.sum((out - yn) ** 2))"),
      (MLP, "L = float(np.mean((out - yn) ** 2))", "L = float(np.sum((out - yn) ** 2))"),
      (MLP, "dy = 2.0 * (out - yn) / (B * n_out)", "dy = 2.0 * (out - yn)")]),
    ("mlp_gelu_constant", "network: cubic coefficient of the tanh GELU off by ten",
     [(MLP, "np.tanh(k0 * (z + 0.044715 * z ** 3))", "np.tanh(k0 * (z + 0.0044715 * z ** 3))")]),
    ("mlp_gelu_grad_term", "network: GELU derivative without the factor 3 of the cubic",
     [(MLP, "(1.0 + 3.0 * 0.044715 * z * z)", "(1.0 + 0.044715 * z * z)")]),
    ("mlp_gelu_grad_dropped", "network: backprop through the GELU without its derivative",
     [(MLP, "dz = dh * gelu_grad(zs[l])", "dz = dh")]),
    ("mlp_hidden_bias", "network: hidden-layer bias dropped in the forward pass",
     [(MLP, "z = a @ r(Ws[l]).T + bs[l]", "z = a @ r(Ws[l]).T")]),
    ("mlp_output_bias_grad", "network: output-bias gradient averaged instead of summed",
     [(MLP, "gb[3] = dy.sum(0)", "gb[3] = dy.mean(0)")]),
    ("mlp_bf16_ties", "network: bfloat16 ties rounded up instead of to even",
     [(MLP, "r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000)", "r = ((u + 0x8000) & 0xFFFF0000)")]),
]

_COPY = ["oracle/__init__.py", "oracle/mlp.py", "oracle/rhd_oracle.c", "oracle/rhd_oracle.h",
         "tests/conftest.py", "tests/golden", "paper_2407_18304_gb300/__init__.py",
         "paper_2407_18304_gb300/build.py", "paper_2407_18304_gb300/rhd.py",
         "paper_2407_18304_gb300/synth.py"]
# fast pins first: -x stops a caught mutant at its first failure
_PINS = ["tests/test_oracle_properties.py", "tests/test_oracle_mlp.py", "tests/test_oracle_ppl_free.py",
         "tests/test_oracle_pins.py"]


def _sandbox(base: str, edits) -> str:
    for rel in _COPY + _PINS:
        src, dst = os.path.join(ROOT, rel), os.path.join(base, rel)
        os.makedirs(os.path.dirname(dst), exist_ok=True)
        if os.path.isdir(src):
            shutil.copytree(src, dst)
        else:
            shutil.copy2(src, dst)
    for rel, old, new in edits:
        path = os.path.join(base, rel)
        with open(path) as f:
            text = f.read()
        if text.count(old) != 1:
            raise AssertionError(f"{rel}: the text to replace occurs {text.count(old)} times: {old!r}")
        with open(path, "w") as f:
            f.write(text.replace(old, new))
    return base


def _run(name: str, edits) -> tuple[int, str]:
    base = tempfile.mkdtemp(prefix=f"oracle_mutant_{name}_")
    try:
        _sandbox(base, edits)
        env = dict(os.environ, OMP_NUM_THREADS="1", PYTHONDONTWRITEBYTECODE="1")
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            "-m", "not gpu"] + _PINS, cwd=base, env=env, capture_output=True,
                           text=True, timeout=900)
        lines = [ln for ln in r.stdout.splitlines() if ln.startswith(("FAILED", "ERROR"))]
        return r.returncode, (lines[0] if lines else r.stdout[-400:] + r.stderr[-400:])
    finally:
        shutil.rmtree(base, ignore_errors=True)


@pytest.fixture(scope="module")
def outcomes():
    jobs = [("unmodified", [])] + [(n, e) for n, _, e in MUTANTS]
    with ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        futs = {n: ex.submit(_run, n, e) for n, e in jobs}
        return {n: f.result() for n, f in futs.items()}


def test_unmodified_copy_passes_the_pins(outcomes):
    rc, why = outcomes["unmodified"]
    assert rc == 0, why


@pytest.mark.parametrize("name,what", [(n, w) for n, w, _ in MUTANTS], ids=[n for n, _, _ in MUTANTS])
def test_planted_mistake_fails_a_pin(outcomes, name, what):
    rc, why = outcomes[name]
    assert rc != 0, f"no pin fails when the oracle has this mistake: {what}"
    assert rc == 1, f"the pins did not run to completion (exit code {rc}): {why}"
