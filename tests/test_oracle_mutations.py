"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a private copy of oracle/rlb_oracle.c (on the
CPU, in a temporary directory), builds it, and runs the pin suite against it
in a subprocess; the suite must fail.  The mistakes are the ones a careful
reader could make transcribing the paper: the printed Delta f^{a+} in Eq. 50,
the printed one-cell-downstream flux difference of Eq. 47, a doubled
off-diagonal equilibrium coefficient, a sign in Eq. 58, lambda_0 != 0 in
Eq. 55, a dropped nu in the collision prefactor of Eq. 57, the wrong sign of
the extrapolated equilibrium, n = N^0 gamma, a flipped lattice vector, tau
without nu^2 (Eq. 41), minmod taking the larger slope (Eq. 53), and in the
solid cells of the astrophysical run (Sec. III): no reset, a moving or a
wrong-pressure cloud state; in the basic model's lattice (Sec. II): a
mistyped weight, doubled diagonals, swapped number weights; Euler mode
(Sec. III) taking the equilibria of the unstreamed state; the bulk term of
Eq. 57 applied to the number distribution as well; an inlet ghost whose
pressure drops the temperature; open ends that reflect instead of copying
the edge cell; the h equation relaxing to h^eq(t) instead of the
extrapolated 2 h^eq(t) - h^eq(t - dt), and the f equation doing the same;
nu = 1 in place of sqrt(13) in every constant of the extended lattice (a
reading of the garbled lattice constants that the tests of the readings
reject).
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rlb_oracle.c")
PINS = ["tests/test_oracle_lattice.py", "tests/test_oracle_equilibrium.py",
        "tests/test_oracle_stream.py", "tests/test_oracle_step.py", "tests/test_oracle_solid.py",
        "tests/test_oracle_basic.py", "tests/test_oracle_hydro.py"]

MUTATIONS = {
    "printed_delta_plus_in_fR": ("fR -= 0.5 * orc_minmod(dm_y, dm_yp1);",
                                 "fR -= 0.5 * orc_minmod(dp_y, fplus(p, q2) - fplus(p, q1));"),
    "flux_difference_one_cell_downstream": (
        "        s += flux(pa[a], q[1], q[2], q[3], q[4], p->limiter)\n"
        "           - flux(pa[a], q[0], q[1], q[2], q[3], p->limiter);",
        "        s += flux(pa[a], q[2], q[3], q[4], q[4], p->limiter)\n"
        "           - flux(pa[a], q[1], q[2], q[3], q[4], p->limiter);"),
    "off_diagonal_coefficient_doubled": ("const double a2 = 4.0 * P / L->m22;",
                                         "const double a2 = 8.0 * P / L->m22;"),
    "heq_first_order_sign": ("(L->c0_over_ct + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu)",
                             "(L->c0_over_ct - 3.0 * cu + 4.5 * cu * cu - 1.5 * uu)"),
    "bulk_on_rest_population": ("if (i != 0) sf[i] += kbulk", "if (i >= 0) sf[i] += kbulk"),
    "collision_prefactor_without_nu": ("omega = L->c0_over_ct * NU * dt / tau;",
                                       "omega = L->c0_over_ct * dt / tau;"),
    "extrapolation_sign": ("omega * (2.0 * feq[i] - feqp[i])", "omega * (2.0 * feqp[i] - feq[i])"),
    "density_times_gamma": ("macro[4] = mom[4] / gamma;", "macro[4] = mom[4] * gamma;"),
    "flipped_lattice_vector": ("l->c[i][b] = dshell * ca * s2;",
                               "l->c[i][b] = (i == 12 ? -dshell : dshell) * ca * s2;"),
    "tau_without_nu_squared": ("return 0.5 + NU * NU * eta / (4.0 * P);",
                               "return 0.5 + eta / (4.0 * P);"),
    "basic_diagonal_weight_typo": ("w2 = r2 * nu * nu / 1083.0;", "w2 = r2 * nu * nu / 1038.0;"),
    "basic_diagonals_doubled": ("const double dshell = basic ? 1.0 : 2.0;",
                                "const double dshell = basic ? 2.0 : 2.0;"),
    "basic_number_weights_swapped": ("for (i = 1; i <= 6; ++i) l->wh[i] = 1.0 / 18.0;",
                                     "for (i = 1; i <= 6; ++i) l->wh[i] = 1.0 / 36.0;"),
    "solid_reset_skipped": ("if (!mask[idx]) continue;", "if (mask[idx] || !mask[idx]) continue;"),
    "solid_state_moving": ("const double rest[3] = {0.0, 0.0, 0.0};", "const double rest[3] = {0.05, 0.0, 0.0};"),
    "solid_pressure_without_T": ("orc_feq(n * T, rest, fe);", "orc_feq(n, rest, fe);"),
    "euler_mode_without_streaming": ("            fs[i] = f[i] + sf[i];\n            hs[i] = h[i] + sh[i];",
                                     "            fs[i] = f[i];\n            hs[i] = h[i];"),
    "bulk_term_on_number_distribution": (
        "sh[i] = stream_at(p, H, i, k->ghost_h[i], L->c[i], kstream, x, y, z);  /* no lambda term */",
        "sh[i] = stream_at(p, H, i, k->ghost_h[i], L->c[i], kstream, x, y, z)"
        " + (i != 0 ? kbulk * lap_at(p, H, i, k->ghost_h[i], x, y, z) : 0.0);"),
    "inlet_pressure_without_T": ("orc_feq(p->inlet_n * p->inlet_T, up, k->ghost_f);",
                                 "orc_feq(p->inlet_n, up, k->ghost_f);"),
    "outflow_ghosts_reflecting": ("if (bc == ORC_BC_OUTFLOW) return c < 0 ? 0 : n - 1;",
                                  "if (bc == ORC_BC_OUTFLOW) return c < 0 ? -c : 2 * n - 2 - c;"),
    "equilibrium_not_extrapolated": (
        "fo[i] = (f[i] + sf[i] + omega * (2.0 * feq[i] - feqp[i])) / (1.0 + omega);",
        "fo[i] = (f[i] + sf[i] + omega * feq[i]) / (1.0 + omega);"),
    "nu_one_everywhere": ("const double nu = basic ? sqrt(19.0) : sqrt(13.0);",
                          "const double nu = basic ? sqrt(19.0) : 1.0;"),
    "number_equilibrium_not_extrapolated": (
        "ho[i] = (h[i] + sh[i] + omega * (2.0 * heq[i] - heqp[i])) / (1.0 + omega);",
        "ho[i] = (h[i] + sh[i] + omega * heq[i]) / (1.0 + omega);"),
    "minmod_takes_larger_slope": ("return 0.5 * fmin(fabs(X), fabs(Y)) * (sgn(X) + sgn(Y));",
                                  "return 0.5 * fmax(fabs(X), fabs(Y)) * (sgn(X) + sgn(Y));"),
}


def _run_pins(tmp_path, source):
    mutated = tmp_path / "rlb_oracle.c"
    mutated.write_text(source)
    (tmp_path / "rlb_oracle.h").write_text(open(os.path.join(ROOT, "oracle", "rlb_oracle.h")).read())
    lib = tmp_path / "liboracle_mut.so"
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-o", str(lib), str(mutated), "-lm"], check=True)
    env = dict(os.environ, RLB_ORACLE_LIB=str(lib))
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           *PINS], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_unmutated_copy_passes(tmp_path):
    r = _run_pins(tmp_path, open(SRC).read())
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    r = _run_pins(tmp_path, src.replace(old, new))
    assert r.returncode != 0, f"pins did not catch mutation {name}:\n{r.stdout[-2000:]}"
