"""The pins must catch plausible mistakes: each mutant below plants one in a copy of
the oracle (on the CPU), and the pin suite has to fail on it."""
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

MUTANTS = {
    "equilibrium_printed_1_6": ("4.5 * cu * cu", "(1.0 / 6.0) * cu * cu"),
    "forcing_second_order_sign": ("double B = 1.0 - 0.5 * omega_p;", "double B = 1.0 + 0.5 * omega_p;"),
    "forcing_first_order_unweighted": ("double A = 3.0 * (1.0 - 0.5 * omega_m);", "double A = 3.0;"),
    "trt_rates_swapped": ("- omega_p * (fp - ep) - omega_m * (fm - em)", "- omega_m * (fp - ep) - omega_p * (fm - em)"),
    "half_force_shift_dropped": ("u[a] = (j[a] + 0.5 * F[a]) / r;", "u[a] = j[a] / r;"),
    "source_transposed_gradient": ("b += T[k][j] * G[k * 3 + i];", "b += T[k][j] * G[i * 3 + k];"),
    "source_relaxation_dropped": (" - inv_l * T[i][j];", ";"),
    "ctu_transverse_axes": ("int a = (k + 1) % 3, b = (k + 2) % 3;", "int a = k, b = (k + 2) % 3;"),
    "ctu_inflow_overlap_of_receiver": ("tin = (1.0 - fabs(u[(long)a * n + nb])) * (1.0 - fabs(u[(long)b * n + nb]));",
                                       "tin = (1.0 - fabs(u[(long)a * n + r])) * (1.0 - fabs(u[(long)b * n + r]));"),
    "divu_offdiagonal_trace": ("double divu = (G[0] + G[4]) + G[8];", "double divu = (G[0] + G[1]) + G[8];"),
    "giesekus_sign": ("S[c] = S[c] - s->gk * q;", "S[c] = S[c] + s->gk * q;"),
    "giesekus_product_index": ("q += tr[COMP[i][k]] * tr[COMP[k][j]];", "q += tr[COMP[i][k]] * tr[COMP[i][j]];"),
    "upwind_inflow_sign": ("double vin = -sg * u[(long)k * n + nb];", "double vin = sg * u[(long)k * n + nb];"),
    "force_extrapolation_zero": ("double tf = fl ? 0.5 * (tr + tau[(long)c * s->n + nb]) : tr;",
                                 "double tf = fl ? 0.5 * (tr + tau[(long)c * s->n + nb]) : 0.0;"),
    "wall_gradient_uses_cell": ("double up = is_fluid(s, np_) ? 0.5 * (ur + u[(long)j * n + np_]) : ubp[j];",
                                "double up = is_fluid(s, np_) ? 0.5 * (ur + u[(long)j * n + np_]) : ur;"),
    "moving_wall_sign": ("s->fn[(long)OPP[i] * n + r] = fsi - X;", "s->fn[(long)OPP[i] * n + r] = fsi + X;"),
    "momentum_exchange_sign": ("double m = 2.0 * s->f[(long)i * n + r] - X;", "double m = 2.0 * s->f[(long)i * n + r] + X;"),
    "created_stress_mean": ("sum[c] / (double)(Nf[r] + 1)", "sum[c] / (double)(Nf[r] ? Nf[r] : 1)"),
    "destroyed_impulse_sign": ("P->dP[a] += Pm[a];", "P->dP[a] -= Pm[a];"),
    "symplectic_order": ("P->X[a] += P->v[a];\n", "P->X[a] += P->v[a] - (P->Fme[a] + P->Fext[a]) / P->m;\n"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", "lbve_oracle.c")).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    src = src.replace(old, new)
    (tmp_path / "lbve_oracle.c").write_text(src)
    shutil.copy(os.path.join(ROOT, "oracle", "lbve_oracle.h"), tmp_path / "lbve_oracle.h")
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                    str(tmp_path / "lbve_oracle.c"), "-o", str(so), "-lm"], check=True)
    env = dict(os.environ, LBVE_ORACLE_LIB=str(so), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(HERE, "test_oracle_pins.py")], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
