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
    "force_extrapolation_zero": ("double tf = fl ? 0.5 * (tr + tn6[c]) : tr;",
                                 "double tf = fl ? 0.5 * (tr + tn6[c]) : 0.0;"),
    "wall_gradient_uses_cell": ("double up = is_fluid(s, np_) ? 0.5 * (ur + u[(long)j * n + np_]) : ubp[j];",
                                "double up = is_fluid(s, np_) ? 0.5 * (ur + u[(long)j * n + np_]) : ur;"),
    "moving_wall_sign": ("s->fn[(long)OPP[i] * n + r] = fsi - X;", "s->fn[(long)OPP[i] * n + r] = fsi + X;"),
    "momentum_exchange_sign": ("double m = 2.0 * s->f[(long)i * n + r] - X;", "double m = 2.0 * s->f[(long)i * n + r] + X;"),
    "created_stress_mean": ("sum[c] / (double)(Nf[r] + 1)", "sum[c] / (double)(Nf[r] ? Nf[r] : 1)"),
    "destroyed_impulse_sign": ("P->dP[a] += Pm[a];", "P->dP[a] -= Pm[a];"),
    "symplectic_order": ("P->X[a] += P->v[a];\n", "P->X[a] += P->v[a] - (P->Fme[a] + P->Fext[a]) / P->m;\n"),
    "fene_relaxation_without_closure": ("S[c] = a + b - s->inv_l * (fA * tr[c] - (i == j ? 1.0 : 0.0));",
                                        "S[c] = a + b - s->inv_l * (tr[c] - (i == j ? 1.0 : 0.0));"),
    "fene_stress_identity_scaled": ("tau[c] = (eta_p / lambda_p) * (f * A[c] - (c < 3 ? 1.0 : 0.0));",
                                    "tau[c] = (eta_p / lambda_p) * f * (A[c] - (c < 3 ? 1.0 : 0.0));"),
    "fene_trace_offdiagonal": ("double fA = 1.0 / (1.0 - (tr[0] + tr[1] + tr[2]) / s->p.fene_L2);",
                               "double fA = 1.0 / (1.0 - (tr[0] + tr[1] + tr[3]) / s->p.fene_L2);"),
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


# Mistakes in the arithmetic of single boundary-adjacent cells.  Each keeps every integral,
# balance and analytic profile of the pin suite intact (it survives test_oracle_pins.py),
# and only the cell-by-cell brute-force comparison (test_oracle_brute_force.py) sees it.
BRUTE_FORCE_ONLY = {
    # a cell between two solid faces along an axis (a one-cell gap) gets no gradient there
    "gradient_between_two_solid_faces": (
        "G[k * 3 + j] = up - um;",
        "G[k * 3 + j] = (!is_fluid(s, np_) && !is_fluid(s, nm_)) ? 0.0 : up - um;"),
    # the stress face value towards a particle cell taken as zero, not tau(r)
    "force_extrapolation_next_to_particle": (
        "double tf = fl ? 0.5 * (tr + tn6[c]) : tr;",
        "double tf = fl ? 0.5 * (tr + tn6[c]) : (nb >= 0 && s->flag[nb] >= ORC_PART0 ? 0.0 : tr);"),
    # the torque lever arm of a momentum-exchange link measured from the fluid cell
    "torque_lever_arm_of_fluid_cell": (
        "displacement(s, nb, P->X, d);\n                cross(d, Fl, T);",
        "displacement(s, r, P->X, d);\n                cross(d, Fl, T);"),
    # the density of a created cell averaged over its D3Q7 neighbours only
    "created_density_face_neighbours_only": (
        "for (int i = 1; i < 19; ++i) {\n            long nb = neighbour(s, r, C[i][0], C[i][1], C[i][2]);\n"
        "            if (nb < 0 || kind[nb] != 1) continue;",
        "for (int i = 1; i < 7; ++i) {\n            long nb = neighbour(s, r, C[i][0], C[i][1], C[i][2]);\n"
        "            if (nb < 0 || kind[nb] != 1) continue;"),
}


def _mutant_lib(tmp_path, old, new):
    src = open(os.path.join(ROOT, "oracle", "lbve_oracle.c")).read()
    assert src.count(old) == 1, "mutation site not found or not unique"
    (tmp_path / "lbve_oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ROOT, "oracle", "lbve_oracle.h"), tmp_path / "lbve_oracle.h")
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                    str(tmp_path / "lbve_oracle.c"), "-o", str(so), "-lm"], check=True)
    return so


def _run_suite(so, test_file):
    env = dict(os.environ, LBVE_ORACLE_LIB=str(so), OMP_NUM_THREADS="2")
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           os.path.join(HERE, test_file)], env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.parametrize("name", sorted(BRUTE_FORCE_ONLY))
def test_only_the_brute_force_catches_mutant(name, tmp_path):
    so = _mutant_lib(tmp_path, *BRUTE_FORCE_ONLY[name])
    pins = _run_suite(so, "test_oracle_pins.py")
    assert pins.returncode == 0, f"mutant {name} is caught by the pins as well:\n{pins.stdout[-1500:]}"
    brute = _run_suite(so, "test_oracle_brute_force.py")
    assert brute.returncode != 0, f"mutant {name} survived the brute-force comparison:\n{brute.stdout[-2000:]}"


# Plausible mistakes in the two-dimensional oracle, each caught by its pin suite.
MUTANTS_2D = {
    "2d_forcing_first_order_unweighted": ("double A = 3.0 * (1.0 - 0.5 * s->omega_m)", "double A = 3.0 * (1.0 + 0.0 * s->omega_m)"),
    "2d_moving_wall_sign": ("s->f[(long)OPP2[i] * n + r] = fsi - 6.0 * W2[i] * s->rho[r] * cub;",
                           "s->f[(long)OPP2[i] * n + r] = fsi + 6.0 * W2[i] * s->rho[r] * cub;"),
    "2d_source_transposed_gradient": ("for (int k = 0; k < 2; ++k) b += tr[CMP[k][j]] * G[k * 2 + i];",
                                      "for (int k = 0; k < 2; ++k) b += tr[CMP[k][j]] * G[i * 2 + k];"),
    "2d_field_force_dropped": ("F[a] = (s->p.g[a] + s->Ff[(long)a * n + r]) + Fp[a];", "F[a] = s->p.g[a] + Fp[a];"),
    "2d_wall_gradient_uses_cell": ("double up = fluid2(s, np_) ? 0.5 * (ur + u[(long)j * n + np_]) : ubp[j];",
                                   "double up = fluid2(s, np_) ? 0.5 * (ur + u[(long)j * n + np_]) : ur;"),
    "2d_diagonal_weight": ("for (int i = 5; i < 9; ++i) W2[i] = 1.0 / 36.0;", "for (int i = 5; i < 9; ++i) W2[i] = 1.0 / 35.0;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS_2D))
def test_2d_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS_2D[name]
    src = open(os.path.join(ROOT, "oracle", "lbve2d_oracle.c")).read()
    assert src.count(old) == 1, f"mutation site for {name} not found or not unique"
    (tmp_path / "lbve2d_oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ROOT, "oracle", "lbve2d_oracle.h"), tmp_path / "lbve2d_oracle.h")
    so = tmp_path / "mutant2d.so"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                    str(tmp_path / "lbve2d_oracle.c"), "-o", str(so), "-lm"], check=True)
    env = dict(os.environ, LBVE_ORACLE2D_LIB=str(so), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(HERE, "test_oracle2d_pins.py")], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the 2-D pins:\n{r.stdout[-2000:]}"
