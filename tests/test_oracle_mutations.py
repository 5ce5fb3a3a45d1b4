"""The pins catch plausible mistakes: each case plants one mistake in a copy
of the oracle (on the CPU, in a temporary folder), runs the pin that should
see it against that copy, and expects it to fail.  The unchanged copy passes
the same pins (the first case), so a failure is the mistake's doing."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.join(ROOT, "tests")

SRC3, SRC2 = "cslbm_oracle.c", "cslbm_oracle2d.c"
CASES = [
    # (what, file, old, new, pin)
    ("the unchanged oracle", SRC3, None, None,
     "test_oracle_pins.py::test_equilibrium_moments_any_metric"),
    ("f^eq with delta for g^ij", SRC3,
     "a2[a][b] = rho * (theta * gi[a][b] - CS2 * (a == b)) + rho * u[a] * u[b];",
     "a2[a][b] = rho * (theta * (a == b) - CS2 * (a == b)) + rho * u[a] * u[b];",
     "test_oracle_pins.py::test_equilibrium_moments_any_metric"),
    ("b2 without -c_s^2 delta A", SRC3,
     "b2[a][b] = C[a][b] - CS2 * (a == b) * A;", "b2[a][b] = C[a][b];",
     "test_oracle_pins.py::test_forcing_recomposition_moments"),
    ("collision with the whole F(t-1)", SRC3,
     "fs[q] = fb[q] - om * (fb[q] - fe[q]) + F[q] - 0.5 * Fprev[q];",
     "fs[q] = fb[q] - om * (fb[q] - fe[q]) + F[q] - 1.0 * Fprev[q];",
     "test_oracle_step.py::test_flat_periodic_is_textbook_bgk"),
    ("Christoffel symbol with a flipped sign", SRC3,
     "s += gi[i][l] * (dg[j][k][l] + dg[k][j][l] - dg[l][j][k]);",
     "s += gi[i][l] * (dg[j][k][l] + dg[k][j][l] + dg[l][j][k]);",
     "test_oracle_pins.py::test_geometry_closed_forms"),
    ("transform with J J~^-1 for J~^-1 J", SRC3,
     "D[i][j] += Jni[i][k] * Jo[k][j];", "D[i][j] += Jo[i][k] * Jni[k][j];",
     "test_oracle_step.py::test_transform_equilibrium_to_equilibrium_and_round_trip"),
    ("B^i without Gamma^i_jk T^jk", SRC3,
     "b -= gam[k][jj][k] * T[i][jj] + gam[i][jj][k] * T[jj][k] + gam[jj][jj][k] * T[k][i];",
     "b -= gam[k][jj][k] * T[i][jj] + gam[jj][jj][k] * T[k][i];",
     "test_oracle_circular_couette.py::test_circular_couette_second_order"),
    ("outflow copy without sqrt(g) ratio", SRC3,
     "for (int l = 0; l < Q; l++) fout[l * N + v] = fin[l * N + vi] * sgi / sgw;",
     "for (int l = 0; l < Q; l++) fout[l * N + v] = fin[l * N + vi];",
     "test_oracle_boundary.py::test_boundary_fields_dynamic_channel"),
    ("wall stress with (1 - 1/tau)", SRC3,
     "T[a][b] += (fe[l] + (1.0 - 0.5 / p->tau) * (fl - fe[l])) * CV[l][a] * CV[l][b] * sg;\n        }\n"
     "        for (int a = 0; a < 3; a++)\n            for (int i = 0; i < 3; i++) acc[a]",
     "T[a][b] += (fe[l] + (1.0 - 1.0 / p->tau) * (fl - fe[l])) * CV[l][a] * CV[l][b] * sg;\n        }\n"
     "        for (int a = 0; a < 3; a++)\n            for (int i = 0; i < 3; i++) acc[a]",
     "test_oracle_boundary.py::test_flat_couette_wall_force_is_the_exact_stress"),
    ("nabla_k rho u^i without Gamma^i_kl rho u^l", SRC3,
     "for (int l = 0; l < 3; l++) s += gam[i][k][l] * j[l];",
     "for (int l = 0; l < 3; l++) s += 0.0 * gam[i][k][l] * j[l];",
     "test_oracle_pins.py::test_forcing_C_parallel_field_has_no_theta_part"),
    ("nabla_k rho u^i with Gamma^l_ki rho u^l", SRC3,
     "for (int l = 0; l < 3; l++) s += gam[i][k][l] * j[l];",
     "for (int l = 0; l < 3; l++) s += gam[l][k][i] * j[l];",
     "test_oracle_pins.py::test_forcing_C_parallel_field_has_no_theta_part"),
    ("literal-a2 transform subtracting c_s^2 rho delta twice", SRC3,
     "t2[i][j] = tM[i][j] - (p->literal_a2 ? 0.0 : CS2 * a0 * (i == j));",
     "t2[i][j] = tM[i][j] - CS2 * a0 * (i == j);",
     "test_oracle_step.py::test_transform_literal_mode_under_stretch_and_shear"),
    ("2-D outflow copy without sqrt(g) ratio", SRC2,
     "for (int l = 0; l < Q2; l++) fout[l * N + v] = fin[l * N + vi] * sgi / sgw;",
     "for (int l = 0; l < Q2; l++) fout[l * N + v] = fin[l * N + vi];",
     "test_oracle2d.py::test_boundary_fields_on_every_boundary_node"),
    ("2-D b2 without -c_s^2 delta A", SRC2,
     "b2[a][b] = C[a][b] - CS2_2 * (a == b) * A;", "b2[a][b] = C[a][b];",
     "test_oracle2d.py::test_forcing_recomposition_moments_2d"),
    ("2-D nabla_k rho u^i without Gamma^i_kl rho u^l", SRC2,
     "for (int l = 0; l < 2; l++) s += gam[i][k][l] * j[l];",
     "for (int l = 0; l < 2; l++) s += 0.0 * gam[i][k][l] * j[l];",
     "test_oracle2d.py::test_forcing_C_parallel_field_has_no_theta_part_2d"),
    ("2-D transform with J J~^-1 for J~^-1 J", SRC2,
     "D[i][j] = Jni[i][0] * Jo[0][j] + Jni[i][1] * Jo[1][j];",
     "D[i][j] = Jo[i][0] * Jni[0][j] + Jo[i][1] * Jni[1][j];",
     "test_oracle2d.py::test_chart_change_keeps_density_and_cartesian_velocity"),
]


@pytest.mark.parametrize("what,src,old,new,pin", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_its_pin(tmp_path, what, src, old, new, pin):
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle", ignore=shutil.ignore_patterns("_build"))
    if old is not None:
        p = tmp_path / "oracle" / src
        text = p.read_text()
        assert text.count(old) >= 1, what  # every occurrence (both transformations share a line)
        p.write_text(text.replace(old, new))
    # the pins run from the temporary folder, without the suite's conftest,
    # so that `import oracle` finds the copy
    for name in ("windows.py", pin.split("::")[0]):
        shutil.copy(os.path.join(HERE, name), tmp_path)
    shutil.copytree(os.path.join(HERE, "golden"), tmp_path / "golden")
    env = dict(os.environ, PYTHONPATH=f"{tmp_path}{os.pathsep}{ROOT}")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-x", pin],
                       cwd=tmp_path, env=env, capture_output=True, text=True, timeout=600)
    if old is None:
        assert r.returncode == 0, r.stdout[-2000:]
    else:
        assert r.returncode == 1 and "failed" in r.stdout, (what, r.stdout[-2000:])
