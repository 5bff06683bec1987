"""Plant plausible mistakes in a copy of the oracle and check the pins catch each.

Every mutation below edits one expression of ``oracle/glbm_oracle.c`` (a sign,
a dropped term, a wrong index or factor), compiles the copy, and runs the oracle
pin tests against it in a subprocess; the run must fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "glbm_oracle.c")

MUTATIONS = {
    "P+ sign of c*u": ("*Pp = (cs2 + c * u + u * u / N)", "*Pp = (cs2 - c * u + u * u / N)"),
    "dropped u^2/N": ("*Pm = (cs2 - c * u + u * u / N)", "*Pm = (cs2 - c * u)"),
    "factorial index": ("orc_factorial(n + m) * orc_factorial(m)",
                        "orc_factorial(n) * orc_factorial(m)"),
    "mirror not swapped": ("        Pp = Pm;\n        Pm = t;\n", "        (void)t;\n"),
    "omega without 1/2": ("double omega = 1.0 / (c->tau + 0.5);", "double omega = 1.0 / c->tau;"),
    "force sign": ("if (!c->guo) return W * vx * Gx;", "if (!c->guo) return -W * vx * Gx;"),
    "force theta": ("const double Gx = c->g / thx;", "const double Gx = c->g;"),
    "stream x sign": ("int xd = orc_wrap(x + nx, Lx);", "int xd = orc_wrap(x - nx, Lx);"),
    "wall speeds swapped": ("orc_axis_eq(&ax, c->uw_lo, Elo);", "orc_axis_eq(&ax, c->uw_hi, Elo);"),
    "emission rows": ("for (int k = 0; k < (ny > 0 ? ny : -ny); ++k) {",
                      "for (int k = 0; k < (ny > 0 ? ny : -ny) - 1; ++k) {"),
    "bounce-back offset": ("F[(-n + N) * L + (-1 - xd)] = v;", "F[(-n + N) * L + (-xd)] = v;"),
    "temperature dims": ("out[3 * plane + node] = e2 / (2.0 * rho);",
                         "out[3 * plane + node] = e2 / rho;"),
    "tangent of omega": ("if (d == 1) v += domega * (feq - f);", "if (d == 1) v += omega * (feq - f);"),
    "tangent of P0": ("const double dP0 = -dPp - dPm;", "const double dP0 = dPp + dPm;"),
    "2N+2 at full speed": ("orc_eq_lattice(N, 0.5 * u, En);", "orc_eq_lattice(N, u, En);"),
    "2N+2 one neighbour": ("const int lo = (a->v[j] - 1) / 2, hi = (a->v[j] + 1) / 2;",
                           "const int lo = (a->v[j] - 1) / 2, hi = lo;"),
    "2N+2 theta without c^2/4": ("return a->zv ? (4.0 * a->N + 3.0) / 3.0 : a->N / 3.0;",
                             "return a->N / (a->zv ? 0.75 : 3.0);"),
    "2N+2 even velocities": ("a->v[j] = zv ? 2 * j - (2 * N + 1) : j - N;",
                             "a->v[j] = zv ? 2 * j - 2 * N : j - N;"),
    "3D z stream sign": ("zd = orc_wrap(z + nz, Lz);", "zd = orc_wrap(z - nz, Lz);"),
    "3D emission without W^z": ("rlo * Elo[ix] * Wy[iy] * Wz[iz];", "rlo * Elo[ix] * Wy[iy];"),
    "heat flux without 1/2": ("out[4 * plane + node] = 0.5 * qx;", "out[4 * plane + node] = qx;"),
    "shear stress about zero": ("                sxy += dx * dy * f;\n            }\n        }\n        out[0 * plane",
                                "                sxy += ax.v[ix] * ay.v[iy] * f;\n            }\n        }\n        out[0 * plane"),
    "wall denominator without |ny|": ("if (ay.v[iy] > 0) den += ay.v[iy] * Elo[ix] * Wy[iy];",
                                      "if (ay.v[iy] > 0) den += Elo[ix] * Wy[iy];"),
    "Kn with theta for 2 theta": ("    double theta = N / 3.0;\n    return kn * H / sqrt(2.0 * theta);",
                                  "    double theta = N / 3.0;\n    return kn * H / sqrt(theta);"),
    "3D heat flux without 1/2": ("e2 / (3.0 * rho), 0.5 * qx, 0.5 * qy", "e2 / (3.0 * rho), qx, 0.5 * qy"),
    "1D heat flux without 1/2": ("out[3 * L + x] = 0.5 * e3;", "out[3 * L + x] = e3;"),
    "3D force sign": ("Wx[ix] * Wy[iy] * Wz[iz], ix - NX, iy - NY", "Wx[ix] * Wy[iy] * Wz[iz], NX - ix, iy - NY"),
    "3D force theta": ("        const double theta_x = NX / 3.0;\n", "        const double theta_x = NX;\n"),
    "tangent of g without theta": ("const double wxg = Wx[nx + NX] * Wy[ny + NY] * nx / theta_x;",
                                   "const double wxg = Wx[nx + NX] * Wy[ny + NY] * nx;"),
    "stream y sign": ("                    int yd = y + ny;", "                    int yd = y - ny;"),
    "3D stream y sign": ("const int yd = y + ny;", "const int yd = y - ny;"),
    "tangent of rho dropped": ("const double dfeq = rho[d] * Ex[nx + NX] * Ey[ny + NY] +\n                                        rho[0] *",
                               "const double dfeq = 0.0 * rho[d] * Ex[nx + NX] * Ey[ny + NY] +\n                                        rho[0] *"),
    "tangent of u without rho term": ("dux[d] = (jx[d] - ux * rho[d]) / rho[0];", "dux[d] = jx[d] / rho[0];"),
    "tangents not streamed": ("for (int d = 0; d < ORC_NT; ++d) orc_stream2d(c, X + d * n, F + d * n);",
                              "for (int d = 0; d < 1; ++d) orc_stream2d(c, X + d * n, F + d * n);"),
    "force theta of the y axis": ("double theta_x = orc_axis_theta(&ax), theta_y", "double theta_x = orc_axis_theta(&ay), theta_y"),
    "collision x axis with the y flag": ("    orc_axis_make(c->NX, ORC_ZVX(c), &ax);\n    orc_axis_make(c->NY, ORC_ZVY(c), &ay);\n    int Lx = c->Lx, Ly = c->Ly;\n    size_t plane = (size_t)Lx * Ly;\n    double Wx[",
                                         "    orc_axis_make(c->NX, ORC_ZVY(c), &ax);\n    orc_axis_make(c->NY, ORC_ZVY(c), &ay);\n    int Lx = c->Lx, Ly = c->Ly;\n    size_t plane = (size_t)Lx * Ly;\n    double Wx["),
    "m sum one term short": ("for (int m = 0; m <= (N - n) / 2; ++m) {", "for (int m = 0; m < (N - n) / 2; ++m) {"),
    "P0 power": ("pow(P0, N - n - 2 * m);", "pow(P0, N - n - m);"),
    "P0 closure sign": ("*P0 = 1.0 - *Pp - *Pm;", "*P0 = 1.0 - *Pp + *Pm;"),
    "Guo without (1 - omega/2)": ("return (1.0 - 0.5 * omega) * W * ((vx - ux) * Gx + xiU * vx * Gx);",
                                  "return W * ((vx - ux) * Gx + xiU * vx * Gx);"),
    "Guo without the half-force shift": ("return (c->guo ? jx + 0.5 * c->g : jx) / rho;",
                                         "return jx / rho;"),
    "Guo shift of a whole g": ("return (c->guo ? jx + 0.5 * c->g : jx) / rho;",
                               "return (c->guo ? jx + c->g : jx) / rho;"),
    "Guo without the -u term": ("((vx - ux) * Gx + xiU * vx * Gx)", "(vx * Gx + xiU * vx * Gx)"),
    "Guo xi.U without y": ("const double xiU = vx * ux / thx + vy * uy / thy + vz * uz / thz;",
                           "const double xiU = vx * ux / thx + vz * uz / thz;"),
    "Guo xi.U with theta_x on y": ("const double xiU = vx * ux / thx + vy * uy / thy + vz * uz / thz;",
                                   "const double xiU = vx * ux / thx + vy * uy / thx + vz * uz / thz;"),
    "Guo moments without the shift": ("        double ux = orc_ux(c, jx, rho), uy = jy / rho;\n        double e2",
                                      "        double ux = jx / rho, uy = jy / rho;\n        double e2"),
    "wall-speed tangent without rho_w": ("dF[q * plane + (size_t)y * Lx + x] += rw * dE[nx + NX] * Wy[ny + NY];",
                                         "dF[q * plane + (size_t)y * Lx + x] += dE[nx + NX] * Wy[ny + NY];"),
    "wall-speed tangent with E for dE/du": ("dF[q * plane + (size_t)y * Lx + x] += rw * dE[nx + NX] * Wy[ny + NY];",
                                           "dF[q * plane + (size_t)y * Lx + x] += rw * E[nx + NX] * Wy[ny + NY];"),
    "wall-speed tangent into the far rows": ("const int y = upper ? Ly - 1 - k : k;",
                                             "const int y = upper ? k : Ly - 1 - k;"),
    "3D x and z swapped in q": ("const double f = F[((iz * Qy + iy) * Qx + ix) * plane + node];\n                        rho += f;",
                                "const double f = F[((ix * Qy + iy) * Qx + iz) * plane + node];\n                        rho += f;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor missing: {old!r}"
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new, 1))
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(lib), str(mutated), "-lm"])
    env = dict(os.environ, GLBM_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q",
                        os.path.join(ROOT, "tests", "test_oracle_equilibrium.py"),
                        os.path.join(ROOT, "tests", "test_oracle_dynamics.py"),
                        os.path.join(ROOT, "tests", "test_oracle_gradient.py"),
                        os.path.join(ROOT, "tests", "test_oracle_aniso.py"),
                        os.path.join(ROOT, "tests", "test_oracle_zv.py"),
                        os.path.join(ROOT, "tests", "test_oracle_3d.py"),
                        os.path.join(ROOT, "tests", "test_oracle_guo.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutation {name!r}"
