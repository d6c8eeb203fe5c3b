"""The pins must catch plausible mistakes in the oracle: each mutant below is a copy of
oracle/snap_oracle.c with one planted error (a dropped term, a wrong sign, index or
coefficient, a transposed operand); the CPU pin suite run against it must fail."""
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "snap_oracle.c")
PINS = ["tests/test_oracle_weno.py", "tests/test_oracle_lmars.py", "tests/test_oracle_thermo.py",
        "tests/test_oracle_satadj.py", "tests/test_oracle_scheme.py",
        "tests/test_oracle_adjoint.py", "tests/test_oracle_kessler.py",
        "tests/test_oracle_forcing.py", "tests/test_oracle_theta_e.py",
        "tests/test_oracle_bottom.py"]

MUTANTS = {
    "weno beta0 curvature coefficient": ("b[0] = 13.0 / 12.0 * t * t;", "b[0] = 13.0 / 6.0 * t * t;"),
    "weno linear weights reversed": ("static const double d[3] = {0.1, 0.6, 0.3};\n  double b[3], a[3], s = 0.0;",
                                     "static const double d[3] = {0.3, 0.6, 0.1};\n  double b[3], a[3], s = 0.0;"),
    "weno candidate sign": ("double v2 = q[2] / 3.0 + 5.0 / 6.0 * q[3] - q[4] / 6.0;",
                            "double v2 = q[2] / 3.0 + 5.0 / 6.0 * q[3] + q[4] / 6.0;"),
    "lmars pressure damping sign": ("- 0.5 * rhoc * (uR - uL); /* Eq. rp */", "+ 0.5 * rhoc * (uR - uL); /* Eq. rp */"),
    "lmars velocity correction sign": ("(XR[nv - 1] - XL[nv - 1]) / (2.0 * rhoc); /* Eq. ru */",
                                       "(XL[nv - 1] - XR[nv - 1]) / (2.0 * rhoc); /* Eq. ru */"),
    "lmars upwind side swapped": ("const double *XS = us > 0.0 ? XL : XR;", "const double *XS = us > 0.0 ? XR : XL;"),
    "energy flux without pressure": ("F[nv - 1] = us * (rhoe + pS);", "F[nv - 1] = us * rhoe;"),
    "mixing denominator sign": ("      d -= qij;", "      d += qij;"),
    "gravity source sign": ("dYdt[(long)mw * ncell + c] -= (rho - g->rho_bar[k]) * g->grav;",
                            "dYdt[(long)mw * ncell + c] += (rho - g->rho_bar[k]) * g->grav;"),
    "energy gravity source dropped": ("dYdt[(long)(nv - 1) * ncell + c] -= g->grav * 0.5 * (fb + ft);", "(void)fb; (void)ft;"),
    "divergence operands transposed": ("dYdt[v * ncell + c] -= (F[v * nf + f1] - F[v * nf + f0]) / h;",
                                       "dYdt[v * ncell + c] -= (F[v * nf + f0] - F[v * nf + f1]) / h;"),
    "rk3 second stage weights": ("Yout[c] = 0.75 * Yn[c] + 0.25 * ys;", "Yout[c] = 0.25 * Yn[c] + 0.75 * ys;"),
    "clausius-clapeyron log term sign": ("exp(beta * (1.0 - 1.0 / t) - delta * log(t))", "exp(beta * (1.0 - 1.0 / t) + delta * log(t))"),
    "adjustment transfer direction": ("      } else {\n        drho = dq * g->eps[i] * N;\n      }",
                                      "      } else {\n        drho = -dq * g->eps[i] * N;\n      }"),
    "condensate chemical potential sign": ("return -(g->Lref[i][j] + dc_of(g, i, j) * g->Tref[i]);",
                                           "return (g->Lref[i][j] + dc_of(g, i, j) * g->Tref[i]);"),
    "viscous momentum flux sign": ("Ff[im0 + m] -= rf * g->nu * grad;", "Ff[im0 + m] += rf * g->nu * grad;"),
    "cfl without sound speed": ("r += (fabs(Xc[mom_slot(g, d)]) + cs) / h;", "r += (fabs(Xc[mom_slot(g, d)]) + 0.0 * cs) / h;"),
    "periodic wrap off by one": ("if (bc_hi == ORC_PERIODIC) return idx % n;", "if (bc_hi == ORC_PERIODIC) return (idx + 1) % n;"),
    "adjoint of u* pressure term sign": ("XLb[nv - 1] += usb / (2.0 * rhoc);", "XLb[nv - 1] -= usb / (2.0 * rhoc);"),
    "adjoint energy gravity dropped": ("Fbz[((long)(k + 1) * ny + j) * nx + i] += -0.5 * g->grav * me;", "(void)me;"),
    "adjustment adjoint latent term dropped": ("dFdT += drs * (T * (c_v - c_c) - mu_c);",
                                               "dFdT += drs * (T * (c_v - c_c));"),
    "adjustment adjoint unsaturated routing": ("lam_in[vi] = lam_in[ci] = lam_out[vi];",
                                               "lam_in[vi] = lam_in[ci] = lam_out[ci];"),
    "moist lmars adjoint gamma sign": ("denLb += gLb * gm1 / numL;", "denLb -= gLb * gm1 / numL;"),
    "moist primitive adjoint chemical potential": ("Yb[icond(g, i, j)] += -Ub * mu_of(g, i, j);",
                                                   "Yb[icond(g, i, j)] += Ub * mu_of(g, i, j);"),
    "tracer flux adjoint without dry-air term": ("XSb[t] += wgt * (Fbar[t] - Fbar[0]) * mf;",
                                                 "XSb[t] += wgt * Fbar[t] * mf;"),
    "kessler autoconversion sign": ("phi[1] = k1 * sup - k3 * x[1] * x[2] - k2 * x[1];",
                                    "phi[1] = k1 * sup - k3 * x[1] * x[2] + k2 * x[1];"),
    "kessler evaporation without rain factor": ("    phi[0] = -k4 * x[2] * sup;", "    phi[0] = -k4 * sup;"),
    "sedimentation from the wrong side": ("const double *XS = wt < 0.0 ? XR : XL;",
                                          "const double *XS = wt < 0.0 ? XL : XR;"),
    "theta_e latent heat at the reference temperature": ("const double L = g->Lref[0][0] - dc * (T - g->Tref[0]);",
                                                          "const double L = g->Lref[0][0];"),
    "theta_e exponent without the cloud heat capacity": ("const double cc = cpd * qd + cl * qt;",
                                                         "const double cc = cpd * qd + cl * qv;"),
    "cooling without condensate heat capacity": ("              Cv += g->sig_c[a][b] * c_vd(g) * Y[(long)icond(g, a, b) * ncell + c];",
                                                 "              (void)b;"),
    "sponge time linear in pressure": ("const double r = pk / g->sponge_p0, tau = g->sponge_tau0 * r * r;",
                                       "const double r = pk / g->sponge_p0, tau = g->sponge_tau0 * r;"),
    "no-slip ghost negates the normal velocity only": (
        "  if (bc == ORC_NOSLIP) {\n    for (int m = 0; m < nmom_of(g); ++m)",
        "  if (bc == -1) {\n    for (int m = 0; m < nmom_of(g); ++m)"),
    "bottom ghost density scaled the wrong way": ("X[dst] *= T / g->T_bottom;", "X[dst] *= g->T_bottom / T;"),
    "bottom ghost keeps the mirrored temperature": ("Tx[dst] = g->T_bottom / Px[src];", "Tx[dst] = Tx[src];"),
    "sedimentation through the no-slip floor": (
        "if ((k == 0 && g->bc[4] != ORC_PERIODIC) || (k == g->nz && g->bc[5] != ORC_PERIODIC)) return;",
        "if ((k == 0 && g->bc[4] == ORC_REFLECT) || (k == g->nz && g->bc[5] == ORC_REFLECT)) return;"),
    "sedimentation energy without kinetic part": ("F[nv - 1] += ms * (g->sig_c[i][j] * c_vd(g) * T + 0.5 * u2 + mu_of(g, i, j));",
                                                  "F[nv - 1] += ms * (g->sig_c[i][j] * c_vd(g) * T + mu_of(g, i, j));"),
}


def build_mutant(name, tmp):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site of '{name}' not unique or missing"
    path = os.path.join(tmp, "snap_oracle.c")
    open(path, "w").write(src.replace(old, new))
    shutil.copy(os.path.join(ROOT, "oracle", "snap_oracle.h"), tmp)
    lib = os.path.join(tmp, "libmutant.so")
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", lib, path, "-lm"])
    return lib


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_planted_mistake(name):
    with tempfile.TemporaryDirectory() as tmp:
        lib = build_mutant(name, tmp)
        env = dict(os.environ, SNAP_ORACLE_LIB=lib)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            "-m", "not gpu"] + PINS, cwd=ROOT, env=env, capture_output=True,
                           text=True, timeout=600)
        assert r.returncode != 0, f"no pin caught the mutant '{name}':\n{r.stdout[-2000:]}"
