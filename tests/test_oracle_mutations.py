"""The pins catch plausible mistakes: each mutation below is planted in a copy of
the oracle sources (CPU only), the copy is built, and at least one pin must fail.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (file, original text, mutated text, pin tests that must catch it)
MUTATIONS = [
    ("orc_contact.cpp", "double la = ra - 0.5 * delta, lb = rb - 0.5 * delta;",
     "double la = ra, lb = rb;", "test_p4"),
    ("orc_contact.cpp", "V3 Fn = sub(scl(-fel, n), scl(cn, vn));",
     "V3 Fn = add(scl(-fel, n), scl(cn, vn));", "test_p2"),
    ("orc_contact.cpp", "cn = -2.0 * mat.beta * std::sqrt(Sn * ms);",
     "cn = -2.0 * std::sqrt(5.0 / 6.0) * mat.beta * std::sqrt(Sn * ms);", "test_linear_spring"),
    ("orc_contact.cpp", "fel = p.kn_linear * delta;", "fel = p.kn_linear * delta * std::sqrt(delta / 1e-6);",
     "test_linear_spring"),
    ("orc_contact.cpp", "double kn = (4.0 / 3.0) * mat.Es * std::sqrt(Rs);",
     "double kn = (4.0 / 3.0) * mat.Es * Rs;", "test_p1"),
    ("orc_contact.cpp", "out.Ta = cross(scl(la, n), Ft);", "out.Ta = cross(Ft, scl(la, n));", "test_p4"),
    ("orc_contact.cpp", "out.Ta = cross(scl(l, n), Ft);", "out.Ta = cross(Ft, scl(l, n));", "test_p13"),
    ("orc_contact.cpp", "  if (ft > p.friction * fn) {", "  if (false) {", "test_p13"),
    ("orc_contact.cpp", "out.F = scl(-6.0 * M_PI * mu * r * r * vn / hh, n);",
     "out.F = scl(-6.0 * M_PI * mu * r * vn / hh, n);", "test_p10"),
    ("orc_contact.cpp", "double shape = (2.0 + beta + 2.0 * beta * beta) / ((1.0 + beta) * (1.0 + beta));",
     "double shape = (2.0 + beta + beta * beta) / ((1.0 + beta) * (1.0 + beta));", "test_p17"),
    ("orc_contact.cpp", "double la = ra + 0.5 * h, lb = rb + 0.5 * h;", "double la = ra, lb = rb;",
     "test_p17"),
    ("orc_contact.cpp", "double lg = std::log(dbar / (2.0 * hh));", "double lg = std::log(dbar / hh);",
     "test_p17"),
    ("orc_contact.cpp", "V3 Fs = scl(-6.0 * M_PI * mu * r * (8.0 / 15.0) * lg, vt);",
     "V3 Fs = scl(-6.0 * M_PI * mu * r * (4.0 / 15.0) * lg, vt);", "test_p17"),
    ("orc_step.cpp", "out.tq[j] = orc::add(out.tq[j], l.Tb);", "", "test_p4"),
    ("orc_fluid.cpp", "d * d / std::sqrt(om), cross(w, omega));", "d * d / std::sqrt(om), cross(omega, w));",
     "test_p16"),
    ("orc_fluid.cpp", "d * d / std::sqrt(om), cross(w, omega));", "d * d / om, cross(w, omega));",
     "test_p16"),
    ("orc_fluid.cpp", "f = add(f, lift_force(p, sub(U, u), om, d));",
     "f = add(f, lift_force(p, sub(u, U), om, d));", "test_p16"),
    ("orc_average.cpp", "if (k > 0) op.czm[k] = scale * dtau * D[2] / (zg.hz[k] * (zg.zc[k] - zg.zc[k - 1]));",
     "if (k > 0) op.czm[k] = scale * dtau * D[2] / (zg.hz[k - 1] * (zg.zc[k] - zg.zc[k - 1]));", "test_p18"),
    ("orc_average.cpp", "double dz = zg.graded ? zg.hz[kz] : (p.hi[2] - p.lo[2]) / p.ncell[2];",
     "double dz = zg.graded ? zg.hz[0] : (p.hi[2] - p.lo[2]) / p.ncell[2];", "test_p18"),
    ("orc_fluid.cpp", "ax.f = (x - g.zc[k]) / (g.zc[k + 1] - g.zc[k]);",
     "ax.f = (x - g.zc[k]) / (g.zf[k + 1] - g.zf[k]);", "test_p18"),
    ("orc_fluid.cpp", "if (a == 2 && zg.graded) den = zg.zc[ip[2]] - zg.zc[im[2]];", "", "test_p18"),
    ("orc_fluid.cpp", "std::expm1((double)k * lr) / std::expm1((double)n * lr)", "(double)k / (double)n",
     "test_p18"),
    ("orc_fluid.cpp", "out[3 * c + 1] = g[2][0] - g[0][2];", "out[3 * c + 1] = g[0][2] - g[2][0];",
     "test_p15"),
    ("orc_fluid.cpp", "ip[a] = 1;\n            den = h;", "ip[a] = 1;\n            den = 2.0 * h;",
     "test_p15"),
    ("orc_fluid.cpp", "double c = 0.63 + 4.8 * std::sqrt(Vr / Re);\n  double Cd = c * c;",
     "double c = 0.63 + 0.48 * std::sqrt(Vr / Re);\n  double Cd = c * c;", "test_p3"),
    ("orc_fluid.cpp", "f = add(f, scl(p.c_add * p.rho_f * Vp, sub(Du, a_prev)));",
     "f = add(f, scl(p.c_add * p.rho_f * Vp, sub(a_prev, Du)));", "added_mass_initial"),
    ("orc_fluid.cpp", "double s = (x - p.lo[a]) * inv - 0.5;", "double s = (x - p.lo[a]) * inv;",
     "test_trilinear"),
    ("orc_average.cpp", "if (!p.periodic[a]) continue; /* no flux through this face */",
     "if (!p.periodic[a]) { lap += coef[a] * (0.0 - x[c]); continue; }", "test_p6"),
    ("orc_average.cpp", "double D = 0.25 * p.bandwidth[a] * p.bandwidth[a];",
     "double D = 0.5 * p.bandwidth[a] * p.bandwidth[a];", "test_p7"),
    ("orc_average.cpp", "*q = (int64_t)std::llrint(s);", "*q = (int64_t)s;", "test_p8"),
    ("orc_neighbors.cpp", "  return d2 < rc * rc;", "  return d2 <= rc * rc * 0.999;", "test_p5"),
    ("orc_fluid.cpp", "double A1 = std::pow(eps_f, 4.14);", "double A1 = std::pow(eps_f, 4.41);",
     "test_p9b"),
    ("orc_fluid.cpp", "0.8 * std::pow(eps_f, 1.28)", "0.8 * std::pow(eps_f, 1.82)", "test_p9b"),
    ("orc_fluid.cpp", ": std::pow(eps_f, 2.65);", ": std::pow(eps_f, 2.56);", "test_p9b"),
    ("orc_contact.cpp", "V3 xi = sub(xi_old, scl(dot(xi_old, n), n));", "V3 xi = xi_old;", "test_p19"),
    ("orc_contact.cpp", "if (new_len > 0.0) xi = scl(old_len / new_len, xi);", "", "test_p19"),
    ("orc_step.cpp", "h->x[i] = xn;", "h->x[i] = orc::add(h->x[i], orc::scl(p.dt, orc::sub(h->v[i], orc::scl(p.dt, a))));",
     "test_p1"),
]


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    return tmp_path_factory.mktemp("mut")


@pytest.mark.parametrize("k", range(len(MUTATIONS)))
def test_pin_catches_mutation(workdir, k):
    fname, orig, mut, pin = MUTATIONS[k]
    d = workdir / f"m{k}"
    pkg = d / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), pkg,
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    src = (pkg / fname).read_text()
    assert src.count(orig) == 1, f"mutation anchor not found: {orig!r}"
    (pkg / fname).write_text(src.replace(orig, mut))
    tests = d / "tests"
    shutil.copytree(os.path.join(ROOT, "tests"), tests,
                    ignore=shutil.ignore_patterns("__pycache__", "test_gpu*", "test_zz*",
                                                  "test_abi.py", "test_oracle_mutations.py"))
    env = dict(os.environ, PYTHONPATH=f"{d}:{ROOT}")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "-k", pin, str(tests)], cwd=d, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 1, f"pin {pin} did not catch mutation {k}:\n{r.stdout[-2000:]}"
