"""The oracle's pins are sharp: plausible mistakes planted in copies of the
oracle source (a dropped round, term, dagger or conjugate, a wrong sign, index,
factor or wrap) are each caught by at least one pin of test_oracle_pins.py.

Each mutant is one textual change to su3_oracle.c that must apply exactly once;
it is compiled with the oracle's own flags into a temporary library, the
oracle module is routed through it, and the pins run (cheapest first) until one
fails.  Nothing here touches the GPU or the CUDA library.
"""
import os
import shutil
import tempfile

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "su3_oracle.c")

# (name, text in su3_oracle.c, replacement)
MUTANTS = [
    ("philox: nine rounds", "for (round = 0; round < 10; round++)", "for (round = 0; round < 9; round++)"),
    ("philox: wrong Weyl constant", "k1 += PHILOX_WEYL_B;", "k1 += PHILOX_WEYL_A;"),
    ("uniform: bin edge instead of centre",
     "return ((double)x + 0.5) * 2.220446049250313080847263336181640625e-16;",
     "return ((double)x + 0.0) * 2.220446049250313080847263336181640625e-16;"),
    ("third row: one conjugate dropped", "u->e[2][1] = c_conj(b);", "u->e[2][1] = b;"),
    ("Gram-Schmidt: row 1 not normalised", "n1 = 1.0 / sqrt(n1);", "n1 = 1.0;"),
    ("geometry: backward neighbour wraps forward", "y[nu] = (x[nu] + L[nu] - 1) % L[nu];",
     "y[nu] = (x[nu] + L[nu] + 1) % L[nu];"),
    ("staple: dagger of U_nu(x) dropped", "        t1 = m_dag(&c);\n        t3 = m_mul(&t2, &t1);",
     "        t1 = c;\n        t3 = m_mul(&t2, &t1);"),
    ("staple: backward path at the wrong site", "c = load_link(U, s_mnu, nu, f32);", "c = load_link(U, s, nu, f32);"),
    ("staple: backward path dropped", "        t1 = m_mul(&t3, &c);\n        m_acc(&A, &t1);",
     "        t1 = m_mul(&t3, &c);\n        (void)t1;"),
    ("heatbath: alpha = beta k / 3", "if (kp_one_hit(2.0 * beta * k / 3.0, uu, a))", "if (kp_one_hit(beta * k / 3.0, uu, a))"),
    ("KP: accept test without the 1/2", "if (u[3] * u[3] > 1.0 - 0.5 * delta) return 0;",
     "if (u[3] * u[3] > 1.0 - delta) return 0;"),
    ("KP: cos instead of cos^2", "double delta = -(log(u[0]) + c * c * log(u[2])) / alpha;",
     "double delta = -(log(u[0]) + c * log(u[2])) / alpha;"),
    ("SU(2) embedding: sign of a2 in the lower row", "m[1][0].re = -a[2];", "m[1][0].re = a[2];"),
    ("SU(2) update: R = Y V instead of Y V^+", "vd[p][q] = c_conj(v[q][p]);", "vd[p][q] = v[p][q];"),
    ("SU(2) projection: sign of r2", "r[2] = 0.5 * (W.e[i][j].re - W.e[j][i].re);",
     "r[2] = 0.5 * (W.e[i][j].re + W.e[j][i].re);"),
    ("plaquette: dagger of U_nu(x) dropped", "mat3 cd = m_dag(&c), dd = m_dag(&d);", "mat3 cd = m_dag(&c), dd = d;"),
    ("plaquette: normalised by 4V", "return sum / (6.0 * (double)g.V);", "return sum / (4.0 * (double)g.V);"),
    ("hot start: Box-Muller with two cosines", "gz[2 * call + 1] = rad * sin(2.0 * ORACLE_PI * ub);",
     "gz[2 * call + 1] = rad * cos(2.0 * ORACLE_PI * ub);"),
]

# the pins, cheapest first
PINS = [
    ("philox KAT", pins.test_philox_known_answers),
    ("uniform maps", pins.test_uniform_map_extremes_and_bins),
    ("cold start", pins.test_cold_start_is_identity_and_plaquette_one),
    ("abelian closed form", pins.test_plaquette_closed_form_abelian_field),
    ("Haar moments", pins.test_hot_start_is_haar_su3),
    ("gauge invariance", pins.test_plaquette_gauge_invariant),
    ("staple = action derivative", lambda: [pins.test_staple_is_action_derivative(mu) for mu in range(4)]),
    ("staple translation", pins.test_staple_translation_covariant),
    ("unitarity", pins.test_updates_stay_in_su3),
    ("KP chi-square", lambda: [pins.test_kp_a0_distribution_chisquare(a) for a in (2.0, 8.0)]),
    ("weak coupling", lambda: pins.test_weak_coupling_plaquette(50.0)),
    ("strong coupling", lambda: pins.test_strong_coupling_plaquette(0.2)),
    ("single-link equilibrium", lambda: pins.test_single_link_heatbath_equilibrium(False)),
]


@pytest.fixture(scope="module")
def workdir():
    d = tempfile.mkdtemp(prefix="oracle_mutants_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


def test_pins_pass_on_the_oracle():
    for _, pin in PINS:
        pin()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(workdir, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not found exactly once: %r" % old
    tag = "m%02d" % MUTANTS.index((name, old, new))
    path = os.path.join(workdir, tag + ".c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = oracle.compile_source(path, os.path.join(workdir, tag + ".so"))
    caught = None
    with oracle.use_library(lib):
        for pin_name, pin in PINS:
            try:
                pin()
            except (AssertionError, ValueError, RuntimeError, FloatingPointError):
                caught = pin_name
                break
    assert caught, "no pin caught the mutant %r" % name
