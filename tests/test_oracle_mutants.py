"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a sign, a
transposed operand, a dropped term, a wrong weight, moment group or boundary
rule), builds that copy in a temporary directory, and runs the CPU pin suites
(tests/test_oracle_pins.py, tests/test_oracle_dirichlet.py) against it in a
child process.  The case passes only if some pin fails.  Nothing here touches
the real oracle build or any GPU.
"""

import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_C = os.path.join(ROOT, "oracle", "ms_mrt_oracle.c")
PIN_FILES = [os.path.join(ROOT, "tests", "test_oracle_pins.py"),
             os.path.join(ROOT, "tests", "test_oracle_dirichlet.py")]

# (name, text in the oracle, replacement): one plausible mistake each
MUTANTS = [
    # Eq. 2-10: the off-diagonal entry of B with its two terms swapped
    ("B_offdiag_sign",
     "B[i * S + j] = xi[i] * (1.0 / D[i * n + (n - 1)] - 1.0 / D[i * n + j]);",
     "B[i * S + j] = xi[i] * (1.0 / D[i * n + j] - 1.0 / D[i * n + (n - 1)]);"),
    # Eq. 2-10: the diagonal entry without its own xi_i / D_in term
    ("B_diag_dropped_term",
     "double b = xi[i] / D[i * n + (n - 1)];",
     "double b = 0.0;"),
    # Eq. 2-10: B transposed
    ("B_transposed",
     "B[i * S + j] = xi[i] * (1.0 / D[i * n + (n - 1)]",
     "B[j * S + i] = xi[i] * (1.0 / D[i * n + (n - 1)]"),
    # Eq. 2-3b: closure that forgets the first species
    ("closure_drops_species",
     "xi[S] = 1.0 - sum;",
     "xi[S] = 1.0 - sum + xi[0];"),
    # Eq. 3-26 with c_s^2 = 1/3 on every lattice (wrong for D3Q7 and D2Q4)
    ("cs2_one_third_everywhere",
     "for (int k = 0; k < Q; ++k) L->cs2 += L->w[k] * L->c[k][0] * L->c[k][0];",
     "L->cs2 = 1.0 / 3.0;"),
    # Eq. 3-26: Lambda_1 = (D~/c_s^2 - I/2)^{-1}
    ("lambda1_half_sign",
     "(i == j ? 0.5 : 0.0);",
     "(i == j ? -0.5 : 0.0);"),
    # Eq. 3-26 with D~ transposed
    ("lambda1_Dtilde_transposed",
     "A[i * S + j] = Dt[i * S + j] / cs2",
     "A[i * S + j] = Dt[j * S + i] / cs2"),
    # Eq. 3-16 with the pole at -8
    ("lambda2_rule_pole",
     "8.0 * (l1 - 2.0) / (l1 - 8.0)",
     "8.0 * (l1 - 2.0) / (l1 + 8.0)"),
    # Eq. 3-16 applied to the off-diagonal entries too
    ("lambda2_rule_offdiagonal",
     "if (relax == ORC_SRT || i != j)",
     "if (relax == ORC_SRT)"),
    # Eq. 3-3: every equilibrium population with the rest weight
    ("feq_rest_weight",
     "acq += L->M[a][k] * (L->w[k] * xi[s]);",
     "acq += L->M[a][k] * (L->w[0] * xi[s]);"),
    # Eq. 3-3: every species' equilibrium from the first species
    ("feq_wrong_species",
     "acq += L->M[a][k] * (L->w[k] * xi[s]);",
     "acq += L->M[a][k] * (L->w[k] * xi[0]);"),
    # Sec. 3.1: odd moments relaxed by Lambda_2
    ("odd_moments_by_lambda2",
     "                    lam = L1[i * S + j];\n",
     "                    lam = L2[i * S + j];\n"),
    # Eq. 3-13a with Lambda_1 transposed
    ("odd_moments_lambda1_transposed",
     "                    lam = L1[i * S + j];\n",
     "                    lam = L1[j * S + i];\n"),
    # Eq. 3-13b: the population streamed against its velocity
    ("stream_direction",
     "dst[a] = pos[a] + L.c[k][a];",
     "dst[a] = pos[a] - L.c[k][a];"),
    # periodic wrap that clamps at the low face instead of wrapping
    ("periodic_low_face_clamped",
     "dst[a] += (face & 1) ? -dims[a] : dims[a];",
     "dst[a] += (face & 1) ? -dims[a] : 1;"),
    # Sec. 4 bounce-back into the same direction instead of the opposite one
    ("bounce_back_target",
     "g[c * per + s * Q + L.opp[k]] = fp[s * Q + k];",
     "g[c * per + s * Q + k] = fp[s * Q + k];"),
    # Sec. 4 anti-bounce-back without the factor 2
    ("anti_bounce_back_factor",
     "-fp[s * Q + k] + 2.0 * L.w[k] * xb[wall * n + s];",
     "-fp[s * Q + k] + L.w[k] * xb[wall * n + s];"),
    # Sec. 4 anti-bounce-back with the wrong sign of the reflected population
    ("anti_bounce_back_sign",
     "-fp[s * Q + k] + 2.0 * L.w[k] * xb[wall * n + s];",
     "fp[s * Q + k] + 2.0 * L.w[k] * xb[wall * n + s];"),
    # Eq. xix with the wrong sign
    ("gradient_sign",
     "grad[i][a] = -acc / L.cs2;",
     "grad[i][a] = acc / L.cs2;"),
    # Eq. 2-12 with D~ transposed
    ("flux_Dtilde_transposed",
     "J -= Dt[i * S + j] * grad[j][a];",
     "J -= Dt[j * S + i] * grad[j][a];"),
    # Eq. 3-8: diagonal weight 1/18 instead of 1/36
    ("d2q9_diagonal_weight",
     "(k < 5 ? 1.0 / 9.0 : 1.0 / 36.0)",
     "(k < 5 ? 1.0 / 9.0 : 1.0 / 18.0)"),
    # Eq. 3-10: equal weights 1/7
    ("d3q7_equal_weights",
     "L->w[k] = (k == 0) ? 1.0 / 4.0 : 1.0 / 8.0;",
     "L->w[k] = 1.0 / 7.0;"),
    # D3Q15: the third-order moment x y z counted as even
    ("d3q15_xyz_group",
     "GRP_ODD, GRP_ODD, GRP_EVEN, GRP_EVEN, GRP_EVEN, GRP_EVEN, GRP_EVEN,\n"
     "                     GRP_ODD};",
     "GRP_ODD, GRP_ODD, GRP_EVEN, GRP_EVEN, GRP_EVEN, GRP_EVEN, GRP_EVEN,\n"
     "                     GRP_EVEN};"),
    # D3Q6: a momentum counted as even
    ("d3q6_group",
     "int g[6] = {GRP_CONSERVED, GRP_ODD, GRP_ODD, GRP_ODD, GRP_EVEN, GRP_EVEN};",
     "int g[6] = {GRP_CONSERVED, GRP_ODD, GRP_ODD, GRP_EVEN, GRP_EVEN, GRP_EVEN};"),
    # D2Q4: weights that are not 1/4
    ("d2q4_weights",
     "L->w[k] = 0.25;",
     "L->w[k] = (k == 0) ? 0.3 : 0.7 / 3.0;"),
    # D1Q3: rest weight 1/2 (edges 1/4)
    ("d1q3_rest_weight",
     "L->w[k] = (k == 0) ? 2.0 / 3.0 : 1.0 / 6.0;",
     "L->w[k] = (k == 0) ? 1.0 / 2.0 : 1.0 / 4.0;"),
    # frozen mode that uses the local composition after all
    ("frozen_uses_local_xi",
     "return relax == ORC_FROZEN ? g_xref : xi;",
     "return xi;"),
]

# Child process: point the oracle package at the mutated source and its own
# build path, run the pin suites, and report through the exit code whether a
# pin failed (0), none did (2) or the run broke otherwise (3).
_DRIVER = textwrap.dedent("""
    import os, sys
    root, src, lib = sys.argv[1:4]
    sys.path[:0] = [root, os.path.join(root, "tests")]
    import oracle
    oracle._SRC, oracle._BUILD, oracle._LIB_PATH = src, os.path.dirname(lib), lib
    oracle._lib = None
    import pytest
    rc = pytest.main(["-q", "-x", "-p", "no:cacheprovider", "--no-header", "-o",
                      "addopts="] + sys.argv[4:])
    sys.exit(0 if rc == 1 else (2 if rc == 0 else 3))
""")


def test_every_mutation_site_is_unique():
    src = open(ORACLE_C).read()
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    for name, before, after in MUTANTS:
        assert src.count(before) == 1, name
        assert before != after, name


@pytest.mark.parametrize("name,before,after", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_the_planted_mistake(name, before, after, tmp_path):
    src = open(ORACLE_C).read()
    assert src.count(before) == 1
    mutated = tmp_path / "ms_mrt_oracle.c"
    mutated.write_text(src.replace(before, after))
    lib = tmp_path / "libmsoracle_mutant.so"
    env = dict(os.environ, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "4"))
    r = subprocess.run([sys.executable, "-c", _DRIVER, ROOT, str(mutated), str(lib)] + PIN_FILES,
                       cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 2, "mutant %s survived every pin:\n%s" % (name, r.stdout[-2000:])
    assert r.returncode == 0, "mutant %s: pin run broke (exit %d):\n%s\n%s" % (
        name, r.returncode, r.stdout[-2000:], r.stderr[-2000:])
