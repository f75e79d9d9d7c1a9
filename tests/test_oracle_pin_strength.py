"""The oracle's pins must catch plausible mistakes in the oracle.

Each mutant below is a copy of oracle/dp_oracle.cpp with one mistake planted in it -- a dropped term,
a wrong sign, a wrong index or constant, a transposed operand -- at a place where such a mistake is
easy to make when restating the paper.  Every mutant is compiled on its own and the CPU pins
(tests/test_oracle.py, tests/test_oracle_descriptors.py; not the stored values of tests/golden/, which
would catch any change by construction, nor the comparison of the oracle's two forward restatements
with each other) are run against it in a child process: each run must fail.
An unmodified copy goes through the same steps and must pass, which shows that a failure comes from
the planted mistake and not from the harness.  Mistakes are planted in copies on the CPU only; the
oracle itself is not changed.
"""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "dp_oracle.cpp")
PINS = [os.path.join(HERE, "test_oracle.py"), os.path.join(HERE, "test_oracle_descriptors.py")]
# the oracle's two forward restatements compared with each other: a consistency check, not a pin to
# something outside the oracle, so no mutant may count on it
SELF_CHECKS = ["tests/test_oracle.py::test_generic_forward_equals_reverse_pass_forward"]

# (name, what the mistake contradicts, [(text in the oracle, text planted instead), ...])
MUTANTS = [
    ("switch_polynomial", "Eq. (switch): a wrong coefficient of the smoothing polynomial",
     [("T(15.0) * x - T(10.0)", "T(15.0) * x - T(9.0)")]),
    ("switch_derivative_sign", "Eq. (switch): the sign of the 1/r^2 term of ds/dr",
     [("return -u / (r * r) + du / r;", "return u / (r * r) + du / r;")]),
    ("env_row_divides_by_r2", "Eq. (rij): s x/r written as s x/r^2",
     [("E.R[(size_t)k * 4 + 1 + a] = sv * d[a] / r;", "E.R[(size_t)k * 4 + 1 + a] = sv * d[a] / r2;")]),
    ("pair_vector_reversed", "Eq. (rij): r_ij taken as r_i - r_j",
     [("d[a] = p - xi[a];", "d[a] = xi[a] - p;")]),
    ("embedding_xx_skip_dropped", "Eq. (NN): the {x, x} skip of a width-doubling embedding layer",
     [("outs[l][o] = t + (sk == 1 ? x[o] : (sk == 2 ? x[o % ni] : 0.0));", "outs[l][o] = t + (sk == 1 ? x[o] : 0.0);")]),
    ("embedding_backward_skip_dropped", "Eq. (NN): the {x, x} skip in the embedding's reverse pass",
     [("gx[i] += gz * W[(long)i * no + o];\n      if (sk == 1) gx[o] += gy[o];\n      if (sk == 2) gx[o % ni] += gy[o];", "gx[i] += gz * W[(long)i * no + o];\n      if (sk == 1) gx[o] += gy[o];")]),
    ("fitting_identity_skip_dropped", "Eq. (NN): the identity skip of the 240 -> 240 fitting layers",
     [("fx[l + 1][o] = t + (sk == 1 ? fx[l][o] : (sk == 2 ? fx[l][o % ni] : 0.0));", "fx[l + 1][o] = t;")]),
    ("fitting_output_activated", "Eq. (fitting): tanh applied to the linear output layer",
     [("double t = last ? z : std::tanh(z);", "double t = std::tanh(z);")]),
    ("type_pair_net_transposed", "Eq. (G2): the net of pair (a_i, a_j) taken as that of (a_j, a_i)",
     [("return c.type_one_side ? aj : ai * c.ntypes + aj;", "return c.type_one_side ? aj : aj * c.ntypes + ai;")]),
    ("descriptor_axis_row_shifted", "se_e2_a: D = T T_<^T with the wrong rows of T_<",
     [("acc += S.T[(size_t)m * 4 + q] * S.T[(size_t)l * 4 + q];", "acc += S.T[(size_t)m * 4 + q] * S.T[(size_t)(l + 1) * 4 + q];")]),
    ("descriptor_normalisation_dropped", "se_e2_a: the 1/N_c of T = G^T R / N_c",
     [("S.T[(size_t)m * 4 + q] = acc / nc;", "S.T[(size_t)m * 4 + q] = acc;")]),
    ("generic_descriptor_normalisation", "se_e2_a: 1/N_c^2 instead of 1/N_c in the templated energy",
     [("for (auto& v : Tm) v = v / T((double)nc);", "for (auto& v : Tm) v = v / T((double)nc * nc);")]),
    ("reverse_dT_second_term_dropped", "se_e2_a reverse pass: the T_< branch of dE/dT",
     [("if (p < A)\n", "if (false)\n")]),
    ("reverse_tangential_sign", "chain rule through u = r_ij / r: the sign of the projection term",
     [("(sv / r) * (g[1 + a] - gvu * u[a])", "(sv / r) * (g[1 + a] + gvu * u[a])")]),
    ("virial_sign", "virial: Xi = -sum r_ij (x) dE/dr_ij with the sign flipped",
     [("virial[3 * a + b] -= g[a] * d[b];", "virial[3 * a + b] += g[a] * d[b];")]),
    ("virial_index", "virial: the outer product with a repeated index",
     [("virial[3 * a + b] -= g[a] * d[b];", "virial[3 * a + b] -= g[a] * d[a];")]),
    ("list_order_reversed", "neighbour list: farthest first instead of nearest first",
     [("if (a.r2bits != b.r2bits) return a.r2bits < b.r2bits;", "if (a.r2bits != b.r2bits) return a.r2bits > b.r2bits;")]),
    ("list_images_too_few", "neighbour list: too few periodic images searched in narrow cells",
     [("K[d] = (int)std::ceil(L.lrc / width) + 1;", "K[d] = (int)std::ceil(L.lrc / width) - 1;")]),
    ("se_e2_r_normalisation", "se_e2_r: 1/N_c^2 instead of 1/N_c",
     [("D[P.doff + m] = acc / nc;", "D[P.doff + m] = acc / ((double)nc * nc);")]),
    ("se_e3_theta_radial_only", "se_e3: theta_jk = s_j s_k instead of R_j . R_k",
     [("const double th = dot4(&E.R[(size_t)j * 4], &E.R[(size_t)k * 4]);", "const double th = E.R[(size_t)j * 4] * E.R[(size_t)k * 4];")]),
    ("se_e3_backward_one_sided", "se_e3 reverse pass: dtheta_jk/dR_k = R_j dropped",
     [("gR[(size_t)k * 4 + q] += gth * Rj[q];", "gR[(size_t)k * 4 + q] += 0.0 * Rj[q];")]),
    ("quintic_coefficient", "Eq. (compress): a wrong coefficient of the quintic piece",
     [("(14.0 * d1 + 16.0 * d0)", "(14.0 * d1 + 15.0 * d0)")]),
    ("table_offset_from_wrong_node", "Eq. (compress): the piece evaluated from the interval's far node",
     [("double t = s - tab->node(l);", "double t = s - tab->node(l + 1);")]),
    ("loss_force_coefficient", "Sec. II.B loss: the factor 2 of d(pF |dF|^2 / 3N) dropped",
     [("const double cF = 2.0 * pF / (3.0 * n)", "const double cF = pF / (3.0 * n)")]),
    ("loss_virial_coefficient", "Sec. II.B loss: 1/(3N) instead of 1/(9N) in the virial term's derivative",
     [("cX = v_ref ? 2.0 * pXi / (9.0 * n) : 0.0;", "cX = v_ref ? 2.0 * pXi / (3.0 * n) : 0.0;")]),
    # the same mistake planted consistently in every restatement (forward, reverse pass, templated
    # energy, jets), so that only a pin to something outside the oracle can catch it
    ("identity_skip_dropped_everywhere", "Eq. (NN): no + x skip on equal-width layers, in all paths",
     [("inline int skip_kind(int n_in, int n_out) { return n_out == n_in ? 1 :",
       "inline int skip_kind(int n_in, int n_out) { return n_out == n_in ? 0 :")]),
    ("xx_skip_dropped_everywhere", "Eq. (NN): no {x, x} skip on width-doubling layers, in all paths",
     [("(n_out == 2 * n_in ? 2 : 0); }", "(n_out == 2 * n_in ? 0 : 0); }")]),
    ("descriptor_normalisation_dropped_everywhere", "se_e2_a: no 1/N_c in T, forward and reverse alike",
     [("S.T[(size_t)m * 4 + q] = acc / nc;", "S.T[(size_t)m * 4 + q] = acc;"),
      ("gR[(size_t)k * 4 + q] = acc / nc;", "gR[(size_t)k * 4 + q] = acc;"),
      ("gG[m] = acc / nc;", "gG[m] = acc;"),
      ("for (auto& v : Tm) v = v / T((double)nc);", "for (auto& v : Tm) (void)v;")]),
]


def _run_pins(work, name, text):
    d = os.path.join(work, name)
    os.makedirs(d)
    src = os.path.join(d, "dp_oracle.cpp")
    with open(src, "w") as f:
        f.write(text)
    lib = oracle.compile_source(src, os.path.join(d, "libdporacle.so"))
    env = dict(os.environ, DP_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"] + PINS
    for t in SELF_CHECKS:
        cmd += ["--deselect", t]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    tail = (p.stdout + p.stderr).strip().splitlines()[-3:]
    return p.returncode, tail


@pytest.mark.slow
def test_every_planted_mistake_fails_a_pin():
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    with open(SRC) as f:
        base = f.read()
    jobs = [("unmodified", base)]
    for name, _, sites in MUTANTS:
        text = base
        for old, new in sites:
            assert text.count(old) == 1, f"{name}: each planted site must occur once in the oracle"
            text = text.replace(old, new)
        jobs.append((name, text))
    work = tempfile.mkdtemp(prefix="orc_mutants_")
    try:
        with ThreadPoolExecutor(max_workers=max(1, min(8, (os.cpu_count() or 2) // 2))) as ex:
            results = dict(zip([j[0] for j in jobs], ex.map(lambda j: _run_pins(work, *j), jobs)))
    finally:
        shutil.rmtree(work, ignore_errors=True)
    rc, tail = results.pop("unmodified")
    assert rc == 0, f"the unmodified copy must pass its pins: {tail}"
    survivors = {n: t for n, (rc, t) in results.items() if rc != 1}
    assert not survivors, f"planted mistakes that no pin caught (or that did not fail cleanly): {survivors}"
