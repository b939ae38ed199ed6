"""The oracle's pins catch plausible mistakes (no GPU).

Each mutant below is the oracle source with one planted mistake of the kind
that is easy to make when writing it from the paper: a dropped term, a
flipped sign or handedness, a transposed operand, a wrong index, a tie rule
or boundary taken the other way. Every mutant is compiled on the CPU into
its own library and the oracle's pin tests run against it in a subprocess
(`LIGEN_ORACLE_LIB`); each mutant must make at least one pin fail. The clean
oracle passes the same tests in the ordinary suite.

Not planted: the rotamer-class edges (a reading with no value in the paper,
"parity unpinned") and the restart counter layout of the RNG (a reading the
CUDA path checks bit for bit, but nothing in the paper fixes).
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ligen_oracle.cpp")
PIN_FILES = ["tests/test_oracle_rng_rot.py", "tests/test_oracle_geometry.py", "tests/test_oracle_scoring.py",
             "tests/test_bucketing_and_inputs.py", "tests/test_oracle_search.py"]

# name -> (text in the oracle, replacement, which occurrence (0-based))
MUTANTS = {
    "splitmix_constant": ("0x9E3779B97F4A7C15ull", "0x9E3779B97F4A7C17ull", 0),
    "uniform_bits": ("(double)(z >> 40) * (1.0 / 16777216.0)", "(double)(z >> 41) * (1.0 / 16777216.0)", 0),
    "shoemake_sin_cos": ("q[1] = r1 * std::sin(a);\n  q[2] = r1 * std::cos(a);",
                         "q[1] = r1 * std::cos(a);\n  q[2] = r1 * std::sin(a);", 0),
    "quat_mul_cross_sign": ("double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];",
                            "double x = a[0] * b[1] + a[1] * b[0] - a[2] * b[3] + a[3] * b[2];", 0),
    "quat_to_mat_sign": ("m[1] = 2 * (x * y - w * z);", "m[1] = 2 * (x * y + w * z);", 0),
    "cube_quarter_turn_sign": ("ang = ((k - 4) % 2 == 0) ? kPi / 2 : -kPi / 2;",
                               "ang = ((k - 4) % 2 == 0) ? -kPi / 2 : kPi / 2;", 0),
    "cube_diagonal_bits": ("ax[0] = (m & 4) ? -1 : 1; ax[1] = (m & 2) ? -1 : 1; ax[2] = (m & 1) ? -1 : 1;",
                           "ax[0] = (m & 1) ? -1 : 1; ax[1] = (m & 2) ? -1 : 1; ax[2] = (m & 4) ? -1 : 1;", 0),
    "rodrigues_left_handed": ("scale(cross(k, v), s)", "scale(cross(v, k), s)", 0),
    "fragment_tie_side": ("(na == nb && !side[0])", "(na == nb && side[0])", 0),
    "fragment_larger_side": ("bool a_moves = (na < nb)", "bool a_moves = (na > nb)", 0),
    "axis_endpoints_swapped": ("axis[2 * r] = a_moves ? b : a;\n    axis[2 * r + 1] = a_moves ? a : b;",
                               "axis[2 * r] = a_moves ? a : b;\n    axis[2 * r + 1] = a_moves ? b : a;", 0),
    "trilinear_weights_transposed": (
        "double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);",
        "double w = (dx ? f[1] : 1 - f[1]) * (dy ? f[0] : 1 - f[0]) * (dz ? f[2] : 1 - f[2]);", 0),
    "trilinear_upper_face_outside": ("if (!(u[a] >= 0.0 && u[a] <= n[a] - 1)) {",
                                     "if (!(u[a] >= 0.0 && u[a] < n[a] - 1)) {", 0),
    "gradient_upper_face_outside": ("if (!(u[a] >= 0.0 && u[a] <= n[a] - 1)) {",
                                    "if (!(u[a] >= 0.0 && u[a] < n[a] - 1)) {", 1),
    "gradient_without_spacing": ("grad[0] += sx * wy * wz * v / g->spacing;", "grad[0] += sx * wy * wz * v;", 0),
    "score_sign": ("    s -= e;\n    a += std::fabs(e);", "    s += e;\n    a += std::fabs(e);", 0),
    "penalty_dropped": ("if (!inb) e = penalty;\n    if (E) E[i] = e;", "if (!inb) e = 0.0;\n    if (E) E[i] = e;", 0),
    "norm_without_abs": ("a += std::fabs(e);", "a += e;", 0),
    "centroid_not_subtracted": ("for (int a = 0; a < 3; ++a) c0[a] /= N;",
                                "for (int a = 0; a < 3; ++a) c0[a] = 0.0;", 0),
    "torsion_about_input_axis": (
        "double pv[3] = {y[3 * v], y[3 * v + 1], y[3 * v + 2]};\n"
        "    double dir[3] = {y[3 * v] - y[3 * u], y[3 * v + 1] - y[3 * u + 1], y[3 * v + 2] - y[3 * u + 2]};",
        "double pv[3] = {L->xyz[3 * v], L->xyz[3 * v + 1], L->xyz[3 * v + 2]};\n"
        "    double dir[3] = {L->xyz[3 * v] - L->xyz[3 * u], L->xyz[3 * v + 1] - L->xyz[3 * u + 1], "
        "L->xyz[3 * v + 2] - L->xyz[3 * u + 2]};", 0),
    "torsion_wrap_upper": ("if (deg >= 180) deg -= 360;", "if (deg > 180) deg -= 360;", 0),
    "jitter_halved": ("(2.0 * u[3 + a] - 1.0) * P->jitter", "(u[3 + a] - 0.5) * P->jitter", 0),
    "rigid_world_frame": ("or_quat_mul(qr, gk, qk);\n      fill(qk);", "or_quat_mul(gk, qr, qk);\n      fill(qk);", 0),
    "rigid_tie_highest": ("      if (s > best) {\n        second = best;", "      if (s >= best) {\n        second = best;", 0),
    "sweep_tie_highest": ("          if (s > bs) {", "          if (s >= bs) {", 0),
    "sweep_forgets_base": ("count[b] = (base + jb) % nt;", "count[b] = jb % nt;", 0),
    "sweep_bonds_reversed": ("for (int b = 0; b < n; ++b) {\n        int base = count[b];",
                             "for (int b = n - 1; b >= 0; --b) {\n        int base = count[b];", 0),
    "sweep_gap_second_lost": ("            sc = bs;\n            bs = s;", "            bs = s;", 0),
    "top_k_tie_highest": (
        "std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return scores[a] > scores[b]; });",
        "std::sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) "
        "{ return scores[a] > scores[b] || (scores[a] == scores[b] && a > b); });", 0),
    "exhaustive_identity_only": ("for (int k = 0; k < P->n_rigid; ++k) {\n      double gk[4], q[4];",
                                 "for (int k = 0; k < 1; ++k) {\n      double gk[4], q[4];", 0),
    "grad_quaternion_unprojected": ("grad[3 + k] = (dqh[k] - qh[k] * proj) / qn;", "grad[3 + k] = dqh[k] / qn;", 0),
    "grad_torque_sign": (
        "double c[3] = {om[1] * d[2] - om[2] * d[1], om[2] * d[0] - om[0] * d[2], om[0] * d[1] - om[1] * d[0]};",
        "double c[3] = {om[2] * d[1] - om[1] * d[2], om[0] * d[2] - om[2] * d[0], om[1] * d[0] - om[0] * d[1]};", 0),
    "refine_never_halves": ("st *= 0.5; sq *= 0.5; sth *= 0.5;", "st *= 1.0; sq *= 1.0; sth *= 1.0;", 0),
    "refine_accepts_equal": ("if (S2 > S) {", "if (S2 >= S) {", 0),
    "eq1_ratio_inverted": ("return b * sm * t / ws;", "return b * sm * ws / t;", 0),
    "atom_class_edge": ("if (n_atoms <= 32) return 0;", "if (n_atoms < 32) return 0;", 0),
    "validate_accepts_cycles": ("return count == N ? 0 : 1;", "return 0;", 0),
}


def _plant(text: str, old: str, new: str, nth: int) -> str:
    pos = -1
    for _ in range(nth + 1):
        pos = text.find(old, pos + 1)
        assert pos >= 0, f"mutation site not found: {old[:60]!r}"
    return text[:pos] + new + text[pos + len(old):]


def _run_mutant(name: str, tmp: str) -> tuple[str, int, str]:
    old, new, nth = MUTANTS[name]
    src = os.path.join(tmp, f"{name}.cpp")
    so = os.path.join(tmp, f"{name}.so")
    with open(SRC) as f:
        text = f.read()
    with open(src, "w") as f:
        f.write(_plant(text, old, new, nth))
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", so, src], check=True)
    env = dict(os.environ, LIGEN_ORACLE_LIB=so, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", *PIN_FILES, "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode, r.stdout[-3000:]


@pytest.fixture(scope="module")
def mutant_results(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("oracle_mutants"))
    workers = max(2, min(8, os.cpu_count() or 2))
    with ThreadPoolExecutor(workers) as ex:
        return {n: (rc, out) for n, rc, out in ex.map(lambda n: _run_mutant(n, tmp), MUTANTS)}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(mutant_results, name):
    rc, out = mutant_results[name]
    # exit code 1: at least one pin failed (2+ would be an error or an interrupted run)
    assert rc == 1 and " failed" in out, f"{name} survived the pins (exit {rc}):\n{out}"
