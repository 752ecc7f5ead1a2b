"""The oracle's pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of ``oracle/oracle.c`` (a dropped term,
a flipped sign, a wrong index or operand, the misprinted direction update of
Algorithm 1), compiles it to a temporary library and runs the pin tests of
``test_oracle_operator.py``, ``test_oracle_ainv.py`` and ``test_oracle_pcg.py``
against it in a child process. Every mutant must fail at least one pin; the
unmodified source must fail none in the same harness. The planted mistakes live
only in temporary copies on the CPU."""
import json
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# (name, [(text in oracle.c, replacement), ...]); each text occurs exactly once
MUTANTS = [
    # operator (Section 3, Eq. 9 in SPD form plus the mass shift)
    ("offdiag_sign", [("cnt = row_add(cols, vals, cnt, m, -face[f].c);", "cnt = row_add(cols, vals, cnt, m, face[f].c);")]),
    ("shift_dropped", [("double diag = shift[(size_t)j * nx + i];", "double diag = 0.0;")]),
    ("no_periodic_wrap", [("{ iw, j, c_e[(size_t)j * nx + iw], nx > 1 },", "{ iw, j, c_e[(size_t)j * nx + iw], i > 0 },"),
                          ("{ ie, j, c_e[(size_t)j * nx + i], nx > 1 },", "{ ie, j, c_e[(size_t)j * nx + i], i + 1 < nx },")]),
    ("east_face_index", [("{ ie, j, c_e[(size_t)j * nx + i], nx > 1 },", "{ ie, j, c_e[(size_t)j * nx + ie], nx > 1 },")]),
    ("north_uses_east", [("j + 1 < ny ? c_n[(size_t)j * nx + i] : 0.0", "j + 1 < ny ? c_e[(size_t)j * nx + i] : 0.0")]),
    # factored approximate inverse (Section 3)
    ("update_sign", [("if (pos >= 0) P->zval[pos] -= f * P->zval[t];", "if (pos >= 0) P->zval[pos] += f * P->zval[t];")]),
    ("p_uses_z_i", [("int64_t pos = zfind(P, j, P->scol[t]);", "int64_t pos = zfind(P, i, P->scol[t]);")]),
    ("update_factor_inverted", [("double f = pj / di;", "double f = di / pj;")]),
    ("drop_scale_inverted", [("if (fabs(P->zval[t]) * sqrt(sd[m] / sd[j]) < tau) P->zval[t] = 0.0;",
                              "if (fabs(P->zval[t]) * sqrt(sd[j] / sd[m]) < tau) P->zval[t] = 0.0;")]),
    ("drop_unscaled", [("if (fabs(P->zval[t]) * sqrt(sd[m] / sd[j]) < tau) P->zval[t] = 0.0;",
                        "if (fabs(P->zval[t]) < tau) P->zval[t] = 0.0;")]),
    ("tril_a2_built_as_tril_a", [("case O_PAT_TRIL_A2: q = 2; break;", "case O_PAT_TRIL_A2: q = 1; break;")]),
    ("pattern_rows_below", [("if (m < k) out[cnt++] = m;", "if (m > k) out[cnt++] = m;")]),
    ("band_t_with_wrap_face", [("abs(P->pi[m] - P->pi[k]) == 1);", "(abs(P->pi[m] - P->pi[k]) == 1 || abs(P->pi[m] - P->pi[k]) == P->nx - 1));")]),
    # preconditioner apply s = Z D^-1 Z^T r
    ("apply_d_not_inverted", [("t[j] = acc / P->d[j];", "t[j] = acc * P->d[j];")]),
    ("apply_second_product_transposed", [("s[P->zrow[u]] += P->zval[u] * t[j];", "s[j] += P->zval[u] * t[P->zrow[u]];")]),
    # Algorithm 1
    ("direction_uses_r", [("d[m] = s[m] + beta * d[m];", "d[m] = r[m] + beta * d[m];")]),
    ("beta_inverted", [("double beta = rho_new / rho;", "double beta = rho / rho_new;")]),
    ("alpha_unpreconditioned", [("double alpha = rho / dq;", "double alpha = dot(r, r, n) / dq;")]),
    ("x_update_sign", [("x[m] += alpha * d[m];", "x[m] -= alpha * d[m];")]),
    ("rho_unpreconditioned", [("double rho_new = dot(s, r, n);", "double rho_new = dot(r, r, n);")]),
    ("stop_on_squared_norm", [("      rnorm = sqrt(dot(r, r, n));\n      double beta", "      rnorm = dot(r, r, n);\n      double beta")]),
]

# pin tests run against each mutant: (module, function, keyword arguments as JSON)
PINS = [
    ("test_oracle_operator", "test_hand_derived_operator", {}),
    ("test_oracle_operator", "test_symmetry_rowsums_and_nnz", {"seed_cfg": "TINY0"}),
    ("test_oracle_operator", "test_closed_form_spectrum", {}),
    ("test_oracle_operator", "test_cg_on_eigenvectors_terminates", {}),
    ("test_oracle_ainv", "test_full_pattern_is_exact_inverse", {}),
    ("test_oracle_ainv", "test_pattern_invariants", {"pattern": 0, "q": 1, "tau": 0.0}),
    ("test_oracle_ainv", "test_pattern_invariants", {"pattern": 1, "q": 2, "tau": 0.05}),
    ("test_oracle_ainv", "test_pattern_invariants", {"pattern": 1, "q": 2, "tau": 0.3}),
    ("test_oracle_ainv", "test_proposition3_closed_form_and_decay", {}),
    ("test_oracle_ainv", "test_banded_pattern_is_truncation", {"q": 2}),
    ("test_oracle_ainv", "test_band_t_on_a_grid_uses_row_blocks", {}),
    ("test_oracle_ainv", "test_proposition1_limit_spectrum", {}),
    ("test_oracle_ainv", "test_drop_rule_hand_computed", {}),
    ("test_oracle_ainv", "test_pattern_invariants", {"pattern": 1, "q": 2, "tau": 0.0}),
    ("test_oracle_pcg", "test_matches_dense_solve", {"pattern": 0, "tau": 0.0}),
    ("test_oracle_pcg", "test_matches_dense_solve", {"pattern": 1, "tau": 0.05}),
    ("test_oracle_pcg", "test_convergence_bound_eq10", {}),
    ("test_oracle_pcg", "test_special_cases", {}),
    ("test_oracle_pcg", "test_power_of_two_scaling_is_exact", {}),
]

# child process: load the oracle package against the given library, run the pins
CHILD = r"""
import json, sys, traceback
root, lib, pins = sys.argv[1], sys.argv[2], json.loads(sys.argv[3])
sys.path[:0] = [root, root + "/tests"]
import oracle
oracle.build = lambda force=False: lib
oracle._lib = None
import gridgen, importlib
failed = []
for mod, fn, kw in pins:
    if kw.get("seed_cfg") == "TINY0":
        kw = dict(kw, seed_cfg=(gridgen.TINY, 0))
    try:
        getattr(importlib.import_module(mod), fn)(**kw)
    except Exception as e:                      # AssertionError or an error raised by the mutant
        failed.append("%s.%s%s: %s" % (mod, fn, kw, type(e).__name__))
print(json.dumps(failed))
"""


def _run(name, reps, tmp):
    src = open(SRC).read()
    for old, new in reps:
        assert src.count(old) == 1, (name, old, src.count(old))
        src = src.replace(old, new)
    c = os.path.join(tmp, name + ".c")
    so = os.path.join(tmp, name + ".so")
    with open(c, "w") as f:
        f.write(src)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                           "-o", so, c, "-lm"])
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, so, json.dumps(PINS)], capture_output=True, text=True,
                       timeout=600, env=env)
    if r.returncode != 0:                      # the mutant crashed the pins' process
        return ["process exited with %d" % r.returncode]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("oracle_mutants"))
    cases = [("control", [])] + MUTANTS
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as pool:
        futs = {name: pool.submit(_run, name, reps, tmp) for name, reps in cases}
        return {name: f.result() for name, f in futs.items()}


def test_unmodified_oracle_passes_every_pin(outcomes):
    assert outcomes["control"] == []


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(outcomes, name):
    assert outcomes[name], "no pin fails with the mistake '%s' planted in the oracle" % name
