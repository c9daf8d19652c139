"""The oracle's pins have teeth: each plausible mistake below, planted in a
copy of the oracle's C source (never in the oracle itself), makes at least
one of the oracle pin tests fail.  Each mutant is compiled like the oracle
and the pin tests run against it in a child process (CCS_ORACLE_LIB)."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PINS = ["tests/test_oracle_generator.py", "tests/test_oracle_score.py",
        "tests/test_oracle_decode.py"]

# (name, text in ccs_oracle.c, replacement); the text occurs exactly once
MUTANTS = [
    # the score, Eq. (15) and Alg. 8
    ("score: c_omega + c_0 (wrong sign)",
     "? best_count : best_count - c0;", "? best_count : best_count + c0;"),
    ("score: c_0 term dropped",
     "? best_count : best_count - c0;", "? best_count : best_count;"),
    ("score: count mode subtracts c_0 too",
     "? best_count : best_count - c0;", "? best_count - c0 : best_count - c0;"),
    ("score: tie goes to the larger value",
     "(c == best_count && v[a] < v[best])", "(c == best_count && v[a] > v[best])"),
    ("score: zero can be the mode",
     "        if (v[a] == 0.0) continue;\n", ""),
    ("score: strict threshold",
     "    *score = (score_mode == ORACLE_SCORE_COUNT) ? best_count : best_count - c0;\n"
     "    return *score >= alpha;",
     "    *score = (score_mode == ORACLE_SCORE_COUNT) ? best_count : best_count - c0;\n"
     "    return *score > alpha;"),
    ("shifted score: candidate from the wrong row",
     "const double w = r[rows[pos]];", "const double w = r[rows[(pos + 1) % d]];"),
    ("shifted score: a zero candidate is scored like any other",
     "    if (w == 0.0) {\n        *omega = 0.0;", "    if (0) {\n        *omega = 0.0;"),
    ("iteration cap checked one iteration late",
     "        if (it == max_iter) { status = ORACLE_MAX_ITER; break; }\n        /* T",
     "        if (it == max_iter + 1) { status = ORACLE_MAX_ITER; break; }\n        /* T"),
    ("serial: no stall exit",
     "        if (empty_run == stall_run) { status = ORACLE_STALLED; break; }\n        it += 1;",
     "        it += 1;"),
    ("shifted decode: stalls after one empty iteration",
     "position on the same r) */\n    const int32_t stall_run = shifted ? d : 1;",
     "position on the same r) */\n    const int32_t stall_run = 1; (void)shifted;"),
    ("shifted decode: an empty iteration does not move the position",
     "            it += 1;\n            if (r0_hist) r0_hist[it] = r0;\n            continue;",
     "            continue;"),
    ("serial: shifted decode stalls after one empty sweep",
     "such sweeps in a row */\n    const int32_t stall_run = shifted ? d : 1;",
     "such sweeps in a row */\n    const int32_t stall_run = 1;"),
    ("shifted decode: position does not wrap around d",
     "shifted ? it % d : -1", "shifted ? (it < d ? it : d - 1) : -1"),
    ("shifted score: rows counted from the end",
     "const double w = r[rows[pos]];", "const double w = r[rows[d - 1 - pos]];"),
    ("shifted decode: position counted from 1",
     "shifted ? it % d : -1", "shifted ? (it + 1) % d : -1"),
    # Alg. 2's loop body and stopping rule
    ("apply: x_hat_j overwritten instead of accumulated",
     "if (accept[j]) x_hat[j] = x_hat[j] + omega[j];", "if (accept[j]) x_hat[j] = omega[j];"),
    ("residual: A x_hat - y",
     "r[i] = y[i] - row_sum(csr_ptr, csr_cols, x_hat, i);\n    return 0;",
     "r[i] = row_sum(csr_ptr, csr_cols, x_hat, i) - y[i];\n    return 0;"),
    ("residual: rows summed in descending column order",
     "    double s = +0.0;\n    for (int64_t p = csr_ptr[i]; p < csr_ptr[i + 1]; ++p) {",
     "    double s = +0.0;\n    for (int64_t p = csr_ptr[i + 1] - 1; p >= csr_ptr[i]; --p) {"),
    ("row sum: gathers v[p] instead of v[col(p)]",
     "double vj = v[csr_cols[p]];", "double vj = v[p];"),
    ("no stall exit in Parallel-l0",
     "        if (empty_run == stall_run) { status = ORACLE_STALLED; break; }\n        if (trace)",
     "        if (trace)"),
    ("init: r starts at 0",
     "    for (int64_t i = 0; i < m; ++i) r[i] = y[i];\n    int64_t r0 = oracle_l0(m, r);\n"
     "    int32_t it = 0;\n    if (r0_hist) r0_hist[0] = r0;\n    int32_t status;\n"
     "    /* R3: iterations in a row",
     "    for (int64_t i = 0; i < m; ++i) r[i] = 0.0;\n    int64_t r0 = oracle_l0(m, r);\n"
     "    int32_t it = 0;\n    if (r0_hist) r0_hist[0] = r0;\n    int32_t status;\n"
     "    /* R3: iterations in a row"),
    ("||r||_0 counts -0.0 as nonzero",
     "if (r[i] != 0.0) ++c;", "if (r[i] != 0.0 || signbit(r[i])) ++c;"),
    ("score pass: every column counted as accepted",
     "        accepted += a;\n", "        accepted += 1;\n"),
    ("history: r0 recorded at the old index",
     "        it += 1;\n        if (r0_hist) r0_hist[it] = r0;\n    }\n    out->status = status;\n"
     "    out->iterations = it;\n    out->r0_final = r0;\ndone:",
     "        if (r0_hist) r0_hist[it] = r0;\n        it += 1;\n    }\n    out->status = status;\n"
     "    out->iterations = it;\n    out->r0_final = r0;\ndone:"),
    # Serial-l0 (Alg. 1)
    ("serial: shifted position does not wrap around d",
     "oracle_score_column_shifted(d, rows, r, it % d, alpha,",
     "oracle_score_column_shifted(d, rows, r, it < d ? it : d - 1, alpha,"),
    ("serial: shifted position counted from 1",
     "oracle_score_column_shifted(d, rows, r, it % d, alpha,",
     "oracle_score_column_shifted(d, rows, r, (it + 1) % d, alpha,"),
    ("serial: last row of N(j) not recomputed",
     "            for (int t = 0; t < d; ++t) {\n                int64_t i = rows[t];",
     "            for (int t = 0; t < d - 1; ++t) {\n                int64_t i = rows[t];"),
    ("serial: ||r||_0 not updated",
     "                r0 += (r[i] != 0.0) - was;\n", "                (void)was;\n"),
    # the expander and the measurement
    ("expander: row m-1 never drawn",
     "bounded_draw(&state, (uint32_t)m);", "bounded_draw(&state, (uint32_t)(m - 1));"),
    ("expander: duplicate rows kept",
     "            if (!seen) col[got++] = row;", "            col[got++] = row; (void)seen;"),
    ("expander: rows left unsorted",
     "            while (b >= 0 && col[b] > v) { col[b + 1] = col[b]; --b; }", ""),
    ("transpose: columns visited in descending order",
     "    for (int64_t j = 0; j < n; ++j)\n        for (int t = 0; t < d; ++t) {\n"
     "            int32_t i = csc_rows[j * d + t];",
     "    for (int64_t j = n - 1; j >= 0; --j)\n        for (int t = 0; t < d; ++t) {\n"
     "            int32_t i = csc_rows[j * d + t];"),
    ("Lemire: rejection threshold dropped",
     "        while (low < threshold) {", "        while (0 && low < threshold) {"),
    ("transpose: row pointers not accumulated",
     "    for (int64_t i = 0; i < m; ++i) csr_ptr[i + 1] += csr_ptr[i];\n", ""),
    ("SplitMix64: wrong increment",
     "*state += 0x9e3779b97f4a7c15ULL;", "*state += 0x9e3779b97f4a7c14ULL;"),
    ("unshifted decode scores only row 0",
     "shifted ? it % d : -1", "shifted ? it % d : 0"),
    ("serial: x_hat_j overwritten instead of accumulated",
     "            x_hat[j] = x_hat[j] + omega;", "            x_hat[j] = omega;"),
    # column scaling (Sec. 4.3.3)
    ("scales: 19 bits instead of 20",
     "const uint64_t k = oracle_splitmix64_next(&state) >> 44;",
     "const uint64_t k = oracle_splitmix64_next(&state) >> 45;"),
    ("scales: grid 2^-21",
     "s[j] = 1.0 + (double)k / 1048576.0;", "s[j] = 1.0 + (double)k / 2097152.0;"),
    ("scaled measure: rows summed in descending column order",
     "        double acc = +0.0;\n        for (int64_t p = csr_ptr[i]; p < csr_ptr[i + 1]; ++p) {",
     "        double acc = +0.0;\n        for (int64_t p = csr_ptr[i + 1] - 1; p >= csr_ptr[i]; --p) {"),
    ("scaled measure: scale dropped",
     "const double v = s[j] * x[j];", "const double v = x[j];"),
    ("unscale: multiplies",
     "x[j] = z[j] / s[j];", "x[j] = z[j] * s[j];"),
]


def _build_mutant(tmp, name, old, new):
    src = open(os.path.join(ORACLE, "ccs_oracle.c")).read()
    assert src.count(old) == 1, f"mutant '{name}': its text occurs {src.count(old)} times"
    d = tempfile.mkdtemp(dir=tmp)
    shutil.copy(os.path.join(ORACLE, "ccs_oracle.h"), d)
    with open(os.path.join(d, "ccs_oracle.c"), "w") as f:
        f.write("#include <math.h>\n" + src.replace(old, new))
    so = os.path.join(d, "libmutant.so")
    subprocess.run(["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                    "-fPIC", "-shared", "-o", so, os.path.join(d, "ccs_oracle.c")],
                   check=True, capture_output=True)
    return so


def _pins_fail(so):
    """Run the pin tests against one mutant: (exit code, first failing test).
    A mutant that makes a pin hang (the generator cannot find d distinct
    rows, say) is stopped by the per-test timeout and counts as caught."""
    env = dict(os.environ, CCS_ORACLE_LIB=so, OMP_NUM_THREADS="1",
               OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    proc = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q",
                           "-p", "no:cacheprovider", "-m", "not gpu",
                           "--timeout", "30", "--timeout-method", "thread"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    failed = [ln for ln in proc.stdout.splitlines() if ln.startswith("FAILED")]
    if not failed and "Timeout" in proc.stdout + proc.stderr:
        failed = ["timeout"]
    if proc.returncode < 0:  # the mutant crashed the child (an out-of-bounds write)
        failed = failed or [f"crashed (signal {-proc.returncode})"]
    # exit code 1 (some test failed) or a crash: caught; 2 to 5: the run broke
    return proc.returncode, (failed[0] if failed else proc.stdout[-1500:])


def test_mutant_texts_are_unique():
    src = open(os.path.join(ORACLE, "ccs_oracle.c")).read()
    for name, old, _ in MUTANTS:
        assert src.count(old) == 1, name


@pytest.mark.timeout(900)
def test_every_planted_mistake_fails_a_pin(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    pytest.importorskip("pytest_timeout")  # the child runs stop a hanging pin with it
    sos = {name: _build_mutant(str(tmp_path), name, old, new) for name, old, new in MUTANTS}
    workers = max(1, min(len(sos), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        results = dict(zip(sos, ex.map(_pins_fail, sos.values())))
    for n, (rc, what) in results.items():
        print(f"{n}: exit {rc}, {what}")
    survivors = [n for n, (rc, _) in results.items() if rc == 0]
    broken = {n: out for n, (rc, out) in results.items() if rc > 1}
    assert not broken, broken
    assert not survivors, f"mistakes no pin catches: {survivors}"
