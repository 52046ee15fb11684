"""Each plausible mistake planted in a COPY of the oracle's C source (a
dropped term, a wrong index, a flipped comparison, a transposed lookup) must
make at least one oracle pin fail (or stop terminating: several mistakes
turn the switching loop into an endless one).  The copy is compiled to a temporary
library and the pin suite is run against it in a subprocess."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dgs_oracle.c")

MUTATIONS = {
    "ade_dropped_term": ("int64_t diff = A(i, jp) + A(ip, j) - A(i, j) - A(ip, jp);",
                         "int64_t diff = A(i, jp) + A(ip, j) - A(i, j);"),
    "ade_ties_to_last": ("A(ip, j) - A(i, j) - A(ip, jp);\n        if (diff > best) {\n            best = diff;\n            best_job = jp;",
                         "A(ip, j) - A(i, j) - A(ip, jp);\n        if (diff >= best && diff > 0) {\n            best = diff;\n            best_job = jp;"),
    "jde_wrong_index": ("int64_t diff = A(ip, j) + A(i, jp) - A(i, j) - A(ip, jp);",
                        "int64_t diff = A(ip, j) + A(i, jp) - A(i, j) - A(ip, j);"),
    "cc_partner_not_through_sigma": ("int32_t ip = sigma[agent_job[i]];\n        if (cr[i] || cr[ip]) {",
                                     "int32_t ip = agent_job[i];\n        if (cr[i] || cr[ip]) {"),
    "cc_job_owner_unchecked": ("if (cr[owner] || cr[partner]) {", "if (cr[partner]) {"),
    "reevaluate_wrong_set": ("        if (pick_a && pick_a[i]) continue;", "        if (pick_a && !pick_a[i]) continue;"),
    "ade_transposed_wrong_cell": ("int64_t diff = A(i, jp) + AT(j, ip) - A(i, j) - A(ip, jp);",
                                  "int64_t diff = A(i, jp) + AT(ip, j) - A(i, j) - A(ip, jp);"),
    "jde_transposed_wrong_cell": ("int64_t diff = AT(j, ip) + A(i, jp) - A(i, j) - AT(jp, ip);",
                                  "int64_t diff = AT(j, ip) + A(i, jp) - A(i, j) - AT(ip, jp);"),
    "reevaluate_all_ignored": ("const int all = reeval_rule == ORACLE_REEVAL_ALL;", "const int all = 0;"),
    "random_shuffle_off_by_one": ("% (uint64_t)(i + 1));", "% (uint64_t)i);"),
    "apply_non_improving": ("                if (g > 0) {\n                    do_exchange",
                            "                if (g >= 0) {\n                    do_exchange"),
    "greedy_tie_job_first": ("((uint64_t)i << 17) | (uint64_t)j;", "((uint64_t)j << 17) | (uint64_t)i;"),
    "hungarian_sign": ("-A(row - 1, c - 1) - u[row] - v[c]", "-A(row - 1, c - 1) - u[row] + v[c]"),
    "objective_sign": ("f += A(i, tau[i]);", "f -= A(i, tau[i]);"),
    "sequential_ties_to_agent": ("if (dbar[is] > dund[js]) {", "if (dbar[is] >= dund[js]) {"),
    "sequential_no_outer_repeat": ("        if (f == f_start) break;\n    }\n\nfinish:\n    memcpy(tau_out, tau, nb);\n    *f_out = oracle_objective(a, n, tau);\n    if (status == ORACLE_OK && *f_out != f) status = ORACLE_ERR_INTERNAL;\nout:\n    if (stats) *stats = st;\n    free(sigma); free(tau); free(dbar);",
                                   "        break;\n    }\n\nfinish:\n    memcpy(tau_out, tau, nb);\n    *f_out = oracle_objective(a, n, tau);\n    if (status == ORACLE_OK && *f_out != f) status = ORACLE_ERR_INTERNAL;\nout:\n    if (stats) *stats = st;\n    free(sigma); free(tau); free(dbar);"),
    "rect_padding_pitch": ("memcpy(sq + (size_t)i * s, a + (size_t)i * m_jobs,", "memcpy(sq + (size_t)i * m_jobs, a + (size_t)i * m_jobs,"),
    "rect_dummy_job_kept": ("assign_out[i] = tau[i] < m_jobs ? tau[i] : -1;", "assign_out[i] = tau[i];"),
    "sequential_stale_partner": ("                u = is;\n                v = sigma[jbar[is]];", "                u = is;\n                v = jbar[is];"),
}


# Mistakes after which some pin's solve never ends (the loop keeps finding
# the same candidates); for these a pin run that does not finish counts as
# caught.  Every other mistake must make a pin fail outright.
NON_TERMINATING = set()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fopenmp", "-shared", "-fPIC",
                           "-I", os.path.join(ROOT, "oracle"), "-o", str(lib), str(mutant)])
    env = dict(os.environ, DGS_ORACLE_LIB=str(lib))
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=60)
    except subprocess.TimeoutExpired:
        # only a mistake that makes the switching loop endless may be caught this way
        assert name in NON_TERMINATING, f"mutation {name}: the pins did not finish (and it is not known to loop)"
        return
    assert r.returncode != 0, f"mutation {name} survived the oracle pins"
