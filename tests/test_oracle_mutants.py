"""The pins are sensitive: plausible one-token mistakes planted in a copy of
the oracle (compiled on the CPU, in a temporary directory) make the oracle
pin tests fail.  Each mutant runs the pin suite in a child process with a time
limit, so a mutant that no longer terminates counts as caught."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    # merge takes B on ties (unstable)
    "merge_ties_to_B": ("if (B[k] < A[j]) { C[i] = B[k];", "if (B[k] <= A[j]) { C[i] = B[k];"),
    # second Lemma condition tested non-strictly
    "cond2_strict": ("B[k-1] >= A[j]", "B[k-1] > A[j]"),
    # first Lemma condition tested non-strictly
    "cond1_nonstrict": ("A[j-1] > B[k]", "A[j-1] >= B[k]"),
    # source index of a B element loses its offset m
    "src_offset": ("if (src) src[i] = m + k; k++; }        \\",
                   "if (src) src[i] = k; k++; }        \\"),
    # k_low not raised on the first condition
    "k_low_update": ("k_low = k; k_low_set = 1;", "k_low_set = 1;"),
    # j_low not raised on the second condition
    "j_low_update": ("j_low = j;", "(void)0;"),
    # merge pass: payloads taken from the pair-relative position (offset lost)
    "pass_payload_offset": ("int64_t from = a0 + s[i];", "int64_t from = s[i];"),
    # merge pass: pairs advance by one run instead of two
    "pass_stride": ("for (int64_t a0 = 0; a0 < N; a0 += 2 * w) {",
                    "for (int64_t a0 = 0; a0 < N; a0 += w) {"),
    # Algorithm 2: block end rounded on its own instead of floor((r+1)(m+n)/p)
    "alg2_block_end": ("int64_t i1 = (pe->r + 1) * mn / pe->p;",
                       "int64_t i1 = pe->r * mn / pe->p + mn / pe->p;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    c = tmp_path / "oracle_mutant.c"
    c.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", str(c),
                    "-o", str(lib)], check=True)
    env = dict(os.environ, ORACLE_MUTANT_LIB=str(lib))
    tests = [os.path.join(ROOT, "tests", t) for t in
             ("test_oracle_figures.py", "test_oracle_lemma.py", "test_oracle_kv.py")]
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            *tests], cwd=ROOT, env=env, capture_output=True, timeout=20)
        caught = r.returncode != 0
    except subprocess.TimeoutExpired:
        caught = True
    assert caught, f"mutant {name} passed every pin"
