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


def _run_c_pins(tmp_path, text):
    """Compile `text` as the oracle library, load it in a child pytest run of
    the C-backed pins; returns its exit code (None on timeout)."""
    c = tmp_path / "oracle_mutant.c"
    c.write_text(text)
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", str(c),
                    "-o", str(lib)], check=True)
    env = dict(os.environ, ORACLE_MUTANT_LIB=str(lib))
    tests = [os.path.join(ROOT, "tests", t) for t in
             ("test_oracle_figures.py", "test_oracle_lemma.py", "test_oracle_kv.py")]
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            *tests], cwd=ROOT, env=env, capture_output=True, timeout=20)
        return r.returncode
    except subprocess.TimeoutExpired:
        return None


def test_c_pins_without_mutation_pass(tmp_path):
    """Control: the unchanged source, built and loaded the same way, passes
    the pins, so a failing mutant run means the pins caught the mistake."""
    assert _run_c_pins(tmp_path, open(SRC).read()) == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    rc = _run_c_pins(tmp_path, src.replace(old, new))
    assert rc != 0, f"mutant {name} passed every pin"


# Mistakes in the oracle's key-order map (Python, oracle/__init__.py): the
# child process redefines order_key from a mutated copy of its source in the
# oracle module (merge_in_order calls it through the module) and runs the
# order pins.
ORDER_MUTANTS = {
    # negative floats: only the sign bit flipped (sign-magnitude order kept)
    "float_negatives_sign_only": ("u = np.where(neg, ~u, u | sign).astype(ut)",
                                  "u = np.where(neg, u ^ sign, u | sign).astype(ut)"),
    # signed integers compared as unsigned
    "signed_no_offset": ("    elif base[0] == \"i\":\n        u ^= sign\n",
                         "    elif base[0] == \"i\":\n        pass\n"),
    # signed pairs: the minor half's sign bit not flipped
    "pair_minor_sign": ("u ^= ut((1 << 63) | (1 << 31))", "u ^= ut(1 << 63)"),
    # descending order ignored
    "desc_dropped": ("    if mod == \"desc\":\n        u = ~u\n",
                     "    if mod == \"desc\":\n        pass\n"),
}

_ORDER_CHILD = r"""
import inspect, sys
sys.path.insert(0, {root!r})
import oracle
import pytest
src = inspect.getsource(oracle.order_key)
exec(src.replace({old!r}, {new!r}), oracle.__dict__)
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider",
                      {test!r}]))
"""


def _run_order_child(old, new):
    code = _ORDER_CHILD.format(root=ROOT, old=old, new=new,
                               test=os.path.join(ROOT, "tests", "test_oracle_order.py"))
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True,
                           timeout=60)
        return r.returncode
    except subprocess.TimeoutExpired:
        return None


def test_order_child_without_mutation_passes():
    """Control: the same child with nothing changed passes the order pins, so
    a failing mutant run means the pins caught the mistake."""
    assert _run_order_child("", "") == 0


@pytest.mark.parametrize("name", sorted(ORDER_MUTANTS))
def test_order_mutant_is_caught(name):
    import inspect
    import oracle
    old, new = ORDER_MUTANTS[name]
    assert inspect.getsource(oracle.order_key).count(old) == 1, \
        f"mutation site for {name} not unique"
    rc = _run_order_child(old, new)
    assert rc != 0, f"order mutant {name} passed every pin"
