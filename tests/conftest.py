import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA path)")
    config.addinivalue_line("markers", "slow: full-size cases (minutes)")
    config.addinivalue_line(
        "markers", "host_only: argument checks that pass fake device addresses; they only run "
                   "where no GPU is present, so a check that failed to refuse a call can never "
                   "launch a kernel on them")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:
        have_gpu = False
    if have_gpu:
        skip = pytest.mark.skip(reason="host-only check (fake device addresses) on a GPU machine")
        for it in items:
            if "host_only" in it.keywords:
                it.add_marker(skip)
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def read_golden(name):
    """Parse a whitespace-separated golden file; '#' starts a comment line."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


# A mutated copy of the oracle (see test_oracle_mutants.py) is swapped in when
# this variable names its compiled library; the pins must then fail.
_MUTANT = os.environ.get("ORACLE_MUTANT_LIB")
if _MUTANT:
    import oracle as _oracle
    _oracle.build = lambda force=False: _MUTANT
