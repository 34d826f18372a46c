"""The product path has no CPU fallback: without the CUDA library every call
fails loudly, and host tensors are refused instead of being merged on the
CPU.  Runs in child interpreters so the library state of this session is
untouched."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _child(code):
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True,
                          text=True, timeout=120)


def test_missing_library_raises():
    r = _child(
        "import sys\n"
        "from paper_1303_4312_gb300 import _lib\n"
        "_lib.LIB_PATH = '/nonexistent/libcorank.so'\n"
        "import paper_1303_4312_gb300 as cr\n"
        "try:\n"
        "    cr.tile_size('i32')\n"
        "except RuntimeError as e:\n"
        "    print('raised:', e)\n"
        "    sys.exit(0)\n"
        "sys.exit(3)\n")
    assert r.returncode == 0, r.stdout + r.stderr
    assert "libcorank.so not found" in r.stdout


def test_host_tensors_are_refused():
    r = _child(
        "import sys, torch\n"
        "import paper_1303_4312_gb300 as cr\n"
        "A = torch.arange(0, 100, 2, dtype=torch.int32)\n"
        "B = torch.arange(1, 100, 2, dtype=torch.int32)\n"
        "try:\n"
        "    cr.merge(A, B)\n"
        "except ValueError as e:\n"
        "    print('refused:', e)\n"
        "    sys.exit(0)\n"
        "sys.exit(3)\n")
    assert r.returncode == 0, r.stdout + r.stderr
    assert "CUDA tensors" in r.stdout
