"""The product path (the package and its CUDA library) never uses the oracle: the oracle is
test infrastructure, reachable only from tests/, the smoke check and the bench's baseline."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2609_16408_gb300")


def test_package_sources_do_not_import_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, re.M), f
                assert "orc_" not in txt, f  # no oracle C symbols


def test_importing_the_package_loads_no_oracle_module():
    code = ("import sys; sys.path.insert(0, %r); import paper_2609_16408_gb300, "
            "paper_2609_16408_gb300.shard; print(any(m == 'oracle' or m.startswith('oracle.') "
            "for m in sys.modules))" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == "False"


def test_library_does_not_link_the_oracle():
    import paper_2609_16408_gb300 as R
    so = R.load()._name
    nm = subprocess.run(["nm", "-D", so], capture_output=True, text=True)
    if nm.returncode != 0:
        return
    assert "orc_" not in nm.stdout


def test_missing_cuda_library_fails_loudly(tmp_path):
    """Without a built library and without a CUDA compiler the binding raises instead of
    falling back to anything else."""
    code = (
        "import os, sys; sys.path.insert(0, %r)\n"
        "import paper_2609_16408_gb300 as R\n"
        "R._BUILD = %r; R._SO = os.path.join(R._BUILD, 'librpa.so'); R._LIB = None\n"
        "os.environ['NVCC'] = '/nonexistent/nvcc'\n"
        "try:\n"
        "    R.load()\n"
        "    print('loaded')\n"
        "except Exception as e:\n"
        "    print('raised', type(e).__name__)\n" % (ROOT, str(tmp_path)))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert out.stdout.strip().startswith("raised"), out.stdout + out.stderr[-2000:]
