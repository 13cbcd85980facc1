"""The product path stands alone: the binding fails loudly when its CUDA
library is missing (there is no CPU fallback), and neither the package nor the
input generators touch the oracle, which is test infrastructure."""
import ast
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            names.add(node.module.split(".")[0])
    return names


def test_package_and_inputs_never_import_the_oracle():
    for d in ("paper_2005_05412_gb300", "workloads"):
        for dirpath, _, files in os.walk(os.path.join(ROOT, d)):
            for f in files:
                if f.endswith(".py"):
                    assert "oracle" not in _imports(os.path.join(dirpath, f)), os.path.join(dirpath, f)


def test_csrc_never_includes_the_oracle():
    csrc = os.path.join(ROOT, "paper_2005_05412_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f), errors="replace").read()
        assert "oracle" not in text.lower(), f


def test_missing_library_fails_loudly():
    code = ("import paper_2005_05412_gb300 as mbs\n"
            "mbs.LIB_PATH = '/nonexistent/libmbs.so'\n"
            "try:\n"
            "    mbs.mbs_abi_version()\n"
            "except RuntimeError as e:\n"
            "    print('raised', e)\n"
            "else:\n"
            "    print('no error')\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("raised") and "missing" in out.stdout, out.stdout
