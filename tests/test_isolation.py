"""The oracle stays test infrastructure: the product package and the shared input
generators never import it, the oracle never imports the product, and the product path
raises, rather than falling back to any CPU code, when its native library is missing."""
import ast
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(folder):
    """(file, top-level module) for every import statement in the .py files under folder."""
    out = []
    for dirpath, _, files in os.walk(os.path.join(ROOT, folder)):
        for fn in files:
            if not fn.endswith(".py"):
                continue
            path = os.path.join(dirpath, fn)
            for node in ast.walk(ast.parse(open(path).read())):
                if isinstance(node, ast.Import):
                    out += [(path, a.name.split(".")[0]) for a in node.names]
                elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
                    out.append((path, node.module.split(".")[0]))
    return out


def test_product_and_generators_never_import_the_oracle():
    for folder in ("paper_2411_14977_gb300", "workloads"):
        bad = [p for p, mod in _imports(folder) if mod == "oracle"]
        assert not bad, bad


def test_oracle_never_imports_the_product():
    bad = [p for p, mod in _imports("oracle") if mod in ("paper_2411_14977_gb300", "torch")]
    assert not bad, bad


def test_missing_library_raises():
    code = ("import paper_2411_14977_gb300.pmg as pmg\n"
            "pmg._lib = None\n"
            "pmg._build.LIB = '/nonexistent/libpmg.so'\n"
            "try:\n"
            "    pmg.load()\n"
            "except RuntimeError as e:\n"
            "    print('raised', e)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.startswith("raised") and "missing" in r.stdout
