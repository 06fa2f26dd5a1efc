"""The oracle stays test infrastructure: the product package and the shared input
generators never import it, the oracle never imports the product, bench.py reaches it
only from its CPU-baseline and reference legs, and the product path raises, rather than
falling back to any CPU code, when its native library is missing."""
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


def test_bench_runs_the_oracle_only_in_its_cpu_baseline_and_reference_legs():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    importers, callers = set(), set()
    for fn in ast.walk(tree):
        if not isinstance(fn, ast.FunctionDef):
            continue
        for node in ast.walk(fn):
            if isinstance(node, ast.ImportFrom) and node.module and node.module.split(".")[0] == "oracle":
                importers.add(fn.name)
            if isinstance(node, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in node.names):
                importers.add(fn.name)
            if isinstance(node, ast.Call) and getattr(node.func, "id", None) == "oracle_solve_timed":
                callers.add(fn.name)
    assert importers <= {"oracle_solve_timed", "cpu_baseline_paper", "cpu_baseline_bar"}, importers
    # oracle_one_core_child: the one-core timing of the CPU baseline (a child process)
    assert callers <= {"cpu_baseline_entry", "oracle_one_core_child", "run_reference"}, callers
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    assert not any(getattr(n, "module", None) == "oracle" or
                   any(a.name.split(".")[0] == "oracle" for a in getattr(n, "names", [])) for n in top)
