"""The oracle and the CUDA path share nothing and never call each other: no
Python module of the package imports the oracle (or the reverse), no source
of either side includes a file of the other, and only the seeded input
generators (synth/) serve both.  The product path has no CPU fallback: the
binding raises when its library is missing (tests/test_abi.py checks that)."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1707_00385_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def imported_modules(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            if node.level == 0 and node.module:
                names.add(node.module.split(".")[0])
    return names


def included_files(path):
    return re.findall(r'#\s*include\s*[<"]([^">]+)[">]', open(path).read())


def test_package_never_imports_the_oracle():
    files = glob.glob(os.path.join(PKG, "*.py"))
    assert files
    for f in files:
        assert "oracle" not in imported_modules(f), f


def test_oracle_never_imports_the_package():
    files = glob.glob(os.path.join(ORACLE, "*.py"))
    assert files
    for f in files:
        mods = imported_modules(f)
        assert not any(m.startswith("paper_1707_00385_gb300") or m == "bench" for m in mods), f


def test_bench_runs_the_oracle_only_in_its_cpu_leg():
    """bench.py imports the oracle only inside the functions of its
    cpu_baseline leg (the timed host baseline, which --impl reference also
    runs, and the FP64 answers the precision columns are measured against),
    never at module level or on the device path."""
    path = os.path.join(ROOT, "bench.py")
    tree = ast.parse(open(path).read(), filename=path)
    allowed = {"cpu_baseline", "oracle_answers"}
    found = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in node.names):
                    found.add(fn.name)
                if isinstance(node, ast.ImportFrom) and node.module and node.module.split(".")[0] == "oracle":
                    found.add(fn.name)
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    assert "oracle" not in {m for n in top for m in ([a.name.split(".")[0] for a in n.names]
                                                     if isinstance(n, ast.Import) else [n.module.split(".")[0]])}
    assert found == allowed, found


def test_sources_include_nothing_of_the_other_side():
    cuda = glob.glob(os.path.join(PKG, "csrc", "*"))
    assert cuda
    for f in cuda:
        for inc in included_files(f):
            assert "oracle" not in inc, (f, inc)
    for f in glob.glob(os.path.join(ORACLE, "*.c")) + glob.glob(os.path.join(ORACLE, "*.h")):
        for inc in included_files(f):
            assert "pc_" not in inc and "pcurv" not in inc and "csrc" not in inc, (f, inc)


def test_input_generators_hold_no_method_arithmetic():
    """synth/ renders scenes and noise; it imports neither side."""
    for f in glob.glob(os.path.join(ROOT, "synth", "*.py")):
        mods = imported_modules(f)
        assert "oracle" not in mods and not any(m.startswith("paper_1707_00385_gb300") for m in mods), f
