"""The oracle and the CUDA path share no code, and the product never runs the oracle.

The oracle is test infrastructure: only the tests, the smoke check and the
benchmark's CPU-baseline and reference legs may load it.  The library package
must neither import it nor include anything from it, and the oracle must
neither import the package nor include its headers, so that agreement between
the two is evidence rather than shared arithmetic.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2408_09066_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for dirpath, dirnames, files in os.walk(top):
        dirnames[:] = [d for d in dirnames if not d.startswith(("_build", "__pycache__"))]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name.split(".")[0]
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            yield node.module.split(".")[0]


def test_package_never_imports_the_oracle():
    for path in _files(PKG, (".py",)):
        assert "oracle" not in set(_imports(path)), path


def test_cuda_sources_include_nothing_from_the_oracle():
    for path in _files(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".h", ".cpp")):
        for inc in re.findall(r'#include\s+[<"]([^>"]+)[>"]', open(path).read()):
            assert "oracle" not in inc, (path, inc)


def test_oracle_never_imports_or_includes_the_package():
    for path in _files(ORACLE, (".py",)):
        assert "paper_2408_09066_gb300" not in set(_imports(path)), path
    src = open(os.path.join(ORACLE, "oracle.c")).read()
    for inc in re.findall(r'#include\s+[<"]([^>"]+)[>"]', src):
        assert inc in ("math.h", "stdint.h", "stdlib.h", "string.h", "omp.h"), inc


def _oracle_imports_outside(fn, allowed_if):
    """Imports of the oracle in function `fn` that are not inside an `if` whose
    test mentions `allowed_if`."""
    parents = {}
    for node in ast.walk(fn):
        for child in ast.iter_child_nodes(node):
            parents[child] = node
    bad = []
    for node in ast.walk(fn):
        mods = ([a.name for a in node.names] if isinstance(node, ast.Import) else
                [node.module] if isinstance(node, ast.ImportFrom) and node.module else [])
        if not any(m.split(".")[0] == "oracle" for m in mods):
            continue
        p, guarded = parents.get(node), False
        while p is not None and p is not fn:
            if isinstance(p, ast.If) and allowed_if in ast.unparse(p.test):
                guarded = True
                break
            p = parents.get(p)
        if not guarded:
            bad.append(node.lineno)
    return bad


def test_only_the_allowed_entry_points_load_the_oracle():
    """Outside tests/ and oracle/ itself, only __graft_entry__.py and bench.py
    import the oracle; bench.py only in its CPU-baseline and reference legs
    (their functions, or a branch taken unless --no-cpu-baseline is given)."""
    allowed_bench = {"cpu_baseline", "run_reference", "run_reference_batch", "_oracle_setup",
                     "calibrate_oracle", "oracle_step_time", "batch_oracle_plan",
                     "batch_oracle_time", "oracle_full_step", "sample_fraction", "oracle_legs"}
    for path in _files(ROOT, (".py",)):
        rel = os.path.relpath(path, ROOT)
        if rel.startswith(("tests" + os.sep, "oracle" + os.sep, "_work" + os.sep,
                           "baseline" + os.sep)):
            continue
        if "oracle" not in set(_imports(path)):
            continue
        assert rel in ("__graft_entry__.py", "bench.py"), rel
        if rel == "bench.py":
            tree = ast.parse(open(path).read())
            for fn in tree.body:
                if isinstance(fn, ast.FunctionDef) and fn.name not in allowed_bench:
                    assert not _oracle_imports_outside(fn, "no_cpu_baseline"), fn.name
            top = {a.name for n in tree.body if isinstance(n, ast.Import) for a in n.names}
            assert "oracle" not in top, "bench.py imports the oracle at module level"


def test_committed_code_does_not_use_working_files():
    needle = "_work" + "/"
    for path in _files(ROOT, (".py", ".cu", ".cuh", ".h", ".c")):
        rel = os.path.relpath(path, ROOT)
        if rel.startswith(("_work" + os.sep, "baseline" + os.sep)):
            continue
        assert needle not in open(path, errors="replace").read(), rel
