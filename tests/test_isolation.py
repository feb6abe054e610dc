"""The oracle and the CUDA path stay apart, and the product never routes
through the oracle.

Checked statically on the source text, so it runs anywhere:
- nothing in the package, the input generators or the kernel sources
  imports or includes the oracle;
- the oracle imports nothing of the package and includes none of its headers;
- the two share only the seeded input generators (workloads/), which import
  neither;
- in bench.py only the CPU-baseline function imports the oracle;
- nothing committed imports from the scratch folder.
"""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_1310_4218_gb300"


def py_files(*parts):
    return sorted(glob.glob(os.path.join(ROOT, *parts, "*.py")))


def imported_modules(path):
    tree = ast.parse(open(path, encoding="utf-8").read(), filename=path)
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods.update(a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            if node.level == 0 and node.module:
                mods.add(node.module)
    return mods


def top(mod):
    return mod.split(".")[0]


def c_includes(path):
    return re.findall(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', open(path, encoding="utf-8").read(),
                      flags=re.M)


def test_product_never_imports_the_oracle():
    files = py_files(PKG) + py_files("workloads")
    assert files
    for f in files:
        mods = {top(m) for m in imported_modules(f)}
        assert "oracle" not in mods, f
        assert "_work" not in mods, f


def test_oracle_never_imports_the_product():
    for f in py_files("oracle"):
        mods = {top(m) for m in imported_modules(f)}
        assert PKG not in mods and "bench" not in mods and "_work" not in mods, f


def test_input_generators_import_neither_side():
    for f in py_files("workloads"):
        mods = {top(m) for m in imported_modules(f)}
        assert not mods & {"oracle", PKG, "torch"}, (f, mods)


def test_kernel_and_oracle_sources_share_no_header():
    kernel_dir = os.path.join(ROOT, PKG, "csrc")
    kernel_headers = {os.path.basename(h) for h in glob.glob(os.path.join(kernel_dir, "*.h*"))}
    kernel_headers |= {os.path.basename(h) for h in glob.glob(os.path.join(ROOT, "include", "*.h"))}
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.c")) + glob.glob(os.path.join(ROOT, "oracle", "*.h")):
        for inc in c_includes(f):
            assert os.path.basename(inc) not in kernel_headers, (f, inc)
            assert "csrc" not in inc and "include/" not in inc, (f, inc)
    for f in glob.glob(os.path.join(kernel_dir, "*")):
        for inc in c_includes(f):
            assert "oracle" not in inc, (f, inc)


def test_bench_imports_the_oracle_only_in_its_cpu_baseline():
    path = os.path.join(ROOT, "bench.py")
    tree = ast.parse(open(path, encoding="utf-8").read())
    assert "oracle" not in {top(m) for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))
                            for m in imported_modules_of(n)}
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, (ast.Import, ast.ImportFrom)) and \
                        "oracle" in {top(m) for m in imported_modules_of(node)}:
                    users.add(fn.name)
    assert users == {"cpu_oracle_rate"}


def imported_modules_of(node):
    if isinstance(node, ast.Import):
        return [a.name for a in node.names]
    return [node.module] if node.level == 0 and node.module else []


def test_nothing_committed_reads_the_scratch_folder():
    files = (py_files(PKG) + py_files("workloads") + py_files("oracle") + py_files("tests")
             + [os.path.join(ROOT, "bench.py"), os.path.join(ROOT, "__graft_entry__.py")])
    for f in files:
        if os.path.basename(f) == os.path.basename(__file__):
            continue
        text = open(f, encoding="utf-8").read()
        assert not re.search(r"(?<![A-Za-z0-9_])_work(?![A-Za-z0-9_])", text), f
