"""The design notes, the README and the ncu summaries name files and tests
of this repository; every name they give must exist."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DOCS = ["DESIGN.md", "README.md"] + sorted(
    os.path.relpath(p, ROOT) for p in glob.glob(os.path.join(ROOT, "profiles", "*.md")))
PKG = "paper_1310_4218_gb300"

# a path in backticks: a known top-level folder or a package subfolder,
# then a file name with an extension
PATH = re.compile(r"`((?:tests|oracle|workloads|include|profiles|csrc|" + PKG +
                  r")/[\w./-]+\.\w+)(?:::(\w+))?`")
# a bare test file name, optionally with ::test_name
TEST = re.compile(r"`(test_\w+\.py)(?:::(\w+))?`")


def resolve(path):
    for cand in (path, os.path.join(PKG, path)):
        if os.path.exists(os.path.join(ROOT, cand)):
            return os.path.join(ROOT, cand)
    return None


def references():
    for doc in DOCS:
        with open(os.path.join(ROOT, doc), encoding="utf-8") as f:
            text = f.read()
        for m in PATH.finditer(text):
            yield doc, m.group(1), m.group(2)
        for m in TEST.finditer(text):
            yield doc, "tests/" + m.group(1), m.group(2)


def test_docs_cite_files_that_exist():
    missing = [(doc, path) for doc, path, _ in references() if resolve(path) is None]
    assert not missing, missing


def test_docs_cite_tests_that_exist():
    missing = []
    for doc, path, name in references():
        full = resolve(path)
        if name and full:
            with open(full, encoding="utf-8") as f:
                if not re.search(r"^def %s\(" % re.escape(name), f.read(), re.M):
                    missing.append((doc, path, name))
    assert not missing, missing


def test_docs_cite_test_functions_that_exist():
    """Bare test names (`test_...` without a file) name a test function
    defined somewhere under tests/."""
    src = ""
    for f in sorted(glob.glob(os.path.join(ROOT, "tests", "*.py"))):
        with open(f, encoding="utf-8") as fh:
            src += fh.read()
    missing = []
    for doc in DOCS:
        with open(os.path.join(ROOT, doc), encoding="utf-8") as f:
            for m in re.finditer(r"`(test_\w+)`", f.read()):
                if not re.search(r"^def %s\(" % m.group(1), src, re.M):
                    missing.append((doc, m.group(1)))
    assert not missing, missing


def test_the_check_finds_references():
    refs = list(references())
    assert len(refs) > 20
    assert any(name for _, _, name in refs)
