"""Build liblb.so in-tree for sm_103a (nvcc for .cu, g++ for .cpp).

Objects and the library go to paper_1310_4218_gb300/_build/.  Translation
units compile in parallel; a unit is rebuilt when it or any header is newer
than its object.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "liblb.so")
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblb.so")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(obj, src, hdr_mtime):
    return (not os.path.exists(obj) or os.path.getmtime(obj) < os.path.getmtime(src)
            or os.path.getmtime(obj) < hdr_mtime)


def _compile(src, obj, verbose):
    if src.endswith(".cu"):
        cmd = [_nvcc()] + ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                                  "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC,
                                  "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I", INCLUDE,
               "-I", CSRC, "-I", "/usr/local/cuda/include", "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stderr


def build(force=False, verbose=False, jobs=None):
    """Compile every unit of the library for sm_103a and link liblb.so."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr = max([os.path.getmtime(h) for h in _headers()] + [0])
    todo, objs = [], []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        objs.append(o)
        if force or _stale(o, s, hdr):
            todo.append((s, o))
    jobs = jobs or max(1, min(len(todo), os.cpu_count() or 4))
    logs = {}
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            futs = {ex.submit(_compile, s, o, verbose): s for s, o in todo}
            for f in cf.as_completed(futs):
                logs[futs[f]] = f.result()
    if todo or not os.path.exists(LIB):
        tmp = LIB + ".%d.tmp" % os.getpid()
        cmd = [_nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        os.replace(tmp, LIB)
    if verbose:
        for s, l in logs.items():
            sys.stderr.write("== %s\n%s" % (os.path.basename(s), l))
    return LIB


def strip_comments(text):
    """C/C++/CUDA source text without its comments, trailing blanks and empty
    lines.  String and character literals are kept whole, so a "//" inside
    one is not taken for a comment."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":
            j = i + 1
            while j < n and text[j] != c and text[j] != "\n":
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    lines = (line.rstrip() for line in "".join(out).splitlines())
    return "\n".join(line for line in lines if line)


def source_hash(csrc=CSRC, include=INCLUDE):
    """Hash of every kernel and ABI source, comments ignored: ties a recorded
    profile to the exact code it measured.  An edit that touches only
    comments or blank lines leaves it unchanged; any other edit changes it."""
    import hashlib
    h = hashlib.sha256()
    # the ABI header first, then the kernel sources, each group by name: the
    # value does not depend on where the two directories sit
    files = (sorted(glob.glob(os.path.join(include, "*.h")))
             + sorted(glob.glob(os.path.join(csrc, "*"))))
    for f in files:
        if os.path.isfile(f):
            h.update(os.path.basename(f).encode())
            with open(f, encoding="utf-8") as fh:
                h.update(strip_comments(fh.read()).encode())
            h.update(b"\0")
    return h.hexdigest()[:16]


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
