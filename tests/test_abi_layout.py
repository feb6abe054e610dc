"""The Python binding's view of the C ABI against the header itself.

lb.py restates the structs and enums of include/lb.h for ctypes.  A field
added to one side only, a wrong field type or a shifted enum value would
pass every call's marshalling silently and hand the library garbage.  Here a
small C program built from the header prints each struct's size, every
field's offset and every enum constant that lb.py names.  The numbers must
equal ctypes' own.  Needs gcc only: no GPU and no CUDA library.
"""
import ctypes
import os
import subprocess

import pytest

from paper_1310_4218_gb300 import lb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [lb.lb_grid_desc, lb.lb_vp, lb.lb_options, lb.lb_info]
ENUMS = sorted(n for n, v in vars(lb).items() if n.startswith("LB_") and isinstance(v, int))


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    d = tmp_path_factory.mktemp("abi_layout")
    body = []
    for s in STRUCTS:
        n = s.__name__
        body.append('printf("%s %%zu\\n", sizeof(%s));' % (n, n))
        for f in s._fields_:
            body.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (n, f[0], n, f[0]))
    for e in ENUMS:
        body.append('printf("%s %%ld\\n", (long)%s);' % (e, e))
    src = d / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"lb.h\"\n"
                   "int main(void) {\n    %s\n    return 0;\n}\n" % "\n    ".join(body))
    exe = d / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I",
                           os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)], text=True)
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


@pytest.mark.parametrize("struct", STRUCTS, ids=[s.__name__ for s in STRUCTS])
def test_struct_size_and_field_offsets_match_the_header(struct, c_layout):
    n = struct.__name__
    assert ctypes.sizeof(struct) == c_layout[n]
    for f in struct._fields_:
        assert getattr(struct, f[0]).offset == c_layout["%s.%s" % (n, f[0])], f[0]


def test_enum_constants_match_the_header(c_layout):
    assert len(ENUMS) >= 18
    for e in ENUMS:
        assert getattr(lb, e) == c_layout[e], e


def test_every_status_has_a_name():
    statuses = [e for e in ENUMS if e.startswith("LB_E") or e == "LB_OK"]
    assert sorted(lb.STATUS_NAMES.values()) == sorted(statuses)
    assert all(lb.STATUS_NAMES[getattr(lb, e)] == e for e in statuses)


def _c_prototypes():
    """name -> (return type, [parameter types]) of every lb_* function
    declared in include/lb.h (comments stripped, parameter names dropped)."""
    import re
    with open(os.path.join(ROOT, "include", "lb.h")) as f:
        text = re.sub(r"/\*.*?\*/", " ", f.read(), flags=re.S)
    protos = {}
    for m in re.finditer(r"^(lb_status|void|const char \*)\s*(lb_\w+)\s*\(([^)]*)\)\s*;",
                         text, flags=re.M):
        params = [" ".join(p.split()) for p in m.group(3).split(",")]
        params = [] if params == ["void"] else params
        # a parameter's type is everything but its name; pointers keep their '*'
        types = [re.sub(r"\s*\b\w+$", "", p) if not p.endswith("*") else p for p in params]
        protos[m.group(2)] = (m.group(1), types)
    return protos


def _c_class(t):
    t = t.replace("const ", "").strip()
    if "*" in t:
        return "pointer"
    return {"int32_t": "int32", "int64_t": "int64", "double": "double",
            "lb_status": "int32", "void": "void"}[t]


def _ctypes_class(t):
    if t is None:
        return "void"
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return "pointer"
    if t is ctypes.c_double:
        return "double"
    if issubclass(t, ctypes._SimpleCData) and t._type_ in "bBhHiIlLqQ":
        return "int%d" % (8 * ctypes.sizeof(t))
    return repr(t)


def test_binding_signatures_match_the_header_prototypes():
    """Every function lb.py binds has the header's arity, and each argument
    and return value the header's class (pointer, 32- or 64-bit integer,
    double); every function the header declares is bound."""
    protos = _c_prototypes()
    assert set(protos) == set(lb._SIG)
    for name, (ret, args) in lb._SIG.items():
        c_ret, c_args = protos[name]
        assert _ctypes_class(ret) == _c_class(c_ret), name
        assert len(args) == len(c_args), name
        for i, (a, c) in enumerate(zip(args, c_args)):
            assert _ctypes_class(a) == _c_class(c), "%s argument %d (%s)" % (name, i, c)


def test_every_entry_point_has_a_wrapper_of_the_same_name():
    """The Python binding offers each C entry point under its own name."""
    missing = [n for n in _c_prototypes() if not callable(getattr(lb, n, None))]
    assert missing == []
