"""The binding's ctypes structures against the C header's struct layout (CPU).

The Python binding passes tnlm_geometry_desc, tnlm_params and tnlm_report
by pointer; a field added to the header but not to the binding (or in a
different order) would make the library read the wrong bytes without any
error.  A small C program compiled against include/tnlm.h prints the size
and every field's offset of the three structs; they must equal the ctypes
layout field by field, and the header's field names (parsed from the
text) must be the binding's, in order.
"""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

import paper_1009_1351_gb300 as tn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "tnlm_geometry_desc": tn.GeometryDesc,
    "tnlm_params": tn.ParamsC,
    "tnlm_report": tn.ReportC,
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tnlm.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        s, f, v = line.split()
        table[(s, f)] = int(v)
    return table


@pytest.mark.parametrize("cname", list(STRUCTS))
def test_ctypes_struct_matches_the_header(c_layout, cname):
    py = STRUCTS[cname]
    assert ctypes.sizeof(py) == c_layout[(cname, "size")]
    for fname, _ in py._fields_:
        assert getattr(py, fname).offset == c_layout[(cname, fname)], fname


def header_fields(cname):
    """Field names of 'typedef struct { ... } cname;' in include/tnlm.h, in
    order (comments removed; one or more declarators per declaration)."""
    text = open(os.path.join(ROOT, "include", "tnlm.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    m = re.search(r"typedef\s+struct\s*\{([^}]*)\}\s*" + cname + r"\s*;", text)
    assert m, cname
    names = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        head, _, rest = decl.partition(",")
        first = re.findall(r"[A-Za-z_]\w*", head)[-1]
        names.append(first)
        names += [re.findall(r"[A-Za-z_]\w*", r)[-1] for r in rest.split(",") if r.strip()]
    return names


@pytest.mark.parametrize("cname", list(STRUCTS))
def test_binding_has_every_header_field_in_order(cname):
    assert [f for f, _ in STRUCTS[cname]._fields_] == header_fields(cname)


# ------------------------------------------------------------ prototypes
_SCALARS = {"int": ctypes.c_int, "unsigned": ctypes.c_uint, "unsigned int": ctypes.c_uint,
            "long": ctypes.c_long, "long long": ctypes.c_longlong, "double": ctypes.c_double,
            "float": ctypes.c_float, "size_t": ctypes.c_size_t}


def header_prototypes():
    """{name: (return type, [parameter types])} of every tnlm_* function the
    headers declare (comments removed, parameter names dropped)."""
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    out = {}
    for m in re.finditer(r"([A-Za-z_][\w\s\*]*?)\b(tnlm_[a-z_0-9]+)\s*\(([^;{}]*?)\)\s*;", src):
        ret, name, args = " ".join(m.group(1).split()), m.group(2), " ".join(m.group(3).split())
        params = [] if args in ("", "void") else [a.strip() for a in args.split(",")]
        out[name] = (ret.replace("extern", "").strip(), params)
    return out


def c_param_kind(decl):
    """'pointer', or the ctypes class of a scalar parameter declaration."""
    if "*" in decl:
        return "pointer"
    words = decl.replace("const", " ").split()
    base = " ".join(words[:-1])          # drop the parameter name
    return _SCALARS.get(base, base)


def ctypes_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return "pointer"
    return t


@pytest.fixture(scope="module")
def lib():
    from paper_1009_1351_gb300 import build as tnbuild
    tnbuild.build()
    return tn.load_library()


_RETURNS = {"tnlm_status": ctypes.c_int, "int": ctypes.c_int, "void": None,
            "const char*": ctypes.c_char_p, "long long": ctypes.c_longlong}


def test_argtypes_follow_the_prototypes(lib):
    """Every function the binding gives argtypes takes as many arguments as
    its prototype, pointers where the prototype has pointers and the same
    scalar types elsewhere; functions without argtypes take no argument; and
    every return type is the one ctypes reads."""
    protos = header_prototypes()
    assert set(protos) == set(tn.EXPORTED)
    for name, (ret, params) in protos.items():
        assert getattr(lib, name).restype is _RETURNS[" ".join(ret.replace("*", " * ").split())
                                                      .replace(" *", "*")], name
        at = getattr(lib, name).argtypes
        if at is None:
            assert params == [], name
            continue
        assert len(at) == len(params), name
        for t, decl in zip(at, params):
            assert ctypes_kind(t) == c_param_kind(decl), (name, decl)
