"""The ctypes binding against include/ttnn.h, on the host: every structure
the binding declares has the C compiler's field offsets and size, and every
declared entry point has the header's parameter count and parameter kinds
(pointer, 32/64-bit integer, double, size).  A mismatch here would pass
wrong arguments through the C ABI without any error."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

from paper_2412_06111_gb300 import _sigs as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ttnn.h")

STRUCTS = {"ttnn_tree": S.TtnnTree, "ttnn_opts": S.TtnnOpts, "ttnn_node_info": S.TtnnNodeInfo,
           "ttnn_server_opts": S.TtnnServerOpts, "ttnn_server_report": S.TtnnServerReport}


def _declarations():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    text = re.sub(r"#[^\n]*", " ", text)
    text = re.sub(r"\s+", " ", text)
    out = {}
    for m in re.finditer(r"(ttnn_status|void|const char\s*\*)\s+(\w+)\s*\(([^)]*)\)\s*;", text):
        params = [p.strip() for p in m.group(3).split(",") if p.strip() and p.strip() != "void"]
        out[m.group(2)] = (m.group(1).replace(" ", ""), params)
    return out


def _kind_c(param):
    p = param.replace("const", " ")
    if "*" in p or re.search(r"\bttnn_(plan|state|server)_t\b", p):
        return "ptr"
    # size_t is an unsigned 64-bit integer on the LP64 hosts this library builds for
    for t, k in (("int32_t", "i32"), ("uint32_t", "u32"), ("int64_t", "i64"), ("uint64_t", "u64"),
                 ("double", "f64"), ("size_t", "u64"), ("ttnn_status", "i32")):
        if re.search(r"\b%s\b" % t, p):
            return k
    raise AssertionError("unclassified parameter: " + param)


def _kind_py(t):
    if t in (C.c_void_p, C.c_char_p) or (isinstance(t, type) and issubclass(t, C._Pointer)):
        return "ptr"
    if t is C.c_double:
        return "f64"
    signed = t(-1).value == -1
    return ("i" if signed else "u") + str(8 * C.sizeof(t))


def test_every_bound_function_matches_its_declaration():
    decl = _declarations()
    # the binding covers exactly the declared entry points
    assert set(decl) == set(S.SIGS), sorted(set(decl) ^ set(S.SIGS))
    for name, (res, args) in S.SIGS.items():
        assert name in decl, name
        ret, params = decl[name]
        assert len(params) == len(args), (name, params)
        assert [_kind_c(p) for p in params] == [_kind_py(a) for a in args], name
        if ret == "void":
            assert res is None, name
        elif ret == "ttnn_status":
            assert res is C.c_int32, name
        else:
            assert res is C.c_char_p, name


def test_structure_layouts_match_the_c_compiler(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ttnn.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for cname, py in STRUCTS.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
