"""The ctypes mirrors of the C ABI's structs (paper_2310_06650_gb300/qg.py) against include/qg.h:
a small C program built with the host compiler prints sizeof and every field's offsetof, and each
must match the ctypes layout, so that a field added on one side only fails here, on the CPU."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load_binding_structs():
    """The binding's Structure classes, rebuilt from the _fields_ lists of qg.py (read as source, so
    that no library needs to be built for this test)."""
    import ast
    tree = ast.parse(open(os.path.join(ROOT, "paper_2310_06650_gb300", "qg.py")).read())
    env = {"C": ctypes, "_I32P": ctypes.POINTER(ctypes.c_int32), "_F64P": ctypes.POINTER(ctypes.c_double)}
    out = {}
    for node in tree.body:
        if isinstance(node, ast.ClassDef) and node.name in ("qg_network", "qg_horizon", "qg_contingencies",
                                                             "qg_options"):
            for stmt in node.body:
                if isinstance(stmt, ast.Assign) and stmt.targets[0].id == "_fields_":
                    fields = eval(compile(ast.Expression(stmt.value), "qg.py", "eval"), env)
                    out[node.name] = type(node.name, (ctypes.Structure,), {"_fields_": fields})
    assert len(out) == 4, sorted(out)
    return out


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = _load_binding_structs()
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "qg.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, key, value = line.split()
        layout[(name, key)] = int(value)
    return structs, layout


def test_struct_sizes_and_offsets_match(c_layout):
    structs, layout = c_layout
    for name, cls in structs.items():
        assert ctypes.sizeof(cls) == layout[(name, "size")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == layout[(name, field)], (name, field)


def _header_prototypes():
    """{name: (return type, argument count)} of every qg_* function the header declares."""
    import re
    text = open(os.path.join(ROOT, "include", "qg.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    out = {}
    for m in re.finditer(r"([A-Za-z_][\w\s\*]*?)\b(qg_\w+)\s*\(([^;{}]*?)\)\s*;", text):
        ret, name, args = " ".join(m.group(1).split()), m.group(2), m.group(3).strip()
        if ret.startswith("typedef"):
            continue
        n = 0 if args in ("", "void") else len(args.split(","))
        out[name] = (ret, n)
    return out


def _binding_signatures():
    """{name: (restype, argument count)} of the binding's ctypes table, read from qg.py's source."""
    import ast
    tree = ast.parse(open(os.path.join(ROOT, "paper_2310_06650_gb300", "qg.py")).read())
    load = next(n for n in tree.body if isinstance(n, ast.FunctionDef) and n.name == "_load")
    sig = next(s for s in load.body if isinstance(s, ast.Assign) and getattr(s.targets[0], "id", "") == "sig")
    env = {"C": ctypes, "vp": ctypes.c_void_p, "_I32P": ctypes.POINTER(ctypes.c_int32),
           "_F64P": ctypes.POINTER(ctypes.c_double), **_load_binding_structs()}
    table = eval(compile(ast.Expression(sig.value), "qg.py", "eval"), env)
    return {name: (res, len(args)) for name, (res, args) in table.items()}


RET = {"void": None, "int": 4, "int32_t": 4, "int64_t": 8, "const char *": "str"}


def _ret_kind(res):
    if res is None:
        return None
    if res is ctypes.c_char_p:
        return "str"
    return ctypes.sizeof(res)


def test_every_prototype_has_a_matching_ctypes_signature():
    protos, sigs = _header_prototypes(), _binding_signatures()
    assert set(protos) == set(sigs), (sorted(set(protos) - set(sigs)), sorted(set(sigs) - set(protos)))
    for name, (ret, n) in protos.items():
        res, m = sigs[name]
        assert n == m, (name, n, m)
        assert ret in RET, (name, ret)
        assert RET[ret] == _ret_kind(res), (name, ret, res)


@pytest.mark.parametrize("lang", ["c99", "c++11"])
def test_header_compiles_as_strict_c_and_cxx(tmp_path, lang):
    cc = shutil.which("gcc" if lang == "c99" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / ("h.c" if lang == "c99" else "h.cpp")
    src.write_text('#include "qg.h"\nint main(void) { return qg_version() < 0; }\n')
    subprocess.run([cc, f"-std={lang}", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-I",
                    os.path.join(ROOT, "include"), str(src)], check=True)
