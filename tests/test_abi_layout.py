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
