"""The ctypes mirrors of the C-ABI structs have the header's layout: a small
C program compiled here against include/idf.h prints sizeof and offsetof of
every field, and the binding's ctypes.Structure must agree field by field
(a field added to the header but not to the binding, or in another order,
fails here before any device call)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
INC = os.path.join(os.path.dirname(HERE), "include")

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")


def _c_layout(tmp_path, struct, fields):
    src = tmp_path / f"{struct}.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "idf.h"', "int main(void) {",
             f'  printf("size %zu\\n", sizeof({struct}));']
    for f in fields:
        lines.append(f'  printf("{f} %zu\\n", offsetof({struct}, {f}));')
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / struct
    subprocess.run(["gcc", "-std=c11", "-I", INC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return {out[i]: int(out[i + 1]) for i in range(0, len(out), 2)}


@pytest.mark.parametrize("name", ["idf_level_desc", "idf_model_stack", "idf_world_opts", "idf_volume_desc",
                                  "idf_region"])
def test_ctypes_structs_match_the_header(tmp_path, name):
    import paper_2512_08309_gb300 as idf
    cls = getattr(idf, name)
    fields = [f[0] for f in cls._fields_]
    lay = _c_layout(tmp_path, name, fields)
    assert lay["size"] == __import__("ctypes").sizeof(cls)
    for f in fields:
        assert lay[f] == getattr(cls, f).offset, (name, f)
