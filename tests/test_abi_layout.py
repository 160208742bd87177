"""The ctypes mirrors of the C structs in include/iod.h match the C layout field by field:
a C program compiled against the header prints every field's offset and each struct's
size, and the binding's ctypes definitions must give the same numbers (a mismatch would
let the library write past a Python-owned buffer)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _mirrors():
    from paper_2207_13175_gb300 import _native as N
    return {"iod_options": N.Options, "iod_result_t": N.Result, "iod_request": N.Request,
            "iod_batch_stats": N.BatchStats}


def test_ctypes_layouts_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = _mirrors()
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "iod.h"', "int main(void) {"]
    for cname, S in mirrors.items():
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, *_ in S._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c_side = {}
    for line in out:
        if line.strip():
            cname, field, value = line.split()
            c_side[(cname, field)] = int(value)
    for cname, S in mirrors.items():
        assert c_side[(cname, "sizeof")] == ctypes.sizeof(S), cname
        for fname, *_ in S._fields_:
            assert c_side[(cname, fname)] == getattr(S, fname).offset, (cname, fname)
