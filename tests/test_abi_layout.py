"""The ctypes structures of the Python binding (Mesh, Opts, Stats) have the
layout of the C structures in include/stokes_mg.h: same field names in the
same order, same offsets, same total size.  A small C program compiled
against the header prints offsetof / sizeof; no GPU and no library call."""
import os
import shutil
import subprocess

import pytest

P = pytest.importorskip("paper_2407_07253_gb300._binding")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PAIRS = [("stokes_mesh", P.Mesh), ("stokes_mg_opts", P.Opts), ("stokes_mg_stats", P.Stats)]


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "stokes_mg.h"', "int main(void) {"]
    for cname, py in PAIRS:
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return {tuple(x.split()[:2]): int(x.split()[2]) for x in out.splitlines()}


def _c_fields(cname):
    """Field names of a struct in the header, in declaration order."""
    import re
    hdr = open(os.path.join(ROOT, "include", "stokes_mg.h")).read()
    body = dict((n, b) for b, n in re.findall(r"typedef struct \{(.*?)\}\s*(\w+);", hdr, re.S))[cname]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        decl = re.sub(r"\[[^\]]*\]", "", decl)
        head, *rest = decl.split(",")
        names.append(head.split()[-1].lstrip("*"))
        names += [x.strip().lstrip("*") for x in rest]
    return names


def test_ctypes_structures_match_the_header(tmp_path):
    import ctypes
    lay = _c_layout(tmp_path)
    for cname, py in PAIRS:
        assert [f for f, _ in py._fields_] == _c_fields(cname), cname
        assert ctypes.sizeof(py) == lay[(cname, "sizeof")], cname
        for field, _ in py._fields_:
            assert getattr(py, field).offset == lay[(cname, field)], (cname, field)
