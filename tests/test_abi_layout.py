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


def _prototypes():
    """name -> (return type, [parameter types]) for every function the
    header declares."""
    import re
    hdr = open(os.path.join(ROOT, "include", "stokes_mg.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    out = {}
    for ret, name, params in re.findall(r"((?:const\s+)?\w+\s*\**)\s*\b(stokes_\w+)\s*\(([^)]*)\)\s*;", hdr):
        ps = [" ".join(p.split()) for p in params.split(",")]
        if ps == ["void"]:
            ps = []
        types = []
        for p in ps:
            p = re.sub(r"\[[^\]]*\]", "*", p)              # array parameters decay to pointers
            stars = p.count("*")
            words = [w for w in p.replace("*", " ").split() if w not in ("const",)]
            base = " ".join(words[:-1]) if len(words) > 1 else words[0]
            types.append("ptr" if stars or base == "stokes_mg_t" else base)   # the handle is a pointer
        out[name] = (ret.replace(" ", ""), types)
    return out


def test_binding_signatures_match_the_header():
    """Every function the binding wraps takes as many arguments as its
    prototype, of the same kind (pointer, int, long long, double), and
    returns what the prototype returns."""
    import ctypes
    lib = pytest.importorskip("paper_2407_07253_gb300").lib()
    kind = {ctypes.c_int: "int", ctypes.c_longlong: "long long", ctypes.c_double: "double",
            ctypes.c_ulonglong: "unsigned long long"}
    protos = _prototypes()
    wrapped = 0
    for name, (ret, types) in protos.items():
        f = getattr(lib, name)
        if f.argtypes is None:
            continue
        wrapped += 1
        got = []
        for t in f.argtypes:
            if t in kind:
                got.append(kind[t])
            else:
                assert t is ctypes.c_void_p or t is ctypes.c_char_p or issubclass(t, ctypes._Pointer), (name, t)
                got.append("ptr")
        assert got == types, (name, got, types)
        if ret == "void":
            assert f.restype is None, name
        elif ret.endswith("*"):
            assert f.restype in (ctypes.c_char_p, ctypes.c_void_p), name
        else:
            assert kind.get(f.restype) == ret, (name, f.restype, ret)
    assert wrapped >= 30, wrapped


def test_default_options_are_the_documented_ones():
    """stokes_mg_default_opts gives what the header states: GRADUAL,
    nu_p = nu_h = n_V = 1, 15 Arnoldi steps, seed 0, interval [0.1, 1.1],
    FP64, restart 30, maxit 1000, use_graph 1, batch_tune 1, and zero for
    everything else (no lambda_max overrides, host_only 0, the saddle-block
    patch solver)."""
    o = P.default_opts()
    assert (o.hierarchy, o.nu_p, o.nu_h, o.n_V, o.eig_steps, o.eig_seed) == (P.HIER_GRADUAL, 1, 1, 1, 15, 0)
    assert (o.cheb_lo, o.cheb_hi, o.precision, o.restart, o.maxit) == (0.1, 1.1, P.FP64, 30, 1000)
    assert (o.use_graph, o.batch_tune, o.host_only, o.prof_mask, o.patch_solver, o.n_schedule) == (1, 1, 0, 0, 0, 0)
    assert list(o.lmax_override) == [0.0] * 16 and list(o.schedule) == [0] * 8
