"""The ctypes mirror of the C ABI (paper_2502_03091_gb300/mg.py) against
include/mg.h (no GPU): every enum value the binding uses, and every struct's
field names, order and byte layout -- the offsets and sizes a C compiler
gives for the header (gcc, compiled here) must equal ctypes' own.  A mismatch
would pass wrong values through the ABI without any error."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2502_03091_gb300 import mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mg.h")

MIRRORS = {"mg_problem": mg._Problem, "mg_coarse_problem": mg._CoarseProblem,
           "mg_hierarchy": mg._Hierarchy, "mg_timing_entry": mg._TimingEntry,
           "mg_level_desc": mg._LevelDesc}
SCALARS = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
           "double": ctypes.c_double, "size_t": ctypes.c_size_t, "char": ctypes.c_char}


def _header_code():
    with open(HEADER) as fh:
        return re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)


def _enums():
    return {n: int(v) for n, v in re.findall(r"\b(MG_[A-Z0-9_]+)\s*=\s*(\d+)", _header_code())}


def _structs():
    """{struct name: [(field, C type, is pointer, array length or None)]}"""
    out = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(\w+);", _header_code(), re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"(?:const )?(\w+)\s*(\*?)\s*(.*)", decl)
            ctype, star, names = m.group(1), m.group(2), m.group(3)
            for nm in names.split(","):
                nm = nm.strip()
                ptr = bool(star) or nm.startswith("*")
                nm = nm.lstrip("* ")
                arr = re.match(r"(\w+)\s*\[(\d+)\]", nm)
                fields.append((arr.group(1), ctype, ptr, int(arr.group(2))) if arr
                              else (nm, ctype, ptr, None))
        out[name] = fields
    return out


def test_enum_values_match_the_header():
    en = _enums()
    used = {n: getattr(mg, n) for n in dir(mg) if n.startswith("MG_")}
    assert used, "the binding defines no MG_ constants"
    for n, v in used.items():
        assert en[n] == v, n
    statuses = {v: n for n, v in en.items() if n == "MG_OK" or n.startswith("MG_ERR_")}
    assert mg.STATUS_NAMES == statuses
    for n in ("MG_PREC_FP32", "MG_PREC_MIXED", "MG_PREC_MIXED_FP16", "MG_CALL_SMOOTH",
              "MG_CALL_TRUNCATE", "MG_CALL_COARSEN"):
        assert n in used


def test_struct_fields_match_the_header():
    st = _structs()
    assert set(MIRRORS) <= set(st)
    for cname, mirror in MIRRORS.items():
        fields = st[cname]
        assert [f[0] for f in fields] == [f[0] for f in mirror._fields_], cname
        for (name, ctype, ptr, n), (_, pytype) in zip(fields, mirror._fields_):
            if ptr:
                assert pytype is ctypes.c_void_p, (cname, name)
            elif ctype in MIRRORS:
                assert pytype is MIRRORS[ctype], (cname, name)
            elif n is not None:
                assert pytype._type_ is SCALARS[ctype] and pytype._length_ == n, (cname, name)
            else:
                assert pytype is SCALARS[ctype], (cname, name)


def test_struct_layout_matches_a_c_compiler(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    st = _structs()
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mg.h"', "int main(void) {"]
    for cname in MIRRORS:
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for name, *_ in st[cname]:
            lines.append(f'  printf("{cname} {name} %zu\\n", offsetof({cname}, {name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True,
                               text=True).stdout.splitlines():
        cname, field, val = line.split()
        got[(cname, field)] = int(val)
    for cname, mirror in MIRRORS.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(mirror), cname
        for name, _ in mirror._fields_:
            assert got[(cname, name)] == getattr(mirror, name).offset, (cname, name)
