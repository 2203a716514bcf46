"""The ctypes marshalling in binding.py against the C declarations of include/algmortar.h:
same fields in the same order, and the same sizes and offsets as a C compiler lays them
out (gcc on this host, the ABI the library is built for)."""
import os
import re
import shutil
import subprocess
import tempfile

import ctypes as C
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "algmortar.h")


def header_structs():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", txt, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            m = re.match(r"(.*?)(\w+)\s*(\[\s*\d+\s*\])?$", decl)
            fields.append(m.group(2))
        out[name] = fields
    return out


def binding_structs():
    from paper_2607_22905_b300 import binding as B
    return {"algmortar_csr": B.Csr, "algmortar_opts": B.Opts, "algmortar_stats": B.Stats, "algmortar_info": B.Info}


def test_field_names_and_order():
    hs = header_structs()
    for cname, cls in binding_structs().items():
        assert [f for f, _ in cls._fields_] == hs[cname], cname


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_sizes_and_offsets_match_c():
    structs = binding_structs()
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "abi.c"), os.path.join(d, "abi")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-std=c99", src, "-o", exe], check=True)
        got = dict(l.split() for l in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n") if l)
    for cname, cls in structs.items():
        assert int(got[cname]) == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, f"{cname}.{f}"
