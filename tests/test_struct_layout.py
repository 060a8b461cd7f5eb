"""The binding's ctypes mirrors of the structs in include/kkt.h have the C
layout: for every struct the Python side passes by pointer, a small C
program compiled here against the header prints sizeof and every field's
offsetof, and the ctypes Structure must give the same size, the same field
names in the same order and the same offsets.  A field added on one side
only would shift every later field (and has crashed a process before this
check existed)."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

import paper_2401_13926_b300 as K

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kkt.h")

MIRRORS = {
    "kkt_opts": K._Opts,
    "kkt_info": K._Info,
    "kkt_server_opts": K._ServerOpts,
    "kkt_step_result": K._StepResult,
    "kkt_server_info": K._ServerInfo,
    "kkt_host_stats": K._HostStats,
}


def _fields(struct):
    """Field names of a typedef'd struct in the header, in order."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    end = re.search(r"\}\s*" + struct + r"\s*;", text)
    assert end, struct
    start = text.rfind("typedef struct {", 0, end.start())
    body = text[start + len("typedef struct {"):end.start()]
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        decl = re.sub(r"\[[^\]]*\]", "", decl)           # arrays: the name before [..]
        for part in decl.split(","):
            names.append(re.findall(r"[A-Za-z_]\w*", part)[-1])
    return names


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("layout")
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "kkt.h"', "int main(void) {"]
    for s in MIRRORS:
        src.append(f'printf("{s} size %zu\\n", sizeof({s}));')
        for f in _fields(s):
            src.append(f'printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    src += ["return 0;", "}"]
    (d / "layout.c").write_text("\n".join(src))
    exe = d / "layout"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.dirname(HEADER), str(d / "layout.c"), "-o", str(exe)])
    out = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        s, f, v = line.split()
        out[(s, f)] = int(v)
    return out


@pytest.mark.parametrize("struct", sorted(MIRRORS))
def test_binding_struct_matches_header(c_layout, struct):
    py = MIRRORS[struct]
    names = _fields(struct)
    assert [f for f, _ in py._fields_] == names, (struct, [f for f, _ in py._fields_], names)
    assert C.sizeof(py) == c_layout[(struct, "size")], struct
    for f in names:
        assert getattr(py, f).offset == c_layout[(struct, f)], (struct, f)
