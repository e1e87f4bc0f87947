"""Every struct of the C ABI has the same size and member offsets in include/symgpu.h (compiled here with gcc)
as in the ctypes mirror the Python binding passes across the boundary (no GPU needed)."""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "symgpu.h")

# header struct -> name of its ctypes mirror in the binding
MIRRORS = {
    "sym_profile_entry": "ProfileEntry",
    "sym_csr_upper": "CsrUpper",
    "sym_csr_full": "CsrFull",
    "sym_csr_batch": "CsrBatch",
    "sym_tile_cfg": "TileCfg",
    "sym_tensor_info_t": "TensorInfo",
    "sym_mttkrp_cfg": "MttkrpCfg",
    "sym_ttm_cfg": "TtmCfg",
    "sym_ptensor_info_t": "PTensorInfo",
    "sym_request": "Request",
    "sym_result": "Result",
    "sym_server_cfg": "ServerCfg",
    "sym_server_stats": "ServerStats",
    "sym_devloop_cfg": "DevLoopCfg",
    "sym_devloop_stats": "DevLoopStats",
}


def header_structs():
    """{struct name: [member names in declaration order]} of every `typedef struct { ... } name;`."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"typedef struct\s*\{(.*?)\}\s*(\w+);", text, flags=re.S):
        members = []
        for decl in m.group(1).split(";"):
            decl = decl.strip()
            if not decl:
                continue
            parts = [p.strip() for p in decl.split(",")]
            first = re.sub(r"\[.*?\]", "", parts[0])
            members.append(re.findall(r"[A-Za-z_]\w*", first)[-1])
            for p in parts[1:]:
                members.append(re.findall(r"[A-Za-z_]\w*", re.sub(r"\[.*?\]", "", p))[-1])
        out[m.group(2)] = members
    return out


@pytest.fixture(scope="module")
def c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = header_structs()
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "symgpu.h"', "int main(void) {"]
    for s, members in structs.items():
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for mname in members:
            lines.append(f'  printf("{s} {mname} %zu\\n", offsetof({s}, {mname}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        text = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    size, offsets = {}, {}
    for ln in text.splitlines():
        s, what, v = ln.split()
        if what == "size":
            size[s] = int(v)
        else:
            offsets.setdefault(s, []).append((what, int(v)))
    return structs, size, offsets


def test_every_header_struct_has_a_mirror():
    assert set(header_structs()) == set(MIRRORS)


@pytest.mark.parametrize("cname", sorted(MIRRORS))
def test_struct_layout_matches_binding(cname, c_layout):
    import ctypes

    import paper_2406_09266_gb300 as sg
    structs, size, offsets = c_layout
    py = getattr(sg, MIRRORS[cname])
    assert ctypes.sizeof(py) == size[cname], (cname, ctypes.sizeof(py), size[cname])
    fields = [f[0] for f in py._fields_]
    assert len(fields) == len(offsets[cname]), (cname, fields, offsets[cname])
    for f, (cm, off) in zip(fields, offsets[cname]):
        assert getattr(py, f).offset == off, (cname, f, cm, getattr(py, f).offset, off)
