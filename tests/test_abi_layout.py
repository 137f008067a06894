"""The ctypes structures of the binding against the C ABI's own layout (no GPU needed).

A small C program, compiled here with the host compiler against include/*.h, prints
sizeof and offsetof for every field of every structure that crosses the boundary; the
binding's ctypes definitions must agree byte for byte, or the library would read and
write the wrong fields.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1811_03559_gb300 import serve, spike

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = [("spike_info", spike.SpikeInfo), ("spike_options", spike.SpikeOptions),
           ("spike_tune_result", spike.TuneResult), ("spike_server_config", serve.ServerConfig),
           ("spike_server_stats", serve.ServerStats)]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "spike.h"', '#include "spike_serve.h"',
             "int main(void) {"]
    for cname, cls in STRUCTS:
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, field, cname, field))
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.check_call([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True)
    table = {}
    for line in out.splitlines():
        cname, field, value = line.split()
        table[(cname, field)] = int(value)
    return table


@pytest.mark.parametrize("cname,cls", STRUCTS, ids=[c for c, _ in STRUCTS])
def test_ctypes_layout_matches_header(c_layout, cname, cls):
    assert ctypes.sizeof(cls) == c_layout[(cname, "sizeof")], cname
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == c_layout[(cname, field)], (cname, field)


def test_numerics_bits_match_header():
    hdr = open(os.path.join(ROOT, "include", "spike.h")).read()
    assert "#define SPIKE_NUMERICS_NAN_PIVOT %d" % spike.NUMERICS_NAN_PIVOT in hdr
    assert "#define SPIKE_NUMERICS_SINGULAR_INTERFACE %d" % spike.NUMERICS_SINGULAR_INTERFACE in hdr
    assert "#define SPIKE_PIVOT_R13 %g" % spike.PIVOT_R13 in hdr
