"""CPU-side check that the ctypes structures of the Python binding lay out
their fields exactly as the C header does: a small C program compiled
against include/simdsearch.h prints sizeof and every field's offset, and
each must equal the ctypes Structure's.  A field added on one side only
would make the library write past the binding's buffer."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"

# C struct name -> the binding class that mirrors it
STRUCTS = {
    "ss_devstat": "DevStat",
    "ss_interp_opts": "InterpOpts",
    "ss_plan_opts": "PlanOpts",
    "ss_plan_info": "PlanInfo",
}


def c_layout(tmp_path, cstruct, fields):
    src = ["#include <stddef.h>", "#include <stdio.h>", '#include "simdsearch.h"', "int main(void) {",
           '  printf("%%zu\\n", sizeof(%s));' % cstruct]
    for f in fields:
        src.append('  printf("%%zu\\n", offsetof(%s, %s));' % (cstruct, f))
    src += ["  return 0;", "}"]
    c = tmp_path / ("%s.c" % cstruct)
    exe = tmp_path / cstruct
    c.write_text("\n".join(src) + "\n")
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC, str(c), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(v) for v in out[1:]]


@pytest.mark.skipif(shutil.which("gcc") is None or not os.path.isdir(CUDA_INC), reason="gcc or CUDA headers missing")
@pytest.mark.parametrize("cstruct", sorted(STRUCTS))
def test_ctypes_structures_match_the_header(tmp_path, cstruct):
    import paper_2112_03229_gb300 as ss
    cls = getattr(ss, STRUCTS[cstruct])
    fields = [f[0] for f in cls._fields_]
    size, offsets = c_layout(tmp_path, cstruct, fields)
    assert ctypes.sizeof(cls) == size, (cstruct, ctypes.sizeof(cls), size)
    for name, off in zip(fields, offsets):
        assert getattr(cls, name).offset == off, (cstruct, name, getattr(cls, name).offset, off)
