"""The ctypes mirrors of the C-ABI structs in the Python binding have the C layout:
a small C program that includes include/ieti.h (compiled with the host compiler)
prints sizeof and offsetof of every field, which must equal ctypes.sizeof and the
ctypes field offsets.  Catches a binding that drifts from the header."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _binding():
    # the struct definitions only; loading the library is not needed for layouts,
    # but the module loads it at import, so skip where it is not built
    try:
        from paper_2510_23446_gb300 import ieti
    except Exception as e:   # noqa: BLE001  (a missing build is a skip here, not a failure)
        pytest.skip(f"binding not importable: {e}")
    return ieti


def test_struct_layouts_match_the_header():
    cc = shutil.which("cc") or shutil.which("gcc")
    if not cc:
        pytest.skip("no C compiler")
    ieti = _binding()
    structs = [ieti.ieti_problem, ieti.ieti_options, ieti.ieti_coil, ieti.ieti_stats, ieti.ieti_kernel_stat,
               ieti.ieti_info]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ieti.h"', 'int main(void) {']
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in st._fields_:
            lines.append(f'  printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ['  return 0;', '}']
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "layout.c")
        exe = os.path.join(tmp, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True,
                       capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            parts = line.split()
            got[(parts[0], parts[1])] = int(parts[2])
    for st in structs:
        name = st.__name__
        assert got[(name, "size")] == C.sizeof(st), name
        for fname, _ in st._fields_:
            assert got[(name, fname)] == getattr(st, fname).offset, (name, fname)
