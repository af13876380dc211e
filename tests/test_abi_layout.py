"""The ctypes mirrors of the C-ABI structs (``paper_2603_21444_gb300._abi``)
against the header itself: a small C program compiled with the host's gcc
prints sizeof and offsetof of every mirrored struct and field, which must
equal ctypes' sizes and offsets (a field added to one side only, a changed
type or a padding difference shows here, without a GPU)."""
import ctypes
import shutil
import subprocess
from pathlib import Path

import pytest

from paper_2603_21444_gb300 import _abi

ROOT = Path(__file__).resolve().parents[1]
MIRRORS = {
    "spgemm_csr_in": _abi.CsrIn,
    "spgemm_csr_out": _abi.CsrOut,
    "spgemm_tune": _abi.Tune,
    "spgemm_mcl_params": _abi.MclParams,
}


def test_struct_layouts_match_header(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc on this host")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "trident_spgemm.h"', "int main(void) {"]
    for cname, cls in MIRRORS.items():
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", str(ROOT / "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, cls in MIRRORS.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)

