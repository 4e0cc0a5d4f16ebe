"""The C-ABI library builds, loads and exports every function include/hmg.h declares
(no GPU needed: only the functions that do not touch CUDA are called)."""
import ctypes
import os
import subprocess

import pytest

from paper_2210_11797_gb300 import build as B
from paper_2210_11797_gb300 import hmg


@pytest.fixture(scope="module")
def libpath():
    if not os.path.exists(B.library_path()):
        B.build()
    return B.library_path()


def test_header_declares_the_boundary():
    names = hmg.header_symbols()
    for required in ("hmg_create", "hmg_set_mesh", "hmg_set_coefficients", "hmg_assemble_trace",
                     "hmg_trace_rhs", "hmg_solve", "hmg_solve_host", "hmg_reconstruct", "hmg_destroy",
                     "hmg_apply_trace", "hmg_precond_apply"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in hmg.header_symbols() if n not in exported]
    assert not missing, missing
    # and the binding knows every one of them
    assert set(hmg.header_symbols()) == set(hmg._SIGS)


def test_library_loads_and_reports_defaults(libpath):
    L = hmg.lib()
    o = hmg.Options()
    assert L.hmg_default_options(ctypes.byref(o)) == 0
    assert (o.omega, o.n_pre, o.n_post, o.mg_omega, o.mg_npre, o.mg_npost) == (0.6, 1, 2, 0.9, 1, 2)
    assert o.tol == 1e-6 and o.precond == hmg.PRECOND["nonnested"]
    assert L.hmg_status_string(0) == b"ok"
    assert L.hmg_status_string(4) == b"not converged"
    assert L.hmg_create(None, None, None) == 1          # null output pointer -> INVALID_ARG
    assert L.hmg_assemble_trace(None) == 1


def test_struct_layouts_match_header():
    # sizes follow from the C declarations in include/hmg.h (x86-64 and aarch64 LP64 ABIs)
    assert ctypes.sizeof(hmg.MeshLevel) == 4 * 4 + 8 + 6 * 8
    assert ctypes.sizeof(hmg.Background) == 3 * 8
    assert ctypes.sizeof(hmg.Scalars) == 6 * 8 + 8 + 8 + 8
    assert ctypes.sizeof(hmg.SolveStats) == 4 + 4 + 3 * 8 + 8 + hmg.MAX_HISTORY * 8 + 8 * 8 + 8 * 4 + 8
    assert ctypes.sizeof(hmg.Options) == 136


def test_struct_offsets_match_the_c_compiler(tmp_path):
    """Every field offset of the ctypes mirrors equals the C compiler's offsetof."""
    structs = {"hmg_mesh_level": hmg.MeshLevel, "hmg_background": hmg.Background,
               "hmg_scalars": hmg.Scalars, "hmg_options": hmg.Options, "hmg_solve_stats": hmg.SolveStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hmg.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", B.INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        cname, field, value = line.split()
        py = structs[cname]
        got = ctypes.sizeof(py) if field == "sizeof" else getattr(py, field).offset
        assert got == int(value), (cname, field, got, value)
