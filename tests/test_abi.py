"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/fga.h declares
(no GPU needed: nothing is computed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fga.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fga_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1810_06760_gb300 import build
    return build.build()


def test_header_declares_the_paths_entry_points():
    names = _declared()
    for n in ("fga_decompose", "fga_propagate", "fga_reconstruct", "fga_solve", "fga_model_create", "fga_bin"):
        assert n in names


def test_library_exports_every_declared_symbol(built_lib):
    L = ctypes.CDLL(built_lib)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_1810_06760_gb300 import fga
    assert sorted(fga.EXPORTED) == _declared()


def test_version_and_error_text_without_gpu(built_lib):
    L = ctypes.CDLL(built_lib)
    assert L.fga_version() >= 10000
    L.fga_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    buf = ctypes.create_string_buffer(64)
    L.fga_last_error(buf, 64)   # empty message, no crash
    # argument validation happens before any CUDA call
    L.fga_propagate.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p]
    assert L.fga_propagate(None, None, 0.1, 1, None) == 1
    L.fga_last_error(buf, 64)
    assert b"fga_propagate" in buf.value


_STRUCTS = {"ModelDesc": "fga_model_desc", "InitDesc": "fga_init_desc", "PointForce": "fga_point_force",
            "Profile": "fga_profile_t", "ServerDesc": "fga_server_desc", "RequestInfo": "fga_request_info",
            "ServerStats": "fga_server_stats_t", "Lattice": "fga_lattice", "SolveDesc": "fga_solve_desc"}


def test_binding_structs_match_the_header(tmp_path):
    """Every descriptor the Python binding mirrors with ctypes has the header's size and field offsets (a
    program compiled against include/fga.h prints them), so a field added to the header and not to the
    binding, or in another order, fails here rather than as garbage on the GPU."""
    import subprocess
    from paper_1810_06760_gb300 import fga
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fga.h"', "int main(void) {"]
    want = []
    for py, c in _STRUCTS.items():
        cls = getattr(fga, py)
        lines.append(f'    printf("%zu\\n", sizeof({c}));')
        want.append(ctypes.sizeof(cls))
        for name, _ in cls._fields_:
            lines.append(f'    printf("%zu\\n", offsetof({c}, {name}));')
            want.append(getattr(cls, name).offset)
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == want
