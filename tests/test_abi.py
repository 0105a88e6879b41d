"""The C ABI library builds, loads and exports every entry point include/nbody.h declares, and the
binding names the same set.  No compute call is made (these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2203_08966_gb300 as nb
from paper_2203_08966_gb300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"\bnbody_status\s+(nbody_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib_path():
    return build_lib.build()


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("nbody_create", "nbody_build_tree", "nbody_forces", "nbody_step"):
        assert name in d


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (nbody_\w+)", out))
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_library_loads_and_binding_covers_exports(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name)
    assert set(nb.EXPORTS) == _declared()


def test_struct_layouts_match_header():
    # nbody_params: 4 doubles, int32, uint32; nbody_tree_record: u64, 2 x i32, 2 x i64
    assert ctypes.sizeof(nb.Params) == 40
    assert ctypes.sizeof(nb.TreeRecord) == 32


def test_null_context_is_rejected_without_gpu(lib_path):
    lib = nb.load_library(lib_path)
    assert lib.nbody_destroy(None) == 1
    assert lib.nbody_sync(None) == 1
    assert lib.nbody_set_walk_limits(None, 0, 0, 0) == 1
    assert lib.nbody_create(None, 10, None, None) == 1


def test_forest_create_rejects_bad_offsets_without_gpu(lib_path):
    """nbody_forest_create validates its host arguments before touching the device."""
    lib = nb.load_library(lib_path)
    p = nb.Params(1.0, 0.01, 0.5, 1e-3, nb.FP32, 0)
    h = ctypes.c_void_p()

    def create(off, S=None):
        off = np.ascontiguousarray(off, dtype=np.int64)
        S = len(off) - 1 if S is None else S
        return lib.nbody_forest_create(ctypes.byref(h), S, off.ctypes.data_as(ctypes.c_void_p),
                                       ctypes.byref(p), None)

    assert create([1, 5]) == 1            # offsets[0] != 0
    assert create([0, 5, 3]) == 1         # decreasing
    assert create([0, 0, 0]) == 1         # no bodies at all
    assert create([0, 4], S=0) == 1       # no systems
    bad = nb.Params(1.0, -1.0, 0.5, 1e-3, nb.FP32, 0)
    off = np.array([0, 4], dtype=np.int64)
    assert lib.nbody_forest_create(ctypes.byref(h), 1, off.ctypes.data_as(ctypes.c_void_p),
                                   ctypes.byref(bad), None) == 1   # eps < 0
    assert lib.nbody_forest_create(None, 1, off.ctypes.data_as(ctypes.c_void_p),
                                   ctypes.byref(p), None) == 1


def test_group_mac_flag_rejected_for_fp64_without_gpu(lib_path):
    lib = nb.load_library(lib_path)
    h = ctypes.c_void_p()
    bad = nb.Params(1.0, 0.01, 0.5, 1e-3, nb.FP64, nb.FLAG_GROUP_MAC)
    assert lib.nbody_create(ctypes.byref(h), 10, ctypes.byref(bad), None) == 1
    unknown = nb.Params(1.0, 0.01, 0.5, 1e-3, nb.FP32, 256)
    assert lib.nbody_create(ctypes.byref(h), 10, ctypes.byref(unknown), None) == 1
    cells64 = nb.Params(1.0, 0.01, 0.5, 1e-3, nb.FP64, nb.FLAG_CELL_GROUPS)
    assert lib.nbody_create(ctypes.byref(h), 10, ctypes.byref(cells64), None) == 1


def test_header_is_plain_c_and_a_c_program_links(lib_path, tmp_path):
    """The boundary is a C ABI: the header compiles as strict C99, and a C program that takes
    the address of every entry point links against the library (nothing is run)."""
    names = sorted(_declared())
    src = tmp_path / "abi.c"
    src.write_text("#include \"nbody.h\"\n"
                   "#include <stdio.h>\n"
                   "typedef void (*fn_t)(void);\n"
                   "int main(void) {\n"
                   "    fn_t fns[] = {" + ", ".join(f"(fn_t)&{n}" for n in names) + "};\n"
                   "    nbody_params p = {1.0, 0.01, 0.5, 1e-3, NBODY_FP32_KAHAN, 0u};\n"
                   "    printf(\"%d %d %f\\n\", (int)(sizeof fns / sizeof fns[0]), fns[0] != 0,\n"
                   "           p.theta);\n"
                   "    return 0;\n"
                   "}\n")
    inc = os.path.join(ROOT, "include")
    libdir = os.path.dirname(lib_path)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc,
                        str(src), "-o", str(tmp_path / "abi"), "-L", libdir,
                        "-l:" + os.path.basename(lib_path), "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
