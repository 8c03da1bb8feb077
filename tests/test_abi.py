"""CPU-side checks of the C-ABI boundary: the library builds for sm_103a, loads, exports every
entry point that include/dv.h declares, and the ctypes structs match the C layout."""
import os
import re
import subprocess
import tempfile
import ctypes as C

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dv.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dv_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("dv_create", "dv_destroy", "dv_render", "dv_render_backward", "dv_state_free", "dv_last_error"):
        assert n in names


def test_library_loads_and_exports_every_declared_symbol():
    import paper_2606_23031_gb300 as dv
    path = dv.build()
    lib = C.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"
    lib.dv_version.restype = C.c_char_p
    assert b"sm_103a" in lib.dv_version()


def test_library_is_built_for_sm103a_only():
    import paper_2606_23031_gb300 as dv
    assert dv.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_ctypes_structs_match_the_c_layout():
    import paper_2606_23031_gb300 as dv
    prog = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "dv.h"
    int main(void) {
      printf("%zu %zu %zu %zu\n", sizeof(dv_octree), sizeof(dv_pose), sizeof(dv_camera), sizeof(dv_opts));
      printf("%zu %zu %zu %zu\n", offsetof(dv_octree, center), offsetof(dv_octree, clip_half),
             offsetof(dv_octree, key), offsetof(dv_camera, cam_to_world));
      return 0;
    }
    """
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    sizes = [int(x) for x in out]
    assert sizes[0] == C.sizeof(dv.dv_octree)
    assert sizes[1] == C.sizeof(dv.dv_pose)
    assert sizes[2] == C.sizeof(dv.dv_camera)
    assert sizes[3] == C.sizeof(dv.dv_opts)
    assert sizes[4] == dv.dv_octree.center.offset
    assert sizes[5] == dv.dv_octree.clip_half.offset
    assert sizes[6] == dv.dv_octree.key.offset
    assert sizes[7] == dv.dv_camera.cam_to_world.offset


def test_no_cpu_fallback_when_library_missing(tmp_path):
    import paper_2606_23031_gb300 as dv
    saved = dv._lib
    dv._lib = None
    try:
        with pytest.raises(RuntimeError):
            dv.load(str(tmp_path / "nonexistent_libdv.so"))
    finally:
        dv._lib = saved
