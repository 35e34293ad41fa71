"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, and exports every entry point that include/tsdf.h declares;
the binding's structures match the header's layout."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2311_00626_gb300 as gt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "tsdf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^tsdf_status\s+(\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_binding_names():
    assert _header_functions() == sorted(gt.EXPORTED_SYMBOLS)


def test_library_exports_every_declared_symbol():
    path = gt.build_library()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [f for f in _header_functions() if f not in exported]
    assert not missing, missing
    lib = gt.lib()
    for f in _header_functions():
        assert getattr(lib, f) is not None


def test_struct_layouts_match_header():
    # sizes from the C layout rules of the header's structs
    assert ctypes.sizeof(gt.Pinhole) == 24
    assert ctypes.sizeof(gt.Lidar) == 28
    assert ctypes.sizeof(gt.MapOpts) == 64
    assert ctypes.sizeof(gt.EsdfOpts) == 12
    assert ctypes.sizeof(gt.FrameDesc) == 4 + 4 + 24 + 28 + 4 + 8 + 128 + 8


def test_header_compiles_as_c_and_layouts_agree(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text('#include "tsdf.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(tsdf_pinhole),'
                    ' sizeof(tsdf_lidar), sizeof(tsdf_map_opts), sizeof(tsdf_frame_desc),'
                    ' offsetof(tsdf_frame_desc, depth_dev), offsetof(tsdf_frame_desc, color_dev),'
                    ' sizeof(tsdf_esdf_opts)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(prog), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals == [ctypes.sizeof(gt.Pinhole), ctypes.sizeof(gt.Lidar), ctypes.sizeof(gt.MapOpts),
                    ctypes.sizeof(gt.FrameDesc), gt.FrameDesc.depth_dev.offset,
                    gt.FrameDesc.color_dev.offset, ctypes.sizeof(gt.EsdfOpts)]


def test_pose_argument_marshalling():
    """Poses reach the C calls as 16 row-major doubles: a contiguous float64
    array is passed as its own memory, anything else as a copy with the
    same values."""
    import numpy as np
    T = np.arange(16, dtype=np.float64).reshape(4, 4)
    assert gt._pose_arg(T) == T.ctypes.data
    for other in (T.tolist(), T.astype(np.float32), np.asfortranarray(T), T[:, :]):
        arg = gt._pose_arg(other)
        vals = list(arg) if not isinstance(arg, int) else \
            list((ctypes.c_double * 16).from_address(arg))
        assert vals == T.reshape(16).tolist()


def test_header_constants_match_binding(tmp_path):
    """The sizes a caller of integrate_depth_static allocates and decodes
    with: counter words, key packing and the work-list limit, as the C
    compiler sees them in the header."""
    prog = tmp_path / "consts.c"
    prog.write_text('#include "tsdf.h"\n#include <stdio.h>\n'
                    'int main(void){printf("%d %d %d %d\\n", TSDF_NUM_COUNTERS, TSDF_KEY_BITS,'
                    ' TSDF_KEY_BIAS, TSDF_STATIC_MAX_BLOCKS); return 0;}\n')
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(prog), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals == [gt.NUM_COUNTERS, gt.KEY_BITS, gt.KEY_BIAS, gt.STATIC_MAX_BLOCKS]
