"""The C ABI library loads and exports every function include/guidefill.h declares (no GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "guidefill.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(gf_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1611_05319_gb300 import build
    return build.build()


def test_header_declares_the_api():
    names = _declared()
    for n in ["gf_create", "gf_destroy", "gf_fill", "gf_fill_batched", "gf_guidance_from_splines",
              "gf_status_string"]:
        assert n in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = C.CDLL(built_lib)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_1611_05319_gb300 import _lib
    assert sorted(_lib.EXPORTS) == _declared()


def test_status_strings_and_argument_errors_without_gpu(built_lib):
    lib = C.CDLL(built_lib)
    lib.gf_status_string.restype = C.c_char_p
    assert lib.gf_status_string(0) == b"ok"
    assert b"invalid" in lib.gf_status_string(-1)
    lib.gf_create.argtypes = [C.POINTER(C.c_void_p), C.c_int]
    lib.gf_create.restype = C.c_int
    # a NULL output pointer is an argument error detected before any CUDA call
    assert lib.gf_create(None, 0) == -1
    # calls on a NULL context are argument errors, nothing is launched
    lib.gf_fill.restype = C.c_int
    assert lib.gf_fill(None, None, None, None, None) == -1
    lib.gf_fill_batched.restype = C.c_int
    assert lib.gf_fill_batched(None, 1, None, None, None, None) == -1
    lib.gf_guidance_batched.restype = C.c_int
    assert lib.gf_guidance_batched(None, 1, None, C.c_float(3.0), None) == -1
    lib.gf_detect_splines_batched.restype = C.c_int
    assert lib.gf_detect_splines_batched(None, 1, None, None, None) == -1
    lib.gf_fill_batched_splines.restype = C.c_int
    assert lib.gf_fill_batched_splines(None, 1, None, None, C.c_float(3.0), None, None, None, None, None) == -1


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the ABI structs have the sizes the C compiler gives the header's."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "%s"\nint main(void){printf("%%zu %%zu %%zu %%zu",'
                   'sizeof(gf_frame),sizeof(gf_params),sizeof(gf_spline_frame),sizeof(gf_stats));'
                   'printf(" %%zu %%zu %%zu",sizeof(gf_detect_params),sizeof(gf_detect_frame),'
                   'offsetof(gf_detect_frame,result));return 0;}' % HEADER)
    exe = tmp_path / "sz"
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    sizes = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    from paper_1611_05319_gb300 import _lib
    assert sizes == [C.sizeof(_lib.Frame), C.sizeof(_lib.Params), C.sizeof(_lib.SplineFrame), _lib.STATS_BYTES,
                     C.sizeof(_lib.DetectParams), C.sizeof(_lib.DetectFrame), _lib.DetectFrame.result.offset]


def test_host_batch_pointer_tables():
    """HostBatch holds the frames' sizes, data pointers and spline counts that
    fill_batched_host passes to gf_fill_batched_host, and keeps the arrays alive."""
    import numpy as np
    import paper_1611_05319_gb300 as gf
    rgba = [np.zeros((8 + i, 16, 4), np.float32) for i in range(3)]
    labels = [np.zeros(a.shape[:2], np.uint8) for a in rgba]
    shells = [np.zeros(a.shape[:2], np.int32) for a in rgba]
    guide = [None, np.zeros((9, 16, 2), np.float32), None]
    splines = [(np.array([0, 3, 5]), np.zeros((5, 2), np.float64)), None, (np.array([0, 2]), np.ones((2, 2)))]
    b = gf.HostBatch(rgba, labels, guide, rgba, shells, splines=splines)
    assert b.n == 3
    assert list(b.Hs) == [8, 9, 10] and list(b.Ws) == [16, 16, 16]
    assert [b.p_rgba[i] for i in range(3)] == [a.ctypes.data for a in rgba]
    assert [b.p_out_rgba[i] for i in range(3)] == [a.ctypes.data for a in rgba]
    assert [b.p_labels[i] for i in range(3)] == [a.ctypes.data for a in labels]
    assert [b.p_out_shell[i] for i in range(3)] == [a.ctypes.data for a in shells]
    assert b.p_guide[0] is None and b.p_guide[1] == guide[1].ctypes.data and b.p_guide[2] is None
    assert list(b.ns) == [2, 0, 1] and list(b.npts) == [5, 0, 2]
    assert b.p_offs[1] is None and b.p_pts[1] is None
    # the converted spline arrays (int32 offsets, float32 points) are the ones pointed at
    offs, pts = b._keep[3], b._keep[4]
    assert offs[0].dtype == np.int32 and pts[2].dtype == np.float32
    assert b.p_offs[0] == offs[0].ctypes.data and b.p_pts[2] == pts[2].ctypes.data
