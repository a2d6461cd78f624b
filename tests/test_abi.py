"""The C ABI library builds for sm_103a, loads without a GPU, and exports every
function include/nnm.h declares with the struct layouts the binding assumes."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nnm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nnm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1402_3789_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert set(names) == {"nnm_create", "nnm_nearest", "nnm_cluster", "nnm_get_tree", "nnm_get_stats",
                          "nnm_last_error", "nnm_status_string", "nnm_destroy", "nnm_restrict_static",
                          "nnm_create_batched", "nnm_cluster_host", "nnm_set_wait_limit"}
    for n in names:
        assert hasattr(lib, n), n
    from paper_1402_3789_gb300 import nnm
    assert set(nnm.EXPORTS) == set(names)


def test_status_strings_without_gpu(lib):
    lib.nnm_status_string.restype = ctypes.c_char_p
    assert lib.nnm_status_string(0) == b"NNM_OK"
    assert lib.nnm_status_string(5) == b"NNM_ETIMEOUT"


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    P = ctypes.c_void_p
    lib.nnm_create.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int, ctypes.c_int, P, P, ctypes.POINTER(P)]
    out = P(1)
    dummy = P(16)
    assert lib.nnm_create(dummy, 0, 8, 0, 0, None, None, ctypes.byref(out)) == 1      # N < 1
    assert out.value is None
    assert lib.nnm_create(dummy, 10, 33, 0, 0, None, None, ctypes.byref(out)) == 1    # d > 32
    assert lib.nnm_create(dummy, 10, 0, 0, 0, None, None, ctypes.byref(out)) == 1     # d < 1
    assert lib.nnm_create(None, 10, 4, 0, 0, None, None, ctypes.byref(out)) == 1      # null X
    assert lib.nnm_create(dummy, 1 << 31, 4, 0, 0, None, None, ctypes.byref(out)) == 1
    assert lib.nnm_create(dummy, 10, 4, 3, 0, None, None, ctypes.byref(out)) == 6     # metric
    assert lib.nnm_create(dummy, 10, 4, 1, 1, None, None, ctypes.byref(out)) == 6     # Manhattan on tensor cores
    assert lib.nnm_create(dummy, 10, 4, 2, 3, None, None, ctypes.byref(out)) == 6     # Chebyshev on tensor cores
    assert lib.nnm_create(dummy, 10, 4, 0, 7, None, None, ctypes.byref(out)) == 6     # precision
    assert lib.nnm_create(dummy, 10, 31, 0, 3, None, None, ctypes.byref(out)) == 6    # split form: d <= 30


def test_struct_layouts_match_the_header(tmp_path):
    from paper_1402_3789_gb300 import nnm
    prog = tmp_path / "sizes.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "nnm.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(nnm_merge), sizeof(nnm_edge),'
                    ' sizeof(nnm_restrictions), sizeof(nnm_options), sizeof(nnm_stats),'
                    ' offsetof(nnm_stats, max_abs_err), offsetof(nnm_stats, scale)); return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [nnm.MERGE_DTYPE.itemsize, nnm.EDGE_DTYPE.itemsize, ctypes.sizeof(nnm.nnm_restrictions),
            ctypes.sizeof(nnm.nnm_options), ctypes.sizeof(nnm.nnm_stats),
            nnm.nnm_stats.max_abs_err.offset, nnm.nnm_stats.scale.offset]
    assert got == want


def test_batched_create_rejects_bad_offsets_without_touching_the_gpu(lib):
    # validation happens before any device work: a dummy X pointer is never read
    P = ctypes.c_void_p
    lib.nnm_create_batched.argtypes = [P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int, ctypes.c_int, P, P,
                                       ctypes.POINTER(P)]
    lib.nnm_create_batched.restype = ctypes.c_int
    out = P()
    for offs in ([1, 5, 9], [0, 5, 5], [0, 7, 3], [0]):
        arr = (ctypes.c_int64 * len(offs))(*offs)
        st = lib.nnm_create_batched(P(16), ctypes.cast(arr, P), len(offs) - 1, 4, 0, 0, None, None, ctypes.byref(out))
        assert st == 1 and not out.value, offs   # NNM_EINVAL


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with the CUDA library absent the binding raises instead of
    computing anything."""
    from paper_1402_3789_gb300 import nnm
    monkeypatch.setattr(nnm, "_LIB", None)
    monkeypatch.setattr(nnm, "library_path", lambda: str(tmp_path / "libnnm.so"))
    with pytest.raises(RuntimeError, match="not built"):
        nnm.load_library()
