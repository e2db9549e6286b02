"""The C-ABI library builds, loads without a GPU, and exports every function
that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for path in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.add(name)
    return names


@pytest.fixture(scope="module")
def built_lib():
    import paper_2403_06348_gb300 as alto
    path = alto.build()
    return ctypes.CDLL(path), alto


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("alto_encode", "alto_mttkrp", "cpals_run", "alto_free", "alto_query",
              "alto_decode", "alto_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(built_lib):
    lib, alto = built_lib
    names = _declared_functions()
    assert names, "no declarations parsed"
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    # the Python binding marshals every declared entry point
    assert names <= set(alto.SIGNATURES), sorted(names - set(alto.SIGNATURES))


def test_version_and_error_string_without_gpu(built_lib):
    _, alto = built_lib
    L = alto.lib()
    assert L.alto_version() >= 100
    # argument errors are detected before any device work
    h = ctypes.c_void_p()
    st = L.alto_encode(None, None, None, 0, 0, None, None, ctypes.byref(h))
    assert st == -1
    assert b"nmodes" in L.alto_last_error()
    dims = (ctypes.c_uint64 * 6)(*([1 << 26] * 5 + [1]))
    st = L.alto_encode(None, None, dims, 5, 0, None, None, ctypes.byref(h))
    assert st == -4  # 130 index bits: unsupported, found by the host-side bit plan


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2403_06348_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", text).replace("oracles", ""), f


def test_host_coordinates_are_passed_without_a_copy():
    """int32 host coordinates reach the library as the same memory (read as
    uint32), so a pinned buffer stays pinned; other dtypes are converted."""
    import numpy as np
    import torch
    import paper_2403_06348_gb300 as alto
    c32 = np.arange(12, dtype=np.int32).reshape(3, 4)
    a = alto.host_array(c32, np.uint32)
    assert a.dtype == np.uint32 and np.shares_memory(a, c32)
    np.testing.assert_array_equal(a, c32.astype(np.uint32))
    t = torch.arange(12, dtype=torch.int32).reshape(3, 4)
    b = alto.host_array(t, np.uint32)
    assert b.dtype == np.uint32 and b.ctypes.data == t.data_ptr()
    neg = alto.host_array(np.array([[-1]], dtype=np.int32), np.uint32)
    assert neg[0, 0] == 0xFFFFFFFF            # out of range for any mode: rejected on the device
    c64 = np.arange(6, dtype=np.int64).reshape(2, 3)
    d = alto.host_array(c64, np.uint32)
    assert d.dtype == np.uint32 and not np.shares_memory(d, c64)
    v = np.ones(5, dtype=np.float32)
    assert np.shares_memory(alto.host_array(v, np.float32), v)


def test_coordinates_that_do_not_fit_uint32_are_refused():
    """Host coordinates of a wider or signed type are converted only when every
    value fits uint32; otherwise the binding raises instead of wrapping them
    into another tensor (nothing reaches the library)."""
    import numpy as np
    import paper_2403_06348_gb300 as alto
    big = np.array([[1, 1 << 32]], dtype=np.int64)
    with pytest.raises(ValueError):
        alto.host_array(big, np.uint32, "coords")
    with pytest.raises(ValueError):
        alto.host_array(np.array([[-3]], dtype=np.int64), np.uint32, "coords")
    with pytest.raises(TypeError):
        alto.host_array(np.array([[1.5]]), np.uint32, "coords")
    with pytest.raises(ValueError):
        alto.alto_encode(np.array([[0, 1 << 33]], dtype=np.int64), np.ones(2, np.float32), (4,))
    ok = alto.host_array(np.array([[0, (1 << 32) - 1]], dtype=np.int64), np.uint32, "coords")
    assert ok.dtype == np.uint32 and int(ok[0, 1]) == (1 << 32) - 1
