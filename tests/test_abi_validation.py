"""Host-side validation at the C ABI (CPU only): every invalid argument is rejected with
NL_EINVAL and a message before any device work, and the binding raises instead of falling
back when the library is missing."""
import subprocess
import sys

import numpy as np
import pytest

from paper_2101_08825_gb300 import nl


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2101_08825_gb300.build import build
    build()
    nl.lib()


def _tri_mesh():
    coords = np.array([[0.0, 1.0, 0.0, 1.0], [0.0, 0.0, 1.0, 1.0]])
    conn = np.array([[0, 1, 3], [0, 3, 2]], np.int32)
    return coords, conn, np.ones(2, np.uint8), np.zeros(4, np.uint8)


def _rejects(fn, *args, match):
    with pytest.raises(nl.NLError) as e:
        fn(*args)
    assert e.value.status == nl.NL_EINVAL
    assert match in str(e.value)


def test_mesh_create_rejects_bad_dimension_and_sizes():
    c, t, eio, nf = _tri_mesh()
    _rejects(nl.nl_mesh_create, 4, np.zeros((4, 5)), np.zeros((1, 5), np.int32), eio[:1], nf[:5],
             match="dim must be 2 or 3")
    _rejects(nl.nl_mesh_create, 2, np.zeros((2, 0)), t, eio, nf[:0], match="bad sizes")


def test_mesh_create_rejects_non_finite_coordinates():
    c, t, eio, nf = _tri_mesh()
    for bad in (np.nan, np.inf, -np.inf):
        c2 = c.copy()
        c2[1, 2] = bad
        _rejects(nl.nl_mesh_create, 2, c2, t, eio, nf, match="non-finite coordinate")


def test_mesh_create_rejects_out_of_range_vertices():
    c, t, eio, nf = _tri_mesh()
    for bad in (-1, 4):
        t2 = t.copy()
        t2[1, 2] = bad
        _rejects(nl.nl_mesh_create, 2, c, t2, eio, nf, match="vertex index out of range")


@pytest.mark.parametrize("dim", [2, 3])
def test_mesh_create_rejects_degenerate_elements(dim):
    if dim == 2:
        c = np.array([[0.0, 1.0, 2.0], [0.0, 1.0, 2.0]])  # collinear
        t = np.array([[0, 1, 2]], np.int32)
    else:
        c = np.array([[0.0, 1.0, 0.0, 1.0], [0.0, 0.0, 1.0, 1.0], [0.0, 0.0, 0.0, 0.0]])  # coplanar
        t = np.array([[0, 1, 2, 3]], np.int32)
    _rejects(nl.nl_mesh_create, dim, c, t, np.ones(1, np.uint8), np.zeros(c.shape[1], np.uint8),
             match="degenerate element")


def test_mesh_create_box_rejects_bad_arguments():
    _rejects(nl.nl_mesh_create_box, 1, (4,), 0.25, (0.0,), 1, match="dim must be 2 or 3")
    _rejects(nl.nl_mesh_create_box, 2, (4, 0), 0.25, (0.0, 0.0), 1, match="cells must be >= 1")


def test_null_handles_are_rejected():
    L = nl.lib()
    import ctypes
    out = ctypes.c_void_p()
    assert L.nl_pairs_build(None, 0.1, 0.01, ctypes.byref(out)) == nl.NL_EINVAL
    assert b"NULL" in L.nl_last_error()
    assert L.nl_mesh_info(None, None, None, None) == nl.NL_EINVAL
    assert L.nl_mesh_create(2, 3, None, 1, None, None, None, None, ctypes.byref(out)) == nl.NL_EINVAL


def test_error_state_is_cleared_by_the_next_call():
    L = nl.lib()
    assert L.nl_mesh_info(None, None, None, None) == nl.NL_EINVAL
    assert L.nl_last_error() != b""
    assert L.nl_set_allocator(None, None, None) == nl.NL_OK
    assert L.nl_last_error() == b""


def test_binding_raises_when_the_library_is_missing(tmp_path):
    code = ("import paper_2101_08825_gb300.nl as nl; nl.LIB_PATH = %r\n"
            "try:\n    nl.lib()\nexcept RuntimeError as e:\n    print('raised', e)\n" %
            str(tmp_path / "missing.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("raised") and "missing" in r.stdout
