"""The C ABI loads and exports every declared symbol; its host-side tables agree with the
oracle's independently derived ones (CPU only, no device work)."""
import ctypes
import math

import numpy as np
import pytest

import oracle as O
from paper_2101_08825_gb300 import nl


@pytest.fixture(scope="module")
def L():
    from paper_2101_08825_gb300.build import build
    build()
    return nl.lib()


def test_every_declared_symbol_is_exported(L):
    names = nl.declared_functions()
    assert len(names) >= 20
    raw = ctypes.CDLL(nl.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_version_and_error_strings(L):
    assert b"sm_103a" in L.nl_version()
    assert isinstance(L.nl_last_error(), bytes)


def test_allocator_hook_validation(L):
    assert L.nl_set_allocator(None, None, None) == nl.NL_OK
    fake = ctypes.cast(ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                        ctypes.c_void_p)(lambda *a: None), ctypes.c_void_p)
    assert L.nl_set_allocator(fake, None, None) == nl.NL_EINVAL
    assert L.nl_set_allocator(None, None, None) == nl.NL_OK


@pytest.mark.parametrize("dim", [2, 3])
def test_library_rule_matches_oracle_rule(dim):
    b1, w1 = nl.nl_quad_rule(dim)
    b2, w2 = O.quad_rule(dim)
    assert b1.shape == b2.shape
    # same point set up to ordering: match each library point to an oracle point
    for q in range(len(w1)):
        d = np.abs(b2 - b1[q]).max(axis=1)
        k = int(np.argmin(d))
        assert d[k] < 1e-15 and abs(w2[k] - w1[q]) < 1e-16


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("kernel", [0, 1])
def test_library_constant_matches_oracle(dim, kernel):
    for delta, eps in ((0.1, 0.01), (4 / 256, 4 / 256 / 5), (0.2, 0.1)):
        c1 = nl.nl_kernel_constant(dim, kernel, delta, eps)
        c2 = O.kernel_constant(dim, kernel, delta, eps)
        assert abs(c1 / c2 - 1) < 2e-14


def test_library_constant_rejects_bad_eps():
    assert math.isnan(nl.nl_kernel_constant(2, 0, 0.1, 0.2))
    assert math.isnan(nl.nl_kernel_constant(2, 0, 0.1, 0.0))
