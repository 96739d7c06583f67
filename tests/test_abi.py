"""CPU checks of the C ABI: the library builds, loads and exports every declared symbol."""
import ctypes

import pytest

from paper_2501_10515_gb300 import binding, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    names = binding.symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_and_defaults(lib):
    assert lib.ascc_status_string(0) == b"ok"
    assert lib.ascc_status_string(4) == b"not converged"
    opt = binding.default_options()
    assert opt.precision == binding.ASCC_FP64 and opt.linearize == 1
    assert opt.r_tol == 1e-8 and opt.e_tol == 1e-10 and opt.diis_dim == 16


def test_footprint_grows_with_size(lib):
    a = lib.ascc_footprint_bytes(4, 20, 72, None)
    b = lib.ascc_footprint_bytes(20, 200, 660, None)
    assert 0 < a < b
    # the o=20, v=200 context holds the (xc|bd) block: n v^3 doubles
    assert b > 8 * 220 * 200 ** 3


def test_create_rejects_bad_sizes_without_touching_the_gpu(lib):
    h = ctypes.c_void_p()
    st = lib.ascc_create(ctypes.byref(h), 0, 5, 3, None, None, 0, None, None, None)
    assert st == 1 and not h.value
