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


def test_every_function_of_the_header_is_exported(lib):
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "ascc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(ascc_[a-z0-9_]+)\s*\(", text))
    assert "ascc_gemm_fp64_tc" in names and "ascc_solve" in names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_footprint_by_precision_and_streaming(lib):
    o, v, naux = 20, 200, 660
    fp64 = lib.ascc_footprint_bytes(o, v, naux, ctypes.byref(binding.default_options()))
    mixed = lib.ascc_footprint_bytes(
        o, v, naux, ctypes.byref(binding.default_options(precision=binding.ASCC_MIXED_BF16)))
    digits = lib.ascc_footprint_bytes(
        o, v, naux, ctypes.byref(binding.default_options(precision=binding.ASCC_FP64_TC)))
    streamed = lib.ascc_footprint_bytes(
        o, v, naux, ctypes.byref(binding.default_options(precision=binding.ASCC_MIXED_BF16,
                                                         ladder_stream=1)))
    rows, kk = (o + v) * v, v * v
    # stored ladder blocks: FP64 block + build temporary; 3 split planes + 6 digit planes;
    # 6 digit planes alone
    assert fp64 > 16 * rows * kk
    assert mixed > digits > 12 * rows * kk and mixed > 18 * rows * kk
    # streaming keeps none of them, only ~1 GB chunks
    assert mixed - streamed > 18 * rows * kk - 4e9


def test_default_options_keep_the_ladder_block_automatic(lib):
    opt = binding.default_options()
    assert opt.ladder_stream == 0 and opt.polish_tol == 1e-6
