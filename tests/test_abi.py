"""C-ABI checks that need no GPU: the library builds, loads and exports every
function include/bude.h declares; argument validation that happens before
any CUDA call."""
import ctypes

import pytest

from paper_2509_21039_gb300 import bude
from paper_2509_21039_gb300 import build as build_mod


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return bude.load()


def test_header_declares_the_boundary():
    names = bude.header_functions()
    for n in ("bude_create_deck", "bude_destroy_deck", "bude_energies",
              "bude_energies_batched", "bude_pose_grad", "bude_status_string"):
        assert n in names


def test_every_declared_function_is_exported(lib):
    missing = [n for n in bude.header_functions() if not hasattr(lib, n)]
    assert missing == []


def test_status_strings(lib):
    for code in (bude.OK, bude.ERR_INVALID_ARG, bude.ERR_CUDA, bude.ERR_OOM,
                 bude.ERR_UNSUPPORTED, bude.ERR_DEVICE_FLAG):
        s = lib.bude_status_string(code).decode()
        assert s and s != "unknown status"
    assert lib.bude_status_string(12345).decode() == "unknown status"


def test_null_arguments_are_rejected_without_a_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.bude_create_deck(None, None, ctypes.byref(h)) == bude.ERR_INVALID_ARG
    assert h.value is None
    desc = bude.DeckDesc(4, 4, 0, None, None, None)
    assert lib.bude_create_deck(ctypes.byref(desc), None, ctypes.byref(h)) == bude.ERR_INVALID_ARG
    desc = bude.DeckDesc(-1, 4, 3, None, None, None)
    assert lib.bude_create_deck(ctypes.byref(desc), None, ctypes.byref(h)) == bude.ERR_INVALID_ARG
    desc = bude.DeckDesc(4, 4, bude.MAX_TYPES + 1, None, None, None)
    assert lib.bude_create_deck(ctypes.byref(desc), None, ctypes.byref(h)) == bude.ERR_INVALID_ARG
    o = bude.Options()
    assert lib.bude_energies(None, None, 10, None, ctypes.byref(o), None) == bude.ERR_INVALID_ARG
    assert lib.bude_pose_grad(None, None, 10, None, None, ctypes.byref(o), None) == bude.ERR_INVALID_ARG
    assert lib.bude_energies_batched(None, None, None, None, -1, None, None) == bude.ERR_INVALID_ARG
    assert lib.bude_energies_batched(None, None, None, None, 0, None, None) == bude.OK
    assert "NULL" in lib.bude_last_error().decode() or lib.bude_last_error()


def test_default_options_roundtrip(lib):
    for v in range(4):
        o = bude.default_options(v)
        assert o.variant == v and o.ppwi > 0 and o.block % 32 == 0
    with pytest.raises(bude.BudeError):
        bude.set_default_options(bude.LaunchOptions(variant=0, ppwi=3, block=256))
    with pytest.raises(bude.BudeError):
        bude.set_default_options(bude.LaunchOptions(variant=0, ppwi=8, block=100))
    with pytest.raises(bude.BudeError):
        bude.set_default_options(bude.LaunchOptions(variant=3, ppwi=16, block=256))


def test_pack_atoms_keeps_type_bits():
    import numpy as np
    rec = bude.pack_atoms(np.array([[1.0, 2.0, 3.0]]), np.array([33]))
    assert rec.dtype == np.float32 and rec.shape == (1, 4)
    assert rec[0, 3:].view(np.int32)[0] == 33


def test_laplacian_kernel_selection_is_host_logic(lib):
    # the TMA stencil needs float32, a 16-byte aligned u and rows of a multiple
    # of 16 bytes; the pointer is only inspected, never dereferenced
    path = lib.bude_laplacian_path
    a = ctypes.c_void_p(1 << 20)
    assert path(0, a, 64, 64, 64) == 1
    assert path(0, a, 3, 3, 4) == 1
    assert path(0, ctypes.c_void_p((1 << 20) + 4), 64, 64, 64) == 0   # misaligned base
    assert path(0, a, 64, 64, 62) == 0                                # rows of 248 bytes
    assert path(1, a, 64, 64, 64) == 0                                # float64: register kernel
    assert path(0, a, 2, 64, 64) == 0                                 # no interior
    assert path(0, a, 64, 64, 3) == 0
    assert path(2, a, 64, 64, 64) == bude.ERR_INVALID_ARG
    assert path(0, a, -1, 64, 64) == bude.ERR_INVALID_ARG
    assert lib.bude_wait_timeouts(None, None) == bude.ERR_INVALID_ARG
