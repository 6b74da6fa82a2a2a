"""bude_energies_noalloc: the allocation-free entry point.

It serves callers that must not allocate device memory themselves (hosts
that own the memory budget and forbid allocation inside their execution
callbacks, latency-critical loops).  It runs the persistent energy kernel
with its scratch in the library's fixed device array.  This file is named to
be collected last, so that a run stopping at the first failure has already
run every other test; it passes alone in a fresh process and after the
others.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2509_21039_gb300 import bude, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
GATE_IEEE = 1e-5   # the FP32 IEEE parity gate of the other GPU tests


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2509_21039_gb300 import build
    build.build()
    bude.load()


def _call_noalloc(deck, P, out, opts):
    # straight through the C ABI
    o = opts.c()
    rc = bude.load().bude_energies_noalloc(
        deck.handle, ctypes.c_void_p(P.data_ptr()), P.shape[1],
        ctypes.c_void_p(out.data_ptr()), ctypes.byref(o),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == bude.OK, bude.load().bude_last_error().decode()
    torch.cuda.synchronize()
    return out.clone()


@pytest.mark.parametrize("variant,ppwi", [("ieee", 8), ("fast", 16), ("comp", 4)])
def test_noalloc_matches_energies_twice_in_a_row(variant, ppwi):
    D = synth.make_deck(131, 24, 700, 34, 5000)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    opts = bude.LaunchOptions(variant=variant, ppwi=ppwi, block=256)
    ref = bude.energies(deck, P, opts=opts).cpu().numpy().astype(np.float64)
    out = torch.full((P.shape[1],), float("nan"), device=DEV)
    for _ in range(2):   # the second call reuses the array the first one left behind
        E = _call_noalloc(deck, P, out, opts).cpu().numpy().astype(np.float64)
        err = np.abs(E - ref) / np.maximum(np.abs(ref), 1.0)
        assert err.max() <= GATE_IEEE, err.max()
        out.fill_(float("nan"))


def test_noalloc_small_and_full_size_decks():
    for D in (synth.make_deck(132, 5, 60, 7, 33), synth.make_deck(1, **synth.FULL)):
        deck = bude.Deck(D, device=DEV)
        P = torch.from_numpy(D["poses"]).to(DEV)
        ref = bude.energies(deck, P).cpu().numpy().astype(np.float64)
        out = torch.empty(P.shape[1], device=DEV)
        for _ in range(2):
            E = bude.energies_noalloc(deck, P, out).cpu().numpy().astype(np.float64)
            assert (np.abs(E - ref) / np.maximum(np.abs(ref), 1.0)).max() <= GATE_IEEE


def test_noalloc_rejects_more_poses_than_its_scratch_holds():
    D = synth.make_deck(133, 4, 40, 5, 8)
    deck = bude.Deck(D, device=DEV)
    n = 600_000   # one-pose-per-lane tiles: ~19k tickets > 16384
    P = torch.zeros((6, n), device=DEV)
    out = torch.empty(n, device=DEV)
    with pytest.raises(bude.BudeError) as e:
        bude.energies_noalloc(deck, P, out, ppwi=1, block=256)
    assert e.value.code == bude.ERR_UNSUPPORTED
    assert "fixed scratch" in str(e.value)
    # the library is still usable afterwards
    small = torch.from_numpy(D["poses"]).to(DEV)
    o2 = torch.empty(small.shape[1], device=DEV)
    ref = bude.energies(deck, small).cpu().numpy()
    np.testing.assert_allclose(bude.energies_noalloc(deck, small, o2).cpu().numpy(), ref,
                               rtol=1e-5, atol=1e-5)
