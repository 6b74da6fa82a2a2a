"""bude_energies_host: the end-to-end call with host poses and host energies.
Its results must equal bude_energies of the same launch shape bit for bit,
from pinned and from pageable memory, across staging-buffer growth, and its
argument checks and allocation failures must leave the deck usable."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2509_21039_gb300 import bude, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
OPTS = bude.LaunchOptions(variant="ieee", ppwi=8, block=256)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2509_21039_gb300 import build
    build.build()
    bude.load()


@pytest.mark.parametrize("pinned", [True, False])
def test_host_call_equals_device_call(pinned):
    D = synth.make_deck(160, 16, 700, 34, 3000)
    deck = bude.Deck(D, device=DEV)
    ref = bude.energies(deck, torch.from_numpy(D["poses"]).to(DEV), opts=OPTS).cpu()
    hp = torch.from_numpy(D["poses"])
    if pinned:
        hp = hp.pin_memory()
    got = bude.energies_host(deck, hp, opts=OPTS)
    assert got.device.type == "cpu" and torch.equal(got, ref)
    # larger n grows the staging buffer; smaller n reuses it
    for m in (5000, 100, 3000):
        D2 = synth.make_deck(160, 16, 700, 34, m)
        ref2 = bude.energies(deck, torch.from_numpy(D2["poses"]).to(DEV), opts=OPTS).cpu()
        assert torch.equal(bude.energies_host(deck, torch.from_numpy(D2["poses"]), opts=OPTS), ref2)
    deck.close()


def test_host_call_edge_cases():
    D = synth.make_deck(161, 6, 200, 34, 50)
    deck = bude.Deck(D, device=DEV)
    empty = torch.empty((6, 0), dtype=torch.float32)
    assert bude.energies_host(deck, empty).numel() == 0
    with pytest.raises(ValueError):
        bude.energies_host(deck, torch.from_numpy(D["poses"]).to(DEV))
    lib = bude.load()
    o = OPTS.c()
    rc = lib.bude_energies_host(deck.handle, None, 50, None, ctypes.byref(o), None)
    assert rc == bude.ERR_INVALID_ARG
    rc = lib.bude_energies_host(None, None, 50, None, ctypes.byref(o), None)
    assert rc == bude.ERR_INVALID_ARG
    # a staging allocation that fails leaves the deck usable
    bude.debug_fail_alloc(0)
    big = torch.from_numpy(synth.make_deck(161, 6, 200, 34, 4000)["poses"])
    bude.energies_host(deck, torch.from_numpy(D["poses"]), opts=OPTS)   # small staging exists
    bude.debug_fail_alloc(1)
    try:
        with pytest.raises(bude.BudeError) as e:
            bude.energies_host(deck, big, opts=OPTS)
        assert e.value.code == bude.ERR_OOM
    finally:
        bude.debug_fail_alloc(0)
    ref = bude.energies(deck, big.to(DEV), opts=OPTS).cpu()
    assert torch.equal(bude.energies_host(deck, big, opts=OPTS), ref)
    deck.close()
