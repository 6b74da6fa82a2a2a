"""bude_energies_noalloc: the allocation-free entry point.

It serves callers that must not allocate device memory themselves (hosts
that own the memory budget and forbid allocation inside their execution
callbacks, latency-critical loops).  It runs the persistent energy kernel
with its scratch in the library's fixed device array.  This file is named to
be collected last, so that a run stopping at the first failure has already
run every other test; it passes alone in a fresh process and after the
others.

The two entry points run the same kernel in the same launch shape with the
same fixed-order reductions, so their results must be identical bit for bit:
any difference would mean the shared array leaked one call's partial sums
or tickets into another.
"""
import ctypes

import pytest
import torch

from paper_2509_21039_gb300 import bude, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
# the array's capacity (include/bude.h): partial sums and tickets
STATIC_PARTIAL_DOUBLES = 512 * 1024
STATIC_TICKETS = 16 * 1024


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
    ref = bude.energies(deck, P, opts=opts).clone()
    out = torch.full((P.shape[1],), float("nan"), device=DEV)
    for _ in range(2):   # the second call reuses the array the first one left behind
        E = _call_noalloc(deck, P, out, opts)
        assert torch.equal(E, ref)
        out.fill_(float("nan"))


def test_noalloc_small_and_full_size_decks():
    for D in (synth.make_deck(132, 5, 60, 7, 33), synth.make_deck(1, **synth.FULL)):
        deck = bude.Deck(D, device=DEV)
        P = torch.from_numpy(D["poses"]).to(DEV)
        ref = bude.energies(deck, P).clone()
        out = torch.empty(P.shape[1], device=DEV)
        for _ in range(2):
            E = bude.energies_noalloc(deck, P, out)
            torch.cuda.synchronize()
            assert torch.equal(E, ref)


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
    ref = bude.energies(deck, small).clone()
    assert torch.equal(bude.energies_noalloc(deck, small, o2), ref)


def test_noalloc_partial_sum_bound_alone():
    """A call whose tickets fit but whose partial sums do not: at 16 poses
    per lane and one CTA per SM the grid has one CTA per SM, and a call needs
    (CTAs + tiles) x 512 partial sums.  The largest pose count that fits
    exactly fills the array and must match bude_energies; one pose more needs
    one more tile, which no longer fits."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    opts = dict(variant="ieee", ppwi=16, block=384, ctas_per_sm=1)
    slots = STATIC_PARTIAL_DOUBLES // (32 * 16)
    n_fit = (slots - sms) * 32 * 16
    assert n_fit // 512 < STATIC_TICKETS and (n_fit + 1 + 511) // 512 < STATIC_TICKETS
    D = synth.make_deck(134, 4, 40, 5, n_fit + 1)
    deck = bude.Deck(D, device=DEV)
    P_all = torch.from_numpy(D["poses"]).to(DEV)
    out = torch.empty(n_fit + 1, device=DEV)
    with pytest.raises(bude.BudeError) as e:
        bude.energies_noalloc(deck, P_all, out, **opts)
    assert e.value.code == bude.ERR_UNSUPPORTED
    assert "partial sums" in str(e.value)
    P = P_all[:, :n_fit].contiguous()
    ref = bude.energies(deck, P, **opts).clone()
    E = bude.energies_noalloc(deck, P, out[:n_fit], **opts)
    torch.cuda.synchronize()
    assert torch.equal(E, ref)
