"""Host-side fault injection: every device allocation of the library can be
made to fail (bude_debug_fail_alloc), and each call must then return
BUDE_ERR_OOM, release what it took, and leave the library and the CUDA
context usable.  Nothing here faults, traps or hangs the GPU: the injected
failure is decided on the host before any CUDA call is made.
"""
import numpy as np
import pytest
import torch

from paper_2509_21039_gb300 import bude, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
OPTS = bude.LaunchOptions(variant="ieee", ppwi=4, block=256)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2509_21039_gb300 import build
    build.build()
    bude.load()


@pytest.fixture(autouse=True)
def _disarm():
    bude.debug_fail_alloc(0)
    yield
    bude.debug_fail_alloc(0)


def _energies(deck, P):
    E = bude.energies(deck, P, opts=OPTS)
    torch.cuda.synchronize()
    return E.cpu().numpy()


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_arming_and_argument_checks():
    assert bude.debug_pending_fail_alloc() == 0
    bude.debug_fail_alloc(3)
    assert bude.debug_pending_fail_alloc() == 3
    with pytest.raises(bude.BudeError) as e:
        bude.debug_fail_alloc(-1)
    assert e.value.code == bude.ERR_INVALID_ARG
    bude.debug_fail_alloc(0)
    assert bude.debug_pending_fail_alloc() == 0


def test_every_allocation_of_deck_creation_and_first_call_can_fail():
    D = synth.make_deck(140, 10, 400, 34, 700)
    P = torch.from_numpy(D["poses"]).to(DEV)
    clean = bude.Deck(D, device=DEV)
    ref = _energies(clean, P)
    clean.close()
    free0 = _free_bytes()
    failed_at_creation = []
    for k in range(1, 14):
        bude.debug_fail_alloc(k)
        try:
            deck = bude.Deck(D, device=DEV)
        except bude.BudeError as e:
            assert e.code == bude.ERR_OOM, (k, e)
            failed_at_creation.append(k)
            assert bude.debug_pending_fail_alloc() == 0
            continue
        # the k-th allocation is still ahead: the first energies call makes it
        # (the workspace) or none is left
        try:
            E = _energies(deck, P)
            assert bude.debug_pending_fail_alloc() > 0 or k > 12
        except bude.BudeError as e:
            assert e.code == bude.ERR_OOM, (k, e)
            E = _energies(deck, P)  # the injection is one-shot: the retry works
        np.testing.assert_array_equal(E, ref)
        deck.close()
        bude.debug_fail_alloc(0)
    # creation makes several allocations, and each failure point was reached
    assert failed_at_creation == list(range(1, len(failed_at_creation) + 1))
    assert len(failed_at_creation) >= 5
    # nothing leaked (the caching allocator of torch is not involved)
    assert abs(_free_bytes() - free0) < (16 << 20)
    deck = bude.Deck(D, device=DEV)
    np.testing.assert_array_equal(_energies(deck, P), ref)
    deck.close()


def test_workspace_growth_failure_keeps_the_deck_usable():
    D = synth.make_deck(141, 8, 300, 34, 300)
    deck = bude.Deck(D, device=DEV)
    small = torch.from_numpy(D["poses"][:, :64].copy()).to(DEV)
    _energies(deck, small)           # allocates a small workspace
    big_np = synth.make_deck(142, 8, 300, 34, 200000)["poses"]
    big = torch.from_numpy(big_np).to(DEV)
    bude.debug_fail_alloc(1)
    with pytest.raises(bude.BudeError) as e:
        _energies(deck, big)          # must grow the workspace: injected failure
    assert e.value.code == bude.ERR_OOM
    E = _energies(deck, big)          # and now it grows
    ref = bude.energies(bude.Deck(D, device=DEV), big, opts=OPTS).cpu().numpy()
    np.testing.assert_array_equal(E, ref)
    deck.close()


def test_batched_plan_allocation_failure_is_not_cached():
    decks_np = [synth.make_deck([143, i], 6 + i, 200 + 50 * i, 34, 300 + 100 * i) for i in range(4)]
    decks = [bude.Deck(d, device=DEV) for d in decks_np]
    poses = [torch.from_numpy(d["poses"]).to(DEV) for d in decks_np]
    outs = [torch.empty(p.shape[1], device=DEV) for p in poses]
    bude.debug_fail_alloc(1)
    with pytest.raises(bude.BudeError) as e:
        bude.energies_batched(decks, poses, outs, opts=OPTS)
    assert e.value.code == bude.ERR_OOM
    bude.energies_batched(decks, poses, outs, opts=OPTS)
    torch.cuda.synchronize()
    for d, p, o in zip(decks, poses, outs):
        ref = bude.energies(d, p, opts=OPTS).cpu().numpy().astype(np.float64)
        got = o.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-5
    for d in decks:
        d.close()


def test_refine_plan_allocation_failure_recovers():
    D = synth.make_deck(144, 8, 300, 34, 256)
    deck = bude.Deck(D, device=DEV)
    P0 = torch.from_numpy(D["poses"]).to(DEV)
    P = P0.clone()
    bude.debug_fail_alloc(1)
    with pytest.raises(bude.BudeError) as e:
        bude.refine_device(deck, P, steps=3, opts=OPTS)
    assert e.value.code == bude.ERR_OOM
    torch.cuda.synchronize()
    assert torch.equal(P, P0)         # nothing ran: the poses are untouched
    Ea = bude.refine_device(deck, P, steps=3, opts=OPTS).cpu().numpy()
    Q = P0.clone()
    deck2 = bude.Deck(D, device=DEV)
    Eb = bude.refine_device(deck2, Q, steps=3, opts=OPTS).cpu().numpy()
    np.testing.assert_array_equal(Ea, Eb)
    deck.close()
    deck2.close()


def test_hartree_fock_plan_allocation_failures():
    S = synth.make_he_lattice(5, 8)
    dens = torch.from_numpy(S["dens"]).to(DEV)
    ref = bude.HartreeFock(S["geom"], S["xpnt"], S["coef"], device=DEV).fock(dens).cpu().numpy()
    fails = oks = 0
    for k in range(1, 24):
        bude.debug_fail_alloc(k)
        try:
            hf = bude.HartreeFock(S["geom"], S["xpnt"], S["coef"], device=DEV)
        except bude.BudeError as e:
            assert e.code == bude.ERR_OOM
            fails += 1
            continue
        bude.debug_fail_alloc(0)
        # the Fock build accumulates with atomics: equal up to summation order
        np.testing.assert_allclose(hf.fock(dens).cpu().numpy(), ref, rtol=1e-12, atol=1e-14)
        hf.close()
        oks += 1
    assert fails >= 8 and oks >= 1


def test_noalloc_entry_point_makes_no_allocation():
    D = synth.make_deck(145, 12, 500, 34, 2000)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    ref = bude.energies(deck, P, opts=OPTS).cpu().numpy().astype(np.float64)
    out = torch.empty(P.shape[1], device=DEV)
    bude.debug_fail_alloc(1)          # the next allocation would fail
    bude.energies_noalloc(deck, P, out, opts=OPTS)
    torch.cuda.synchronize()
    assert bude.debug_pending_fail_alloc() == 1   # none was attempted
    got = out.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-5
    deck.close()
