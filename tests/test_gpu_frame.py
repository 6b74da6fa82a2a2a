"""Parity far from the coordinate origin.

Real docking decks sit wherever their structure file puts them, often tens to
hundreds of Angstrom from the origin (the paper's bm1 deck is a real
protein-ligand system, Sec. 3).  The energy depends only on the differences
x' - p (Sec. 2.2: the pair score is a function of the atom-atom distance),
so moving the protein and every pose translation by one vector o leaves
each pose's energy unchanged; the oracle computes it in FP64 from the
shifted inputs as given.  The FP32 kernels must hold the same gates there:
the rounding of x' = R x + t grows with |t|, so the deck works in a frame
centred on its protein.
Offsets 0, 100 and 500 Angstrom along a generic direction; every packed
FAST shape (P = 2, 8, 16) with and without cutoff culling, the other FP32
variants, the adjoint, the forcefield gradient and a batched launch.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_21039_gb300 import bude, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GATE = {"ieee": 1e-5, "fast": 1e-4, "comp": 1e-5}
# a unit vector with no zero component, so every axis is shifted
DIRECTION = np.array([0.6, -0.48, 0.64])


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2509_21039_gb300 import build
    build.build()
    bude.load()


def shifted(D, offset):
    """The deck with its protein and its pose translations moved by offset *
    DIRECTION, rounded to float32 as a caller would hold them."""
    o = (offset * DIRECTION).astype(np.float64)
    S = dict(D)
    S["pro_xyz"] = (D["pro_xyz"].astype(np.float64) + o).astype(np.float32)
    P = D["poses"].astype(np.float64).copy()
    P[3:] += o[:, None]
    S["poses"] = np.ascontiguousarray(P.astype(np.float32))
    return S


def energies_err(D, variant, **kw):
    ref, A = oracle.energies(D, D["poses"], n_threads=-1, with_abs=True)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    E = bude.energies(deck, P, variant=variant, **kw).cpu().numpy().astype(np.float64)
    deck.close()
    return float((np.abs(E - ref) / np.maximum(A, 1.0)).max())


@pytest.fixture(scope="module")
def deck0():
    return synth.make_deck(170, 32, 1200, 34, 1500)


@pytest.mark.parametrize("offset", [0.0, 100.0, 500.0])
@pytest.mark.parametrize("ppwi", [2, 8, 16])
@pytest.mark.parametrize("cull", [0, 1])
def test_fast_energies_far_from_origin(deck0, offset, ppwi, cull):
    # the bench's shapes: P = 16 runs 384 threads brute force; its culled
    # kernel needs more registers than 384 threads can have, so 256
    block = 384 if (ppwi == 16 and not cull) else 256
    err = energies_err(shifted(deck0, offset), "fast", ppwi=ppwi, block=block, cull=cull)
    assert err <= GATE["fast"], (offset, ppwi, cull, err)


@pytest.mark.parametrize("variant,ppwi", [("ieee", 16), ("ieee", 1), ("comp", 8), ("fast", 1)])
def test_other_variants_far_from_origin(deck0, variant, ppwi):
    err = energies_err(shifted(deck0, 500.0), variant, ppwi=ppwi, block=256)
    assert err <= GATE[variant], (variant, ppwi, err)


@pytest.mark.parametrize("variant,ppwi,block", [("fast", 16, 384), ("ieee", 16, 384),
                                                ("comp", 8, 256)])
def test_ten_thousand_angstrom_from_origin(deck0, variant, ppwi, block):
    """At 1e4 A a float32 coordinate resolves only 1e-3 A, and the oracle
    scores the inputs as given.  The deck's frame shift and the translations'
    shift are differences of floats within a factor of two of each other,
    hence exact, so the kernels still see the small coordinates."""
    err = energies_err(shifted(deck0, 1.0e4), variant, ppwi=ppwi, block=block)
    assert err <= GATE[variant], (variant, err)


def test_fp64_far_from_origin(deck0):
    """The FP64 kernel reads the atoms as given: still within 1e-12 plus the
    float32 rounding of the output."""
    D = shifted(deck0, 500.0)
    D["poses"] = np.ascontiguousarray(D["poses"][:, :256])
    ref, A = oracle.energies(D, D["poses"], n_threads=-1, with_abs=True)
    deck = bude.Deck(D, device=DEV)
    E = bude.energies(deck, torch.from_numpy(D["poses"]).to(DEV), variant="fp64")
    d = np.abs(E.cpu().numpy().astype(np.float64) - ref)
    d = np.maximum(d - np.abs(ref) * 2.0 ** -24 * (1 + 1e-9), 0.0)
    assert (d / np.maximum(A, 1.0)).max() <= 1e-12


def test_error_does_not_grow_with_the_offset(deck0):
    """The shifted decks' FAST error stays at the origin deck's level (the
    frame makes the kernel see the same small coordinates)."""
    e0 = energies_err(deck0, "fast", ppwi=16, block=384)
    e500 = energies_err(shifted(deck0, 500.0), "fast", ppwi=16, block=384)
    assert e500 <= max(4.0 * e0, 2e-6), (e0, e500)


@pytest.mark.parametrize("variant,ppwi,cull", [("fast", 8, 0), ("fast", 8, 1), ("ieee", 8, 0),
                                               ("ieee", 1, 0)])
def test_pose_gradient_far_from_origin(deck0, variant, ppwi, cull):
    D = shifted(deck0, 500.0)
    D["poses"] = np.ascontiguousarray(D["poses"][:, :700])
    Eref, Gref, S = oracle.pose_grad(D, D["poses"], n_threads=-1, with_scale=True)
    deck = bude.Deck(D, device=DEV)
    E, G = bude.pose_grad(deck, torch.from_numpy(D["poses"]).to(DEV), variant=variant,
                          ppwi=ppwi, block=256, cull=cull)
    g = G.cpu().numpy().astype(np.float64)
    err = max(np.max(np.abs(g[:3] - Gref[:3]) / np.maximum(S[0], 1)),
              np.max(np.abs(g[3:] - Gref[3:]) / np.maximum(S[1], 1)))
    assert err <= 1e-4, (variant, ppwi, err)


@pytest.mark.parametrize("variant", ["fast", "ieee"])
def test_param_grad_far_from_origin(variant):
    D = shifted(synth.make_deck(171, 14, 350, 12, 600), 500.0)
    GL, GF, SL, SF = oracle.param_grad(D, D["poses"], with_scale=True)
    deck = bude.Deck(D, device=DEV)
    gl, gf = bude.param_grad(deck, torch.from_numpy(D["poses"]).to(DEV), variant=variant,
                             ppwi=8, block=256)
    for g, ref, sc in ((gl, GL, SL), (gf, GF, SF)):
        d = np.abs(g.cpu().numpy().astype(np.float64) - ref)
        err = (d / np.maximum(sc, 1e-9 * sc.max())).max()
        assert err <= 1e-4, (variant, err)


def test_batched_decks_in_different_frames():
    """One launch over decks at different offsets: each instance takes its
    own deck's frame."""
    decks_np = [shifted(synth.make_deck([172, i], 10 + 5 * i, 300 + 200 * i, 34, 400 + 300 * i), off)
                for i, off in enumerate([0.0, 500.0, 100.0, 250.0])]
    decks = [bude.Deck(d, device=DEV) for d in decks_np]
    poses = [torch.from_numpy(d["poses"]).to(DEV) for d in decks_np]
    outs = bude.energies_batched(decks, poses, variant="fast", ppwi=16, block=384)
    torch.cuda.synchronize()
    for d, E in zip(decks_np, outs):
        ref, A = oracle.energies(d, d["poses"], n_threads=-1, with_abs=True)
        err = (np.abs(E.cpu().numpy().astype(np.float64) - ref) / np.maximum(A, 1.0)).max()
        assert err <= GATE["fast"], err
