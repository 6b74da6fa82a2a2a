"""Cutoff culling (bude_options.cull): a warp skips a protein atom when every
one of its poses is beyond the pair's cutoff R + 4 A, where every term (and
its derivative) is exactly zero.  Energies, pose gradients and refinement
must be bit-identical to the unculled kernels of the same launch shape, for
every packed FP32 variant and shape, and on decks where nothing, some or
everything is culled.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_21039_gb300 import bude, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2509_21039_gb300 import build
    build.build()
    bude.load()


def _pair(D, **kw):
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(np.ascontiguousarray(D["poses"])).to(DEV)
    a = bude.energies(deck, P, opts=bude.LaunchOptions(cull=0, **kw)).cpu().numpy()
    b = bude.energies(deck, P, opts=bude.LaunchOptions(cull=1, **kw)).cpu().numpy()
    deck.close()
    return a, b


@pytest.mark.parametrize("variant", ["ieee", "fast", "comp"])
@pytest.mark.parametrize("ppwi,block", [(2, 128), (4, 256), (8, 384), (16, 256)])
def test_culled_energies_are_bit_identical(variant, ppwi, block):
    D = synth.make_deck(150, 20, 900, 34, 3000)
    a, b = _pair(D, variant=variant, ppwi=ppwi, block=block)
    np.testing.assert_array_equal(a, b)


def test_culled_with_chunked_protein_and_many_ctas():
    D = synth.make_deck(151, 16, 1500, 34, 2000)
    for tile, cps in ((100, 1), (257, 3)):
        a, b = _pair(D, variant="fast", ppwi=8, block=256, tile=tile, ctas_per_sm=cps)
        np.testing.assert_array_equal(a, b)


def test_everything_close_nothing_culled():
    # a protein packed around the ligand: every atom within the cutoff of every pose
    D = synth.make_deck(152, 12, 400, 34, 1024)
    rng = np.random.default_rng(7)
    D["pro_xyz"] = rng.uniform(-3.0, 3.0, size=D["pro_xyz"].shape).astype(np.float32)
    D["poses"][3:] *= 0.1
    a, b = _pair(D, variant="ieee", ppwi=8, block=256)
    np.testing.assert_array_equal(a, b)
    ref, A = oracle.energies(D, D["poses"], n_threads=-1, with_abs=True)
    assert (np.abs(b - ref) / np.maximum(A, 1.0)).max() <= 1e-5


def test_everything_far_gives_exact_zero():
    D = synth.make_deck(153, 10, 300, 34, 700)
    D["pro_xyz"] = D["pro_xyz"] + np.float32(200.0)
    a, b = _pair(D, variant="fast", ppwi=16, block=256)
    assert np.all(a == 0.0) and np.all(b == 0.0)


def test_negative_hardness_and_batched_and_noalloc():
    D = synth.make_deck(154, 10, 500, 12, 900)
    D["hardness"] = np.linspace(-30.0, 30.0, 12).astype(np.float32)
    D["poses"][3:] *= 0.3
    a, b = _pair(D, variant="comp", ppwi=4, block=256)
    np.testing.assert_array_equal(a, b)

    decks_np = [synth.make_deck([155, i], 8 + 4 * i, 300 + 200 * i, 34, 500 + 300 * i)
                for i in range(5)]
    decks = [bude.Deck(d, device=DEV) for d in decks_np]
    poses = [torch.from_numpy(d["poses"]).to(DEV) for d in decks_np]
    outs0 = [torch.empty(p.shape[1], device=DEV) for p in poses]
    outs1 = [torch.empty(p.shape[1], device=DEV) for p in poses]
    o0 = bude.LaunchOptions(variant="fast", ppwi=8, block=512, ctas_per_sm=2)
    o1 = bude.LaunchOptions(variant="fast", ppwi=8, block=512, ctas_per_sm=2, cull=1)
    bude.energies_batched(decks, poses, outs0, opts=o0)
    bude.energies_batched(decks, poses, outs1, opts=o1)
    torch.cuda.synchronize()
    for x, y in zip(outs0, outs1):
        assert torch.equal(x, y)

    out = torch.empty(poses[2].shape[1], device=DEV)
    bude.energies_noalloc(decks[2], poses[2], out, opts=o1)
    ref = bude.energies(decks[2], poses[2], opts=o0)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    for d in decks:
        d.close()


@pytest.mark.parametrize("variant,ppwi,block", [("ieee", 4, 384), ("fast", 4, 384), ("comp", 2, 256),
                                                ("fast", 8, 128), ("ieee", 2, 256)])
def test_culled_pose_gradients_are_bit_identical(variant, ppwi, block):
    D = synth.make_deck(157, 16, 800, 34, 1500)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    e0, g0 = bude.pose_grad(deck, P, opts=bude.LaunchOptions(variant=variant, ppwi=ppwi, block=block))
    e1, g1 = bude.pose_grad(deck, P, opts=bude.LaunchOptions(variant=variant, ppwi=ppwi, block=block,
                                                                cull=1))
    torch.cuda.synchronize()
    assert torch.equal(e0, e1) and torch.equal(g0, g1)
    deck.close()


def test_culled_refinement_is_bit_identical():
    D = synth.make_deck(158, 12, 600, 34, 700)
    deck = bude.Deck(D, device=DEV)
    P0 = torch.from_numpy(D["poses"]).to(DEV)
    A, B = P0.clone(), P0.clone()
    ea = bude.refine_device(deck, A, steps=5, opts=bude.LaunchOptions(variant="fast", ppwi=4, block=384))
    eb = bude.refine_device(deck, B, steps=5, opts=bude.LaunchOptions(variant="fast", ppwi=4, block=384,
                                                                      cull=1))
    torch.cuda.synchronize()
    assert torch.equal(ea, eb) and torch.equal(A, B)
    deck.close()


def test_cull_flag_is_checked_and_ignored_where_not_built():
    D = synth.make_deck(156, 6, 200, 34, 300)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    with pytest.raises(bude.BudeError) as e:
        bude.energies(deck, P, opts=bude.LaunchOptions(variant="fast", cull=2))
    assert e.value.code == bude.ERR_INVALID_ARG
    # odd ppwi and FP64 ignore the flag
    for kw in (dict(variant="ieee", ppwi=1), dict(variant="fp64", ppwi=2)):
        a = bude.energies(deck, P, opts=bude.LaunchOptions(cull=0, **kw)).cpu().numpy()
        b = bude.energies(deck, P, opts=bude.LaunchOptions(cull=1, **kw)).cpu().numpy()
        np.testing.assert_array_equal(a, b)
    _, g0 = bude.pose_grad(deck, P, opts=bude.LaunchOptions(variant="ieee", ppwi=4))
    _, g1 = bude.pose_grad(deck, P, opts=bude.LaunchOptions(variant="ieee", ppwi=4, cull=1))
    assert torch.equal(g0, g1)
    deck.close()
