"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Error measure per pose: |E_gpu - E_ref| / max(A_ref, 1), A_ref = 0.5 sum |e|
(the oracle's absolute-term sum).  Gates, from the arithmetic: FP32 with
correctly rounded sqrt keeps every pair term within a few ulp (2^-23 ~ 1.2e-7
relative) and sums of up to ~1e5 terms stay far inside 1e-5; the approximate
sqrt/sin/cos of the fast variant adds ~2^-21 relative per term, gated at 1e-4.
The FP64 variant computes in double and rounds once to the float32 output,
so it must agree with the oracle to half an FP32 ulp of the result plus
1e-12 of the scale (summation order).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2509_21039_gb300 import bude, synth

pytestmark = pytest.mark.gpu

GATE = {"ieee": 1e-5, "fast": 1e-4, "comp": 1e-5, "fp64": 1e-12}
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2509_21039_gb300 import build
    build.build()
    bude.load()


def scaled_error(E, ref, A, variant=None):
    d = np.abs(np.asarray(E, np.float64) - ref)
    if variant == "fp64":
        # remove the one rounding to the float32 output (half an ulp)
        d = np.maximum(d - np.abs(ref) * 2.0 ** -24 * (1 + 1e-9), 0.0)
    return d / np.maximum(A, 1.0)


def run(deck_np, poses=None, variant="ieee", **kw):
    deck = bude.Deck(deck_np, device=DEV)
    P = torch.from_numpy(np.ascontiguousarray(poses if poses is not None else deck_np["poses"])).to(DEV)
    E = bude.energies(deck, P, variant=variant, **kw)
    torch.cuda.synchronize()
    return E.cpu().numpy()


def check(deck_np, variant="ieee", poses=None, **kw):
    poses = poses if poses is not None else deck_np["poses"]
    ref, A = oracle.energies(deck_np, poses, n_threads=-1, with_abs=True)
    E = run(deck_np, poses, variant, **kw)
    err = scaled_error(E, ref, A, variant)
    assert err.max() <= GATE[variant], (variant, kw, err.max())
    return E, ref, A


# --- small decks: several tiles, ragged tails, every launch shape -----------

@pytest.mark.parametrize("variant", ["ieee", "fast", "comp", "fp64"])
def test_small_deck_all_variants(variant):
    D = synth.make_deck(101, 16, 300, 34, 1000)
    check(D, variant)


@pytest.mark.parametrize("ppwi", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("block", [64, 256, 1024])
def test_launch_shapes_ieee(ppwi, block):
    D = synth.make_deck(102, 11, 257, 34, 777)
    try:
        check(D, "ieee", ppwi=ppwi, block=block)
    except bude.BudeError as e:
        # a block too large for this register count cannot be resident
        assert e.code == bude.ERR_UNSUPPORTED and block == 1024


@pytest.mark.parametrize("variant,ppwi", [("fast", 4), ("fast", 16), ("comp", 2), ("comp", 8),
                                          ("fp64", 1), ("fp64", 4)])
def test_launch_shapes_other_variants(variant, ppwi):
    D = synth.make_deck(103, 9, 190, 34, 600)
    check(D, variant, ppwi=ppwi, block=128)


@pytest.mark.parametrize("tile", [32, 100, 257])
@pytest.mark.parametrize("cps", [1, 2, 3])
def test_protein_chunking_and_grid(tile, cps):
    D = synth.make_deck(104, 13, 640, 34, 900)
    check(D, "ieee", ppwi=4, block=128, tile=tile, ctas_per_sm=cps)


@pytest.mark.parametrize("tile", [32, 257])
@pytest.mark.parametrize("variant,ppwi", [("fast", 16), ("fp64", 4), ("fp64", 1)])
def test_protein_chunking_other_layouts(tile, variant, ppwi):
    # the packed kernels stage each protein atom as two duplicated float4
    # pairs and the FP64 kernel as two double pairs; chunks that cut the
    # type runs exercise both layouts, for energies and pose gradients
    D = synth.make_deck(105, 11, 700, 34, 640)
    _, ref, A = check(D, variant, ppwi=ppwi, block=128, tile=tile)
    Eref, Gref, S = oracle.pose_grad(D, D["poses"], n_threads=-1, with_scale=True)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    E, G = bude.pose_grad(deck, P, variant=variant, ppwi=min(ppwi, 8), block=128, tile=tile)
    assert scaled_error(E.cpu().numpy(), Eref, A, variant).max() <= GATE[variant]
    assert grad_error(G.cpu().numpy(), Gref, S, variant) <= GRAD_GATE[variant]


def test_small_config_seed0_every_variant():
    D = synth.make_deck(0, **synth.SMALL)
    ref, A = oracle.energies(D, D["poses"], n_threads=-1, with_abs=True)
    for v in ("ieee", "fast", "comp", "fp64"):
        E = run(D, variant=v)
        err = scaled_error(E, ref, A, v)
        assert err.max() <= GATE[v], (v, err.max())


@pytest.mark.parametrize("variant,ppwi,block", [("fast", 16, 384), ("ieee", 8, 256),
                                                ("comp", 4, 256), ("fast", 2, 128)])
def test_partial_last_tile_every_size_class(variant, ppwi, block):
    """Pose counts that are not a multiple of the 32 P-pose tile: the last
    tile's lanes beyond the count compute a clamped pose and write nothing.
    Tails of 1, 63, 64, 65 poses, one pose either side of half a tile and one
    short of a full tile, alone and after two full tiles; energies and pose
    gradients against the oracle."""
    TP = 32 * ppwi
    tails = sorted({1, 63, 64, 65, TP // 2 - 1, TP // 2 + 1, TP - 1} - {0})
    D = synth.make_deck(109, 12, 300, 34, 2 * TP + TP - 1)
    deck = bude.Deck(D, device=DEV)
    for n in [t for t in tails if t < TP] + [2 * TP + t for t in tails if t < TP]:
        P = np.ascontiguousarray(D["poses"][:, :n])
        ref, A = oracle.energies(D, P, n_threads=-1, with_abs=True)
        E = bude.energies(deck, torch.from_numpy(P).to(DEV), variant=variant, ppwi=ppwi,
                          block=block).cpu().numpy()
        assert scaled_error(E, ref, A).max() <= GATE[variant], (n, variant, ppwi)
        if variant != "comp":
            Eg, G = bude.pose_grad(deck, torch.from_numpy(P).to(DEV), variant=variant,
                                   ppwi=min(ppwi, 8), block=256)
            Eref, Gref, S = oracle.pose_grad(D, P, n_threads=-1, with_scale=True)
            g = G.cpu().numpy().astype(np.float64)
            err = max(np.max(np.abs(g[:3] - Gref[:3]) / np.maximum(S[0], 1)),
                      np.max(np.abs(g[3:] - Gref[3:]) / np.maximum(S[1], 1)))
            assert err <= 1e-4, (n, variant, err)


def test_deterministic_repeat():
    D = synth.make_deck(105, 20, 500, 34, 2048)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    a = bude.energies(deck, P).clone()
    b = bude.energies(deck, P).clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b)


# --- edge cases -----------------------------------------------------------

def test_zero_poses_is_noop():
    D = synth.make_deck(106, 4, 50, 5, 0)
    deck = bude.Deck(D, device=DEV)
    E = bude.energies(deck, torch.zeros((6, 0), device=DEV))
    assert E.numel() == 0


@pytest.mark.parametrize("which", ["lig", "pro"])
def test_empty_molecule_gives_zero(which):
    D = synth.make_deck(107, 5, 60, 6, 70)
    if which == "lig":
        D["lig_xyz"] = D["lig_xyz"][:0]
        D["lig_type"] = D["lig_type"][:0]
    else:
        D["pro_xyz"] = D["pro_xyz"][:0]
        D["pro_type"] = D["pro_type"][:0]
    E = run(D)
    assert np.all(E == 0.0)


def test_single_pose_single_pair_closed_form():
    # one ligand atom at the origin, one protein atom at 2 A: types A and B of
    # the hand-worked table give E = 1/9
    D = dict(lig_xyz=np.zeros((1, 3), np.float32), lig_type=np.array([0], np.int32),
             pro_xyz=np.array([[2.0, 0, 0]], np.float32), pro_type=np.array([1], np.int32),
             radius=np.array([1.5, 1.5], np.float32), hardness=np.array([10, 30], np.float32),
             elsc=np.array([0.5, -0.5], np.float32), hbtype=np.array([1, 2], np.int32),
             poses=np.zeros((6, 1), np.float32))
    # e = 20/9 - 2 cancels: compare at the scale A = (20/9 + 2)/2 of the terms
    A = (20.0 / 9.0 + 2.0) / 2.0
    for v in ("ieee", "fast", "comp", "fp64"):
        E = run(D, variant=v)
        assert abs(E[0] - 1.0 / 9.0) <= GATE[v] * A + (2.0 ** -24 if v == "fp64" else 0.0)


def test_atom_on_atom_is_finite():
    D = synth.make_deck(108, 6, 80, 7, 40)
    D["pro_xyz"][5] = D["lig_xyz"][2]          # exact overlap at the identity pose
    P = np.zeros((6, 40), np.float32)
    P[3:, 1:] = D["poses"][3:, 1:]
    E, ref, A = check(D, "ieee", poses=P)
    assert np.isfinite(E).all()
    check(D, "fast", poses=P)
    check(D, "fp64", poses=P)


def test_nan_pose_gives_nan_and_far_pose_gives_zero():
    D = synth.make_deck(109, 6, 80, 7, 64)
    P = D["poses"].copy()
    P[0, 3] = np.nan
    P[4, 7] = np.nan
    P[1, 9] = np.inf
    P[3, 11] = np.inf        # infinitely far ligand: every pair beyond the cutoff
    P[3, 12] = 1e6
    ref = oracle.energies(D, P)
    for v in ("ieee", "fast", "comp", "fp64"):
        E = run(D, P, v)
        assert np.isnan(E[[3, 7, 9]]).all()
        assert E[11] == 0.0 and E[12] == 0.0
        ok = np.isfinite(ref)
        np.testing.assert_array_equal(np.isnan(E), ~ok)


@pytest.mark.parametrize("variant,ppwi", [("ieee", 2), ("fast", 16), ("comp", 8), ("ieee", 1),
                                           ("fp64", 4), ("fp64", 1)])
def test_negative_and_zero_hardness(variant, ppwi):
    # The packed kernels and the FP64 kernel take the steric term as
    # sign(H) z^2 with z = max(0, sqrt|H| (1 - d/R)); a forcefield with
    # negative, zero and positive hardness exercises both signs and the H = 0
    # edge.  Close contacts (small translations) keep the steric term active.
    D = synth.make_deck(131, 10, 260, 12, 600)
    D["hardness"] = np.linspace(-30.0, 30.0, 12).astype(np.float32)
    D["hardness"][5] = 0.0
    D["poses"][3:] *= 0.3
    _, ref, A = check(D, variant, ppwi=ppwi, block=128)
    assert (np.asarray(D["hardness"]) < 0).any()
    Eref, Gref, S = oracle.pose_grad(D, D["poses"], n_threads=-1, with_scale=True)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    E, G = bude.pose_grad(deck, P, variant=variant, ppwi=min(ppwi, 8 if variant != "fp64" else 4),
                          block=128)
    assert scaled_error(E.cpu().numpy(), Eref, A, variant).max() <= GATE[variant]
    assert grad_error(G.cpu().numpy(), Gref, S, variant) <= GRAD_GATE[variant]


@pytest.mark.parametrize("hb", [(0,), (1, 2), (0, 0), (0, 1), (2, 0, 1)])
@pytest.mark.parametrize("variant,ppwi,block", [("ieee", 16, 384), ("fast", 8, 512),
                                                ("comp", 4, 256), ("ieee", 1, 128)])
def test_degenerate_type_sets(hb, variant, ppwi, block):
    # one type (a single run per chunk), only polar types (no desolvation term
    # anywhere, donor-acceptor doubling), only apolar types, and mixtures: the
    # packed kernels' runs, desolvation skip and row-cost split at their limits
    nt = len(hb)
    D = synth.make_deck(170 + nt, 9, 333, nt, 700)
    D["hbtype"] = np.array(hb, np.int32)
    D["poses"][3:] *= 0.4
    check(D, variant, ppwi=ppwi, block=block)
    E1 = run(D, D["poses"][:, :1].copy(), variant, ppwi=ppwi, block=block)   # one pose
    ref1, A1 = oracle.energies(D, D["poses"][:, :1], n_threads=-1, with_abs=True)
    assert scaled_error(E1, ref1, A1).max() <= GATE[variant]


def test_type_indexing_is_exact_with_many_types():
    # FP64 on the GPU matches to 1e-12: any wrong type lookup would be gross
    D = synth.make_deck(110, 40, 400, 64, 256)
    E, ref, A = check(D, "fp64")
    check(D, "ieee")
    # and every ligand type maps to its own table row
    deck = bude.Deck(D, device=DEV)
    assert deck.n_rows == len(np.unique(D["lig_type"]))


def test_pair_table_too_large_is_a_clean_error():
    # 60 ligand rows x 600 types of 32-byte records cannot be staged
    D = synth.make_deck(116, 200, 300, 600, 64)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    with pytest.raises(bude.BudeError) as e:
        bude.energies(deck, P)
    assert e.value.code == bude.ERR_UNSUPPORTED
    # the device is still healthy afterwards
    D2 = synth.make_deck(117, 5, 50, 6, 32)
    check(D2, "ieee")


def test_invalid_decks_are_rejected():
    D = synth.make_deck(111, 5, 50, 6, 8)
    bad = dict(D, pro_type=D["pro_type"].copy())
    bad["pro_type"][7] = 6
    with pytest.raises(bude.BudeError) as e:
        bude.Deck(bad, device=DEV)
    assert e.value.code == bude.ERR_INVALID_ARG
    bad = dict(D, lig_type=D["lig_type"].copy())
    bad["lig_type"][0] = -1
    with pytest.raises(bude.BudeError):
        bude.Deck(bad, device=DEV)
    bad = dict(D, radius=D["radius"].copy())
    bad["radius"][2] = 0.0
    with pytest.raises(bude.BudeError):
        bude.Deck(bad, device=DEV)
    bad = dict(D, hbtype=D["hbtype"].copy())
    bad["hbtype"][1] = 3
    with pytest.raises(bude.BudeError):
        bude.Deck(bad, device=DEV)
    bad = dict(D, pro_xyz=D["pro_xyz"].copy())
    bad["pro_xyz"][3, 1] = np.nan
    with pytest.raises(bude.BudeError):
        bude.Deck(bad, device=DEV)


def test_bad_options_are_rejected():
    D = synth.make_deck(112, 5, 50, 6, 8)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    for kw in (dict(ppwi=3), dict(block=48), dict(block=2048), dict(variant=7),
               dict(variant="fp64", ppwi=8), dict(tile=-1)):
        with pytest.raises(bude.BudeError):
            bude.energies(deck, P, **kw)


# --- full-size workload: every pose computed, a sample checked --------------

def _bench_options(variant, n_lig, n_pro, n_poses, mode="plain"):
    # the launch configuration bench.py times: the tuned shape for this workload
    from paper_2509_21039_gb300 import tune
    o = tune.lookup(variant, n_lig, n_pro, n_poses, mode=mode)
    return o if o is not None else bude.LaunchOptions(variant=variant)


def test_full_size_sampled_against_oracle():
    D = synth.make_deck(1, **synth.FULL)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(D["poses"].shape[1], 48, replace=False))
    idx[-1] = D["poses"].shape[1] - 1
    ref, A = oracle.energies(D, D["poses"][:, idx], n_threads=-1, with_abs=True)
    n = D["poses"].shape[1]
    for v in ("ieee", "fast", "comp"):
        for mode in ("plain", "cull"):
            o = _bench_options(v, 64, 2672, n, mode)
            E = bude.energies(deck, P, opts=o).cpu().numpy()
            assert np.isfinite(E).all()
            err = scaled_error(E[idx], ref, A)
            assert err.max() <= GATE[v], (v, mode, err.max())


def test_flat_work_index_beyond_2_pow_31():
    # 2^23 poses of the full deck: the flat space (tiles x 64 x 2672 pairs) is
    # 2.8e9 iterations or more at any P <= 16, past 32-bit indexing; sampled
    # against the oracle, the last pose included
    D = synth.make_deck(9, 64, 2672, 34, 1 << 23)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    o = _bench_options("fast", 64, 2672, 65536)
    tiles = -(-P.shape[1] // (32 * o.ppwi))
    assert tiles * 64 * 2672 > 2 ** 31
    E = bude.energies(deck, P, opts=o).cpu().numpy()
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(P.shape[1], 40, replace=False))
    idx[-1] = P.shape[1] - 1
    ref, A = oracle.energies(D, D["poses"][:, idx], n_threads=-1, with_abs=True)
    assert np.isfinite(E).all()
    assert scaled_error(E[idx], ref, A).max() <= GATE["fast"]
    deck.close()


def test_long_protein_many_ligand_atoms():
    # 60000 protein atoms cannot be staged at once: many chunks per tile, and
    # 300 ligand rows in the warp split's cost prefix
    D = synth.make_deck(10, 300, 60000, 34, 300)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    idx = np.arange(0, 300, 5)
    ref, A = oracle.energies(D, D["poses"][:, idx], n_threads=-1, with_abs=True)
    for kw in (dict(variant="ieee", ppwi=8, block=512), dict(variant="fast", ppwi=16, block=384),
               dict(variant="comp", ppwi=2, block=256, cull=1)):
        E = bude.energies(deck, P, opts=bude.LaunchOptions(**kw)).cpu().numpy()
        assert scaled_error(E[idx], ref, A).max() <= GATE[kw["variant"]], kw
    deck.close()


# --- batched --------------------------------------------------------------

def test_batched_uneven_against_oracle_and_plain():
    shapes = [(8, 500, 300), (3, 40, 1), (17, 1200, 1025), (5, 77, 33), (1, 1, 7),
              (30, 640, 4097)]
    decks_np = [synth.make_deck([7, i], nl, npro, 34, n) for i, (nl, npro, n) in enumerate(shapes)]
    decks = [bude.Deck(d, device=DEV) for d in decks_np]
    poses = [torch.from_numpy(d["poses"]).to(DEV) for d in decks_np]
    outs = bude.energies_batched(decks, poses)
    outs2 = bude.energies_batched(decks, poses)    # graph replay
    torch.cuda.synchronize()
    for d, p, o, o2, dnp in zip(decks, poses, outs, outs2, decks_np):
        assert torch.equal(o, o2)
        n = dnp["poses"].shape[1]
        idx = np.unique(np.linspace(0, n - 1, min(n, 40)).astype(int))
        ref, A = oracle.energies(dnp, dnp["poses"][:, idx], n_threads=-1, with_abs=True)
        E = o.cpu().numpy()
        assert scaled_error(E[idx], ref, A).max() <= GATE["ieee"]
        plain = bude.energies(d, p).cpu().numpy()
        assert scaled_error(E, plain.astype(np.float64), np.abs(plain)).max() <= 2 * GATE["ieee"]


@pytest.mark.parametrize("opts", [dict(variant="ieee"),
                                  dict(variant="fast", ppwi=8, block=256, ctas_per_sm=4),
                                  dict(variant="comp", ppwi=2, block=128, ctas_per_sm=2),
                                  dict(variant="fp64", ppwi=1, block=128)])
def test_batched_cost_weighted_split(opts):
    # decks whose pairs cost differently (none, about half or most of them
    # with a desolvation term) weight the CTAs' split of the flat space; with
    # many CTAs and tiny decks some CTAs get no units at all
    specs = [(0, 9, 300, 700), (1, 4, 50, 3), (2, 13, 800, 2100), (0, 2, 7, 40), (3, 20, 1500, 5000)]
    decks_np = []
    for i, (pattern, nl, npro, n) in enumerate(specs):
        d = synth.make_deck([17, i], nl, npro, 12, n)
        if pattern == 0:
            d["hbtype"][:] = 0          # no polar type: no desolvation pair
        elif pattern == 1:
            d["hbtype"][:] = 1          # all polar: no desolvation pair either
        elif pattern == 2:
            d["hbtype"][:] = np.arange(12) % 2   # half polar
        decks_np.append(d)
    decks = [bude.Deck(d, device=DEV) for d in decks_np]
    poses = [torch.from_numpy(d["poses"]).to(DEV) for d in decks_np]
    o = bude.LaunchOptions(**opts)
    outs = bude.energies_batched(decks, poses, opts=o)
    outs2 = bude.energies_batched(decks, poses, opts=o)
    torch.cuda.synchronize()
    gate = GATE["fp64"] if opts["variant"] == "fp64" else GATE[opts["variant"]]
    for d, p, out, out2, dnp in zip(decks, poses, outs, outs2, decks_np):
        assert torch.equal(out, out2)
        n = dnp["poses"].shape[1]
        idx = np.unique(np.linspace(0, n - 1, min(n, 30)).astype(int))
        ref, A = oracle.energies(dnp, dnp["poses"][:, idx], n_threads=-1, with_abs=True)
        E = out.cpu().numpy()
        assert scaled_error(E[idx], ref, A, opts["variant"]).max() <= gate
        plain = bude.energies(d, p, opts=o).cpu().numpy()
        # FP64: both are FP64 sums rounded once to float32, so within two ulps
        between = 2.0 ** -22 if opts["variant"] == "fp64" else 2 * gate
        assert scaled_error(E, plain.astype(np.float64), np.abs(plain)).max() <= between
    for d in decks:
        d.close()


@pytest.mark.parametrize("variant", ["fast", "ieee"])
def test_batched_full_64_deck_workload_sampled_against_oracle(variant):
    """The batched workload the bench times (64 uneven decks: ligand 8-128,
    protein 500-5000, poses 1024-65536, log-uniform, seed 3) in the bench's
    tuned batched shape, brute force and culled: 16 poses of every deck (its
    last one included) against the oracle at the variant's gate."""
    from paper_2509_21039_gb300 import tune
    decks_np = synth.make_batched(3, 64)
    decks = [bude.Deck(d, device=DEV) for d in decks_np]
    poses = [torch.from_numpy(d["poses"]).to(DEV) for d in decks_np]
    e = tune.load_table().get(tune.key(variant, "n64", "batched"))
    o = (bude.LaunchOptions(variant=variant, ppwi=e["ppwi"], block=e["block"],
                            ctas_per_sm=e["ctas_per_sm"], tile=e["tile"]) if e
         else bude.LaunchOptions(variant=variant))
    # the culled launch in the bench's culled shape
    c = tune.lookup(variant, 64, 2672, 65536, mode="cull")
    oc = bude.LaunchOptions(variant=variant, ppwi=c.ppwi if c else 8, block=c.block if c else 256,
                            ctas_per_sm=c.ctas_per_sm if c else 1, tile=c.tile if c else 0, cull=1)
    outs = [x.cpu().numpy() for x in bude.energies_batched(decks, poses, opts=o)]
    outs_c = [x.cpu().numpy() for x in bude.energies_batched(decks, poses, opts=oc)]
    worst = 0.0
    for dnp, E, Ec in zip(decks_np, outs, outs_c):
        n = dnp["poses"].shape[1]
        idx = np.unique(np.linspace(0, n - 1, 16).round().astype(np.int64))
        assert idx[-1] == n - 1
        ref, A = oracle.energies(dnp, np.ascontiguousarray(dnp["poses"][:, idx]), n_threads=-1,
                                 with_abs=True)
        for x in (E, Ec):
            assert np.isfinite(x).all()
            worst = max(worst, float(scaled_error(x[idx], ref, A).max()))
    assert worst <= GATE[variant], worst
    for d in decks:
        d.close()


@pytest.mark.parametrize("shape", [((5, 1, 0), (4, 5, 2)), ((1, 2, 1), (3, 6, 2)),
                                   ((5, 1, 2), (20, 1, 0)), ((2, 3, 0), (7, 2, 2), (1, 9, 1))])
@pytest.mark.parametrize("variant,ppwi", [("fast", 16), ("ieee", 1)])
def test_batched_tiny_launch_every_tile_finished(shape, variant, ppwi):
    """Batched launches of a few dozen units, where one unit's cost is close
    to a CTA's share of the total: every CTA's piece must hold at least one
    unit, or a tile would count an arrival that never comes and stay
    unwritten (the outputs start as NaN to catch that).  hb pattern 0: no
    polar type, 1: all polar, 2: half polar, so the units' costs differ."""
    decks_np = []
    for i, (nl, npro, pattern) in enumerate(shape):
        d = synth.make_deck([19, i], nl, npro, 6, 37 + 11 * i)
        d["hbtype"][:] = {0: 0, 1: 1, 2: np.arange(6) % 2}[pattern]
        decks_np.append(d)
    decks = [bude.Deck(d, device=DEV) for d in decks_np]
    poses = [torch.from_numpy(d["poses"]).to(DEV) for d in decks_np]
    outs = [torch.full((p.shape[1],), float("nan"), device=DEV) for p in poses]
    bude.energies_batched(decks, poses, outs, variant=variant, ppwi=ppwi, block=128)
    torch.cuda.synchronize()
    for dnp, o in zip(decks_np, outs):
        ref, A = oracle.energies(dnp, dnp["poses"], n_threads=-1, with_abs=True)
        E = o.cpu().numpy()
        assert np.isfinite(E).all()
        assert scaled_error(E, ref, A).max() <= GATE[variant]


def test_batched_with_empty_instances():
    d0 = synth.make_deck(113, 6, 90, 8, 50)
    d1 = synth.make_deck(114, 6, 90, 8, 0)
    d2 = synth.make_deck(115, 6, 90, 8, 20)
    d2["lig_xyz"], d2["lig_type"] = d2["lig_xyz"][:0], d2["lig_type"][:0]
    decks = [bude.Deck(d, device=DEV) for d in (d0, d1, d2)]
    poses = [torch.from_numpy(d["poses"]).to(DEV) for d in (d0, d1, d2)]
    outs = [torch.full((p.shape[1],), 7.0, device=DEV) for p in poses]
    bude.energies_batched(decks, poses, outs)
    torch.cuda.synchronize()
    assert torch.all(outs[2] == 0)
    ref, A = oracle.energies(d0, d0["poses"], with_abs=True)
    assert scaled_error(outs[0].cpu().numpy(), ref, A).max() <= GATE["ieee"]


# --- adjoint --------------------------------------------------------------

GRAD_GATE = {"ieee": 1e-4, "fast": 1e-4, "comp": 1e-4, "fp64": 1e-10}


def grad_error(G, Gref, S, variant=None):
    G = np.asarray(G, np.float64)
    d = np.abs(G - Gref)
    if variant == "fp64":
        d = np.maximum(d - np.abs(Gref) * 2.0 ** -24 * (1 + 1e-9), 0.0)
    sa = np.maximum(S[0], 1.0)
    st = np.maximum(S[1], 1.0)
    return max(np.max(d[:3] / sa), np.max(d[3:] / st))


@pytest.mark.parametrize("variant", ["ieee", "fast", "comp", "fp64"])
def test_pose_gradient_against_oracle(variant):
    D = synth.make_deck(120, 12, 300, 34, 700)
    Eref, Gref, S = oracle.pose_grad(D, D["poses"], n_threads=-1, with_scale=True)
    _, A = oracle.energies(D, D["poses"], n_threads=-1, with_abs=True)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    E, G = bude.pose_grad(deck, P, variant=variant)
    torch.cuda.synchronize()
    assert scaled_error(E.cpu().numpy(), Eref, A, variant).max() <= GATE[variant]
    assert grad_error(G.cpu().numpy(), Gref, S, variant) <= GRAD_GATE[variant]


@pytest.mark.parametrize("ppwi", [1, 2, 4, 8])
def test_pose_gradient_launch_shapes(ppwi):
    D = synth.make_deck(121, 7, 210, 34, 333)
    Eref, Gref, S = oracle.pose_grad(D, D["poses"], n_threads=-1, with_scale=True)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    _, G = bude.pose_grad(deck, P, want_energy=False, ppwi=ppwi, block=128, tile=64)
    assert grad_error(G.cpu().numpy(), Gref, S) <= GRAD_GATE["ieee"]


def test_pose_gradient_matches_central_differences_of_gpu_fp64():
    D = synth.make_deck(122, 8, 200, 34, 64)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    _, G = bude.pose_grad(deck, P, variant="fp64")
    _, _, S = oracle.pose_grad(D, D["poses"], with_scale=True)
    h = 1e-3   # float32 poses: the step must be representable around |pose| <= 5
    G = G.cpu().numpy().astype(np.float64)
    for j in range(6):
        Pp, Pm = D["poses"].copy(), D["poses"].copy()
        Pp[j] += np.float32(h)
        Pm[j] -= np.float32(h)
        step = (Pp[j].astype(np.float64) - Pm[j].astype(np.float64))
        fd = (run(D, Pp, "fp64").astype(np.float64) - run(D, Pm, "fp64").astype(np.float64)) / step
        scale = np.maximum(S[0] if j < 3 else S[1], 1.0)
        assert np.median(np.abs(fd - G[j]) / scale) < 1e-3, j


def test_gradient_full_size_sampled():
    D = synth.make_deck(4, **synth.GRAD)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    E, G = bude.pose_grad(deck, P)
    idx = np.sort(np.random.default_rng(1).choice(P.shape[1], 24, replace=False))
    Eref, Gref, S = oracle.pose_grad(D, D["poses"][:, idx], n_threads=-1, with_scale=True)
    _, A = oracle.energies(D, D["poses"][:, idx], n_threads=-1, with_abs=True)
    assert scaled_error(E.cpu().numpy()[idx], Eref, A).max() <= GATE["ieee"]
    assert grad_error(G.cpu().numpy()[:, idx], Gref, S) <= GRAD_GATE["ieee"]


def test_autograd_function_and_refinement():
    D = synth.make_deck(123, 10, 400, 34, 256)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV).requires_grad_(True)
    E = bude.PoseEnergy.apply(P, deck, None)
    w = torch.linspace(0.5, 1.5, E.numel(), device=DEV)
    (E * w).sum().backward()
    _, G = bude.pose_grad(deck, P.detach())
    torch.testing.assert_close(P.grad, G * w.unsqueeze(0))
    # a few steps of refinement on the device lower the mean energy
    p2 = P.detach().clone()
    e0 = bude.energies(deck, p2).mean().item()
    e10 = bude.refine_device(deck, p2, steps=10, step0=0.05).mean().item()
    assert e10 < e0


def test_ieee_square_root_is_correctly_rounded_everywhere():
    mism, first = bude.selfcheck_sqrt()
    assert mism == 0, f"{mism} mismatches, first at bits {first:#010x}"


@pytest.mark.parametrize("variant", ["ieee", "fast", "fp64"])
def test_gradient_with_energy_shaped_defaults(variant):
    # the defaults hold one shape per variant, here the energy kernel's widest
    # (P = 16 or 4 with 384 threads, more threads than the adjoint kernel's
    # registers allow): a gradient call without options still runs, with the
    # block cut to what the adjoint kernel can hold, and matches an explicit shape
    D = synth.make_deck(171, 12, 300, 34, 700)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    saved = bude.default_options(variant)
    try:
        wide = bude.LaunchOptions(variant=variant, ppwi=4 if variant == "fp64" else 16, block=384,
                                  ctas_per_sm=1)
        bude.set_default_options(wide)
        e0, g0 = bude.pose_grad(deck, P, opts=bude.LaunchOptions(variant=variant))
        e1, g1 = bude.pose_grad(deck, P, opts=bude.LaunchOptions(
            variant=variant, ppwi=4 if variant == "fp64" else 8, block=128))
        torch.cuda.synchronize()
        tol = 1e-9 if variant == "fp64" else 1e-4
        np.testing.assert_allclose(e0.cpu().numpy(), e1.cpu().numpy(), rtol=tol, atol=tol)
        np.testing.assert_allclose(g0.cpu().numpy(), g1.cpu().numpy(), rtol=tol * 10, atol=tol * 10)
        assert np.all(np.isfinite(e0.cpu().numpy()))
    finally:
        bude.set_default_options(saved)
        deck.close()


def test_device_named_without_index_is_the_current_device():
    # "cuda" and no device at all both mean the current device, and tensors
    # made there are accepted
    D = synth.make_deck(5, 6, 40, 34, 33)
    P = torch.from_numpy(D["poses"]).to(DEV)
    ref = bude.energies(bude.Deck(D, device=DEV), P)
    for dev in ("cuda", None):
        deck = bude.Deck(D, device=dev)
        assert deck.device == torch.device(DEV)
        assert torch.equal(bude.energies(deck, P), ref)


def test_batched_plan_cache_keeps_the_64_most_recent():
    D = synth.make_deck(150, 8, 60, 34, 40)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    ref = bude.energies_batched([deck], [P])[0].clone()
    outs = [torch.empty(P.shape[1], device=DEV) for _ in range(70)]
    for o in outs:                                  # 70 argument sets: 70 plans built
        bude.energies_batched([deck], [P], outs=[o])
    assert bude.debug_cached_plans()[0] == 64
    assert all(torch.equal(o, ref) for o in outs)
    outs[0].zero_()                                 # dropped long ago: rebuilt
    bude.energies_batched([deck], [P], outs=[outs[0]])
    assert torch.equal(outs[0], ref)
    assert bude.debug_cached_plans()[0] == 64
    deck.close()                                    # every cached plan used this deck
    assert bude.debug_cached_plans()[0] == 0


def test_batched_replay_after_a_smaller_launch_of_the_same_kernel():
    # a kernel's shared-memory limit only grows: a plain launch of the same
    # kernel on a small deck, between two replays of a batch that needs far
    # more shared memory, leaves the replay valid and unchanged
    big = synth.make_deck(160, 32, 5000, 34, 512)
    small = synth.make_deck(161, 4, 40, 34, 64)
    db, ds = bude.Deck(big, device=DEV), bude.Deck(small, device=DEV)
    Pb = torch.from_numpy(big["poses"]).to(DEV)
    Ps = torch.from_numpy(small["poses"]).to(DEV)
    opts = bude.LaunchOptions(variant="ieee", ppwi=8, block=256)
    out = bude.energies_batched([db], [Pb], opts=opts)[0]
    first = out.clone()
    bude.energies(ds, Ps, opts=opts)
    out.zero_()
    bude.energies_batched([db], [Pb], outs=[out], opts=opts)
    torch.cuda.synchronize()
    assert torch.equal(out, first)


def test_launch_counts_of_each_call():
    # bude_last_launch_count reports the kernels a call enqueued (the bench's
    # gpu_launches adds these up): one persistent launch per energy, gradient
    # or batched call, 2 + 3 x steps for a refinement, none for a deck with
    # no atom pairs (its outputs are cleared by a memset)
    D = synth.make_deck(180, 6, 90, 34, 300)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    bude.energies(deck, P)
    assert bude.launch_count() == 1
    bude.energies_noalloc(deck, P, torch.empty(P.shape[1], device=DEV))
    assert bude.launch_count() == 1
    bude.pose_grad(deck, P)
    assert bude.launch_count() == 1
    D2 = synth.make_deck(181, 9, 120, 34, 77)
    deck2 = bude.Deck(D2, device=DEV)
    P2 = torch.from_numpy(D2["poses"]).to(DEV)
    for _ in range(2):                               # first call captures, second replays
        bude.energies_batched([deck, deck2], [P, P2])
        assert bude.launch_count() == 1
    for _ in range(2):
        bude.refine_device(deck, P.clone(), steps=3, step0=0.05)
        assert bude.launch_count() == 2 + 3 * 3
    empty = dict(D, lig_xyz=D["lig_xyz"][:0], lig_type=D["lig_type"][:0])
    E = bude.energies(bude.Deck(empty, device=DEV), P)
    assert bude.launch_count() == 0 and not E.any()
    torch.cuda.synchronize()
