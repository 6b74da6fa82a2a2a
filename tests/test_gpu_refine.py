"""bude_refine: per-pose adaptive gradient descent in one CUDA graph, against
the oracle's FP64 restatement of the same rule (oracle.refine).

Accept/reject decisions are taken in FP32 on the GPU and in FP64 in the
oracle, so trajectories may part where E' and E are closer than FP32 can
tell; the tests compare what is unique (energies of the poses the GPU
returns, decisions with a clear margin, the closed-form minimum) and check
that the rest is valid (no energy ever rises).
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


def _pair_deck():
    # types A (donor) and B (acceptor) of the hand-worked table: the minimum
    # e = -2 lies at contact, d = R = 3 A, so E = -1
    return dict(lig_xyz=np.zeros((1, 3), np.float32), lig_type=np.array([0], np.int32),
                pro_xyz=np.zeros((1, 3), np.float32), pro_type=np.array([1], np.int32),
                radius=np.array([1.5, 1.5], np.float32), hardness=np.array([10, 30], np.float32),
                elsc=np.array([0.5, -0.5], np.float32), hbtype=np.array([1, 2], np.int32))


@pytest.mark.parametrize("variant", ["ieee", "fast"])
def test_refine_finds_the_single_pair_minimum(variant):
    D = _pair_deck()
    deck = bude.Deck(D, device=DEV)
    P = torch.zeros((6, 4), device=DEV)
    P[3] = torch.tensor([4.5, -5.0, 0.0, 0.0], device=DEV)
    P[4] = torch.tensor([0.0, 0.0, 3.7, 2.0], device=DEV)
    P[5] = torch.tensor([0.0, 0.0, 0.0, 2.9], device=DEV)
    E = bude.refine_device(deck, P, steps=80, step0=0.2, variant=variant)
    torch.cuda.synchronize()
    d = P[3:].norm(dim=0).cpu().numpy()
    assert np.all(np.abs(E.cpu().numpy() + 1.0) < 2e-3), E
    assert np.all((d > 2.95) & (d < 3.05)), d


def test_refine_energies_match_oracle_and_never_rise():
    D = synth.make_deck(140, 16, 400, 34, 300)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    E0 = bude.energies(deck, P).cpu().numpy()
    E = bude.refine_device(deck, P, steps=10, step0=0.05)
    torch.cuda.synchronize()
    Pf = P.cpu().numpy()
    E = E.cpu().numpy()
    ref, A = oracle.energies(D, Pf, n_threads=-1, with_abs=True)
    assert (np.abs(E - ref) / np.maximum(A, 1.0)).max() <= 1e-5
    assert np.all(E <= E0)
    assert np.mean(E) < np.mean(E0)
    # the oracle's own refinement from the same start lowers the energy by a
    # comparable amount
    _, Eo, _ = oracle.refine(D, D["poses"], steps=10, step0=0.05, n_threads=-1)
    e0 = oracle.energies(D, D["poses"], n_threads=-1)
    gpu_gain, ora_gain = np.mean(e0 - ref), np.mean(e0 - Eo)
    assert gpu_gain == pytest.approx(ora_gain, rel=0.05)


@pytest.mark.parametrize("step0", [0.05, 0.5, 2.0])
def test_one_step_decisions_agree_with_the_oracle(step0):
    D = synth.make_deck(141, 12, 300, 34, 400)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    bude.refine_device(deck, P, steps=1, step0=step0)
    torch.cuda.synchronize()
    Pg = P.cpu().numpy().astype(np.float64)
    P0 = D["poses"].astype(np.float64)
    E, G = oracle.pose_grad(D, P0, n_threads=-1)
    _, A = oracle.energies(D, P0, n_threads=-1, with_abs=True)
    norm = np.sqrt((G * G).sum(0))
    T = P0 - step0 * G / np.where(norm > 0, norm, 1.0)
    Et, At = oracle.energies(D, T, n_threads=-1, with_abs=True)
    band = 1e-5 * np.maximum(np.maximum(A, At), 1.0)
    accept = Et < E - band
    reject = Et > E + band
    assert accept.sum() + reject.sum() > 0.9 * len(E)
    moved = np.any(Pg != D["poses"].astype(np.float64), axis=0)
    assert np.all(moved[accept])
    assert np.all(~moved[reject])
    # an accepted step lands on the oracle's trial pose (up to the FP32
    # gradient direction)
    if accept.any():
        assert np.abs(Pg[:, accept] - T[:, accept]).max() < 1e-3 * max(step0, 1.0)
    if step0 >= 2.0:
        assert reject.sum() > 10       # large steps overshoot: the rule must refuse them
    if step0 <= 0.05:
        assert accept.sum() > 10


def test_refine_replay_continues_and_zero_steps_scores():
    D = synth.make_deck(142, 10, 300, 34, 200)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    E1 = bude.refine_device(deck, P, steps=5, step0=0.05).clone()
    assert bude.launch_count() == 2 + 3 * 5     # init, adjoint, then 3 per step
    E2 = bude.refine_device(deck, P, steps=5, step0=0.05).clone()   # graph replay
    torch.cuda.synchronize()
    assert torch.all(E2 <= E1)
    Q = P.clone()
    E0 = bude.refine_device(deck, Q, steps=0, step0=0.05)
    torch.testing.assert_close(Q, P)
    ref = bude.pose_grad(deck, P)[0]
    torch.testing.assert_close(E0, ref)
    empty = torch.zeros((6, 0), device=DEV)
    bude.refine_device(deck, empty, steps=3)
    with pytest.raises(bude.BudeError):
        bude.refine_device(deck, P, steps=-1)
    with pytest.raises(bude.BudeError):
        bude.refine_device(deck, P, steps=2, step0=0.0)


def test_refine_replay_after_the_deck_workspace_grows():
    # the captured refinement graph owns its workspace: a later call on the
    # deck that needs a larger one (the deck frees and reallocates its own)
    # leaves the replay unchanged, and memory taken after it stays untouched
    D = synth.make_deck(141, 16, 400, 34, 256)
    deck = bude.Deck(D, device=DEV)
    P0 = torch.from_numpy(D["poses"]).to(DEV)
    P, E = P0.clone(), torch.empty(P0.shape[1], device=DEV)
    bude.refine_device(deck, P, steps=4, step0=0.05, energies=E)       # captures
    first_P, first_E = P.clone(), E.clone()
    big = torch.from_numpy(synth.make_deck(142, 16, 400, 34, 200000)["poses"]).to(DEV)
    bude.energies(deck, big, ppwi=1)           # 6250 pose tiles: the deck's workspace grows
    fill = [torch.full((1 << 20,), 7.0, device=DEV) for _ in range(8)]
    P.copy_(P0)
    bude.refine_device(deck, P, steps=4, step0=0.05, energies=E)       # replays
    torch.cuda.synchronize()
    assert torch.equal(P, first_P) and torch.equal(E, first_E)
    assert all(bool((f == 7.0).all()) for f in fill)
