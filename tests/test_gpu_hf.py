"""Hartree-Fock two-electron Fock term on the GPU against the oracle's plain
sum G_ij = sum_kl D_kl [2 (ij|kl) - (ik|jl)] (oracle pinned in
test_hf_oracle.py), element by element against each entry's own scale
S_ij = sum_kl |D_kl| (2 |(ij|kl)| + |(ik|jl)|) (the bound on the rounding of
any evaluation of the sum).  FP64 gate 1e-11 S_ij (atomics reorder the sum);
FP32-integral variant 1e-5 S_ij (primitive integrals rounded to FP32).  With
Schwarz screening at tol, every skipped unique quartet is below tol and
reaches an entry at most three times (once as Coulomb, twice as exchange),
so the screened entries may differ by a further 3 tol sum_kl |D_kl|."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_21039_gb300 import bude, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GATE = {"fp64": 1e-11, "ieee": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2509_21039_gb300 import build
    build.build()
    bude.load()


@pytest.mark.parametrize("n,ng", [(1, 3), (2, 1), (5, 3), (9, 2), (14, 3), (6, 4), (4, 8)])
@pytest.mark.parametrize("variant", ["fp64", "ieee"])
def test_fock_matches_oracle(n, ng, variant):
    s = synth.make_he_lattice(n, n, ng)
    G_ref = oracle.hf_fock(s["geom"], s["xpnt"], s["coef"], s["dens"])
    S = oracle.hf_fock_scale(s["geom"], s["xpnt"], s["coef"], s["dens"])
    hf = bude.HartreeFock(s["geom"], s["xpnt"], s["coef"], device=DEV)
    G = hf.fock(torch.from_numpy(s["dens"]).to(DEV), tol=0.0, variant=variant).cpu().numpy()
    assert np.all(S > 0)
    assert (np.abs(G - G_ref) / S).max() <= GATE[variant]
    np.testing.assert_array_equal(G, G.T)


def test_fock_sampled_entries_64_atoms_with_screening():
    s = synth.make_he_lattice(7, 64, 3)
    hf = bude.HartreeFock(s["geom"], s["xpnt"], s["coef"], device=DEV)
    D = torch.from_numpy(s["dens"]).to(DEV)
    G = hf.fock(D, tol=1e-12).cpu().numpy()
    G32 = hf.fock(D, tol=1e-12, variant="ieee").cpu().numpy()
    rng = np.random.default_rng(0)
    rows = rng.integers(0, 64, 16)
    cols = rng.integers(0, 64, 16)
    ref = oracle.hf_fock_entries(s["geom"], s["xpnt"], s["coef"], s["dens"], rows, cols)
    S = oracle.hf_fock_scale_entries(s["geom"], s["xpnt"], s["coef"], s["dens"], rows, cols)
    # skipped quartets are bounded by the Schwarz threshold
    screen = 3 * 1e-12 * np.abs(s["dens"]).sum()
    assert np.all(np.abs(G[rows, cols] - ref) <= GATE["fp64"] * S + screen)
    assert np.all(np.abs(G32[rows, cols] - ref) <= GATE["ieee"] * S + screen)


def test_fock_linear_in_density_and_rejects_bad_input():
    s = synth.make_he_lattice(8, 6, 3)
    hf = bude.HartreeFock(s["geom"], s["xpnt"], s["coef"], device=DEV)
    D = torch.from_numpy(s["dens"]).to(DEV)
    G1 = hf.fock(D, tol=0.0)
    G2 = hf.fock(3.0 * D, tol=0.0)
    torch.testing.assert_close(G2, 3.0 * G1, rtol=1e-12, atol=1e-14)
    assert torch.all(hf.fock(torch.zeros_like(D), tol=0.0) == 0)
    with pytest.raises(bude.BudeError):
        hf.fock(D, variant="fast")
    with pytest.raises(bude.BudeError):
        bude.HartreeFock(s["geom"], -s["xpnt"], s["coef"], device=DEV)


def test_surviving_quartet_count_matches_a_host_count():
    # the work list's size against a plain count over the unique quartets
    # (IJ >= KL) with the oracle's Schwarz bounds; thresholds a hair apart
    # bracket any product within rounding of the threshold
    s = synth.make_he_lattice(12, 20, 3)
    hf = bude.HartreeFock(s["geom"], s["xpnt"], s["coef"], device=DEV)
    g, x, c = s["geom"], s["xpnt"], s["coef"]
    Q = np.array([np.sqrt(abs(oracle.eri(x, c, g[i], g[j], g[i], g[j])))
                  for i in range(20) for j in range(i + 1)])
    m = len(Q)
    prod = Q[:, None] * Q[None, :]
    iu = np.tril_indices(m)
    assert hf.quartets(0.0) == m * (m + 1) // 2
    for tol in (1e-12, 1e-8, 1e-4):
        lo = int((prod[iu] >= tol * (1 + 1e-9)).sum())
        hi = int((prod[iu] >= tol * (1 - 1e-9)).sum())
        assert lo <= hf.quartets(tol) <= hi, tol
    with pytest.raises(bude.BudeError):
        hf.quartets(-1.0)
    hf.close()


@pytest.mark.parametrize("variant", ["fp64", "ieee"])
def test_everything_screened_gives_zero_and_screening_is_monotone(variant):
    # a threshold above every Schwarz product leaves no quartet (every warp's
    # range is empty) and G = 0
    s = synth.make_he_lattice(13, 12, 3)
    hf = bude.HartreeFock(s["geom"], s["xpnt"], s["coef"], device=DEV)
    D = torch.from_numpy(s["dens"]).to(DEV)
    assert hf.quartets(1e30) == 0
    G = hf.fock(D, tol=1e30, variant=variant)
    torch.cuda.synchronize()
    assert torch.all(G == 0)
    # the surviving set only grows as the threshold falls, to every unique
    # quartet at 0; a coarse threshold removes some and changes G
    counts = [hf.quartets(t) for t in (1e30, 1e-2, 1e-6, 1e-10, 0.0)]
    m = 12 * 13 // 2
    assert counts == sorted(counts) and counts[-1] == m * (m + 1) // 2
    full = hf.fock(D, tol=0.0, variant=variant).cpu().numpy()
    coarse = hf.fock(D, tol=1e-2, variant=variant).cpu().numpy()
    assert counts[1] < counts[-1]
    assert np.abs(coarse - full).max() > 1e-6 * np.abs(full).max()
    hf.close()
