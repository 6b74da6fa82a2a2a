"""bude_param_grad: gradient of sum_k w_k E_k with respect to the ligand
coordinates and the per-type forcefield parameters, against the oracle
(whose gradients are pinned by central differences in test_oracle.py).

Gate, per element: |g_gpu - g_ref| <= 1e-4 * S, where S is that element's
sum of its terms in absolute value (oracle.param_grad(..., with_scale=True)).
FP32 terms summed in FP32 over a run of protein atoms and the lane's poses,
then in FP64, stay within a small multiple of 2^-24 S; 1e-4 leaves room for
the approximate roots and sines of the FAST variant.  The floor 1e-9 of the
largest scale only keeps elements whose terms are all zero from dividing by
zero."""
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


def _err(g, ref, scale):
    """Largest per-element error against the element's own scale."""
    d = np.abs(np.asarray(g, np.float64) - ref)
    return float((d / np.maximum(scale, 1e-9 * max(scale.max(), 1e-300))).max())


@pytest.mark.parametrize("variant", ["ieee", "fast"])
@pytest.mark.parametrize("ppwi,block,tile", [(8, 256, 0), (4, 128, 0), (2, 512, 97), (1, 64, 0)])
def test_param_grad_matches_oracle(variant, ppwi, block, tile):
    D = synth.make_deck(160, 14, 350, 12, 600)
    w = np.random.default_rng(2).uniform(0.0, 2.0, 600).astype(np.float32)
    GL, GF, SL, SF = oracle.param_grad(D, D["poses"], w.astype(np.float64), with_scale=True)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    gl, gf = bude.param_grad(deck, P, torch.from_numpy(w).to(DEV), variant=variant,
                             ppwi=ppwi, block=block, tile=tile)
    torch.cuda.synchronize()
    assert _err(gl.cpu().numpy(), GL, SL) <= 1e-4
    for col in range(3):
        assert _err(gf.cpu().numpy()[:, col], GF[:, col], SF[:, col]) <= 1e-4, col


def test_param_grad_unit_weights_full_types_and_repeat():
    D = synth.make_deck(161, 30, 900, 34, 2000)
    GL, GF, SL, SF = oracle.param_grad(D, D["poses"], with_scale=True)
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    gl, gf = bude.param_grad(deck, P)
    gl2, gf2 = bude.param_grad(deck, P)
    torch.cuda.synchronize()
    assert _err(gl.cpu().numpy(), GL, SL) <= 1e-4
    for col in range(3):
        assert _err(gf.cpu().numpy()[:, col], GF[:, col], SF[:, col]) <= 1e-4
    torch.testing.assert_close(gl2, gl, rtol=1e-6, atol=1e-6)
    torch.testing.assert_close(gf2, gf, rtol=1e-6, atol=1e-6)


def test_param_grad_scaling_identity_on_gpu():
    # sum_t h_t dL/dh_t equals the steric energy (energy is linear in hardness)
    D = synth.make_deck(162, 10, 300, 8, 500)
    D["hbtype"] = np.zeros_like(D["hbtype"])
    D["elsc"] = np.zeros_like(D["elsc"])
    deck = bude.Deck(D, device=DEV)
    P = torch.from_numpy(D["poses"]).to(DEV)
    _, gf = bude.param_grad(deck, P)
    E = bude.energies(deck, P).double().sum().item()
    lhs = float(np.dot(D["hardness"].astype(np.float64), gf.cpu().numpy()[:, 1]))
    assert lhs == pytest.approx(E, rel=1e-4)


def test_param_grad_edge_cases():
    D = synth.make_deck(163, 5, 60, 6, 10)
    deck = bude.Deck(D, device=DEV)
    gl, gf = bude.param_grad(deck, torch.zeros((6, 0), device=DEV))
    assert torch.all(gl == 0) and torch.all(gf == 0)
    E = dict(D, pro_xyz=D["pro_xyz"][:0], pro_type=D["pro_type"][:0])
    deck2 = bude.Deck(E, device=DEV)
    gl, gf = bude.param_grad(deck2, torch.from_numpy(D["poses"]).to(DEV))
    assert torch.all(gl == 0) and torch.all(gf == 0)
    with pytest.raises(bude.BudeError):
        bude.param_grad(deck, torch.from_numpy(D["poses"]).to(DEV), variant="fp64")
