"""The diagnostic build (libbude_debug.so, BUDE_DEVICE_CHECKS) on every call
path: its device-side bounds checks (shared-memory carve-up, protein chunk,
table row, protein type, partial-sum slot, tile ticket, instance search)
must stay silent on valid inputs, and its results must match the oracle.

Runs in a child process so the diagnostic library is the only one loaded.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
import oracle
from paper_2509_21039_gb300 import bude, synth
assert bude.load()._name.endswith("libbude_debug.so")
dev = "cuda:0"
def err(E, D, P):
    ref, A = oracle.energies(D, P, n_threads=-1, with_abs=True)
    return float((np.abs(E.cpu().numpy() - ref) / np.maximum(A, 1)).max())
D = synth.make_deck(150, 20, 700, 34, 1500)
deck = bude.Deck(D, device=dev)
P = torch.from_numpy(D["poses"]).to(dev)
for v, p in (("ieee", 16), ("fast", 8), ("comp", 4), ("fp64", 2), ("ieee", 1)):
    assert err(bude.energies(deck, P, variant=v, ppwi=p, block=256), D, D["poses"]) < 1e-5
assert err(bude.energies(deck, P, ppwi=4, block=128, tile=96, ctas_per_sm=3), D, D["poses"]) < 1e-5
E, G = bude.pose_grad(deck, P, ppwi=4, block=128, tile=200)
assert err(E, D, D["poses"]) < 1e-5
out = torch.empty(P.shape[1], device=dev)
assert err(bude.energies_noalloc(deck, P, out), D, D["poses"]) < 1e-5
decks_np = [synth.make_deck([8, i], nl, npro, 34, n)
            for i, (nl, npro, n) in enumerate([(8, 500, 300), (30, 4500, 700), (3, 40, 1)])]
decks = [bude.Deck(d, device=dev) for d in decks_np]
poses = [torch.from_numpy(d["poses"]).to(dev) for d in decks_np]
for d, o in zip(decks_np, bude.energies_batched(decks, poses, ppwi=16, block=384)):
    assert err(o, d, d["poses"]) < 1e-5
Q = P.clone()
E = bude.refine_device(deck, Q, steps=3, step0=0.05)
assert err(E, D, Q.cpu().numpy()) < 1e-5
gl, gf = bude.param_grad(deck, P, ppwi=4, block=128, tile=150)
GL, GF = oracle.param_grad(D, D["poses"])
assert float(np.abs(gl.cpu().numpy() - GL).max()) <= 1e-4 * max(np.abs(GL).max(), 1)
assert float(np.abs(gf.cpu().numpy() - GF).max()) <= 1e-4 * max(np.abs(GF).max(), 1)
print("device checks silent")
'''


def test_diagnostic_build_is_silent_on_valid_inputs():
    from paper_2509_21039_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, BUDE_LIB=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "device checks silent" in r.stdout
