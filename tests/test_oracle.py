"""Pins for the FP64 oracle against facts that do not come from the oracle.

* hand-worked single-pair energies on every branch (tests/golden),
* textbook rotations and a library Euler routine for the pose transform,
* a brute-force assembly from library distances and rotations,
* invariances that hold for any correct implementation: joint rigid motion,
  atom permutations, type relabelling, ligand/protein translation duality,
* the cutoff (exact zero beyond it) and the scaling laws of each term,
* analytic derivatives against central finite differences.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2509_21039_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "single_pair_energy.txt")


def _load_golden():
    types, rows = {}, []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "type":
                types[tok[1]] = (float(tok[2]), float(tok[3]), float(tok[4]), int(tok[5]))
            else:
                rows.append((tok[0], tok[1], float(tok[2]), Fraction(tok[3])))
    return types, rows


def _single_pair_deck(ta, tb, d):
    return dict(
        lig_xyz=np.zeros((1, 3)), lig_type=np.array([0], np.int32),
        pro_xyz=np.array([[d, 0.0, 0.0]]), pro_type=np.array([1], np.int32),
        radius=np.array([ta[0], tb[0]]), hardness=np.array([ta[1], tb[1]]),
        elsc=np.array([ta[2], tb[2]]), hbtype=np.array([ta[3], tb[3]], np.int32))


GOLD_TYPES, GOLD_ROWS = _load_golden()


@pytest.mark.parametrize("a,b,d,expected", GOLD_ROWS,
                         ids=[f"{a}{b}-{d}" for a, b, d, _ in GOLD_ROWS])
def test_single_pair_closed_form(a, b, d, expected):
    ta, tb = GOLD_TYPES[a], GOLD_TYPES[b]
    # through the full pose/ligand/protein loop with the identity pose
    E = oracle.energies(_single_pair_deck(ta, tb, d), np.zeros((6, 1)))[0]
    assert E == pytest.approx(float(expected), rel=1e-14, abs=1e-14)
    # the pair function on its own, both argument orders (symmetric rules)
    assert 0.5 * oracle.pair_energy(ta, tb, d) == pytest.approx(float(expected), abs=1e-14)
    assert 0.5 * oracle.pair_energy(tb, ta, d) == pytest.approx(float(expected), abs=1e-14)


def test_single_pair_protein_on_any_axis():
    ta, tb = GOLD_TYPES["A"], GOLD_TYPES["D"]
    ref = 0.5 * oracle.pair_energy(ta, tb, 4.0)
    for v in ([0, 4.0, 0], [0, 0, -4.0], [4 / math.sqrt(3)] * 3):
        deck = _single_pair_deck(ta, tb, 0.0)
        deck["pro_xyz"] = np.array([v], np.float64)
        assert oracle.energies(deck, np.zeros((6, 1)))[0] == pytest.approx(ref, rel=1e-14)


# --- rotation -------------------------------------------------------------

def test_rotation_textbook_quarter_turns():
    h = math.pi / 2
    ex, ey, ez = np.eye(3)
    np.testing.assert_allclose(oracle.rotation(h, 0, 0) @ ey, ez, atol=1e-15)
    np.testing.assert_allclose(oracle.rotation(0, h, 0) @ ez, ex, atol=1e-15)
    np.testing.assert_allclose(oracle.rotation(0, 0, h) @ ex, ey, atol=1e-15)
    # composition order: first about x, then y, then z
    np.testing.assert_allclose(oracle.rotation(h, h, 0) @ ey, ex, atol=1e-15)
    np.testing.assert_allclose(oracle.rotation(0, h, h) @ ez, ey, atol=1e-15)


def test_rotation_first_element_matches_listing():
    # Listing 4 fills the first matrix entry with cy*cz
    rng = np.random.default_rng(3)
    for a in rng.uniform(-math.pi, math.pi, size=(20, 3)):
        R = oracle.rotation(*a)
        assert R[0, 0] == pytest.approx(math.cos(a[1]) * math.cos(a[2]), abs=1e-15)


def test_rotation_matches_library_euler():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(4)
    for a in rng.uniform(-math.pi, math.pi, size=(50, 3)):
        ref = Rot.from_euler("xyz", a).as_matrix()  # extrinsic x, y, z = Rz Ry Rx
        np.testing.assert_allclose(oracle.rotation(*a), ref, atol=1e-14)
        R = oracle.rotation(*a)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)


# --- assembly -------------------------------------------------------------

def _as64(deck):
    return {k: (np.asarray(v, np.float64) if v.dtype.kind == "f" else v)
            for k, v in deck.items()}


def test_brute_force_assembly_from_library_parts():
    """Sum over pairs built from scipy's rotation and distance routines and the
    (separately pinned) pair function; checks loops, type lookup and the 1/2."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    cdist = pytest.importorskip("scipy.spatial.distance").cdist
    D = synth.make_deck(11, 6, 40, 5, 12)
    ff = np.stack([D["radius"], D["hardness"], D["elsc"], D["hbtype"]], 1).astype(np.float64)
    E = oracle.energies(D, D["poses"])
    P = D["poses"].astype(np.float64)
    for k in range(P.shape[1]):
        R = Rot.from_euler("xyz", P[:3, k]).as_matrix()
        x = D["lig_xyz"].astype(np.float64) @ R.T + P[3:, k]
        dist = cdist(x, D["pro_xyz"].astype(np.float64))
        tot = 0.0
        for l in range(dist.shape[0]):
            for p in range(dist.shape[1]):
                tot += oracle.pair_energy(ff[D["lig_type"][l]], ff[D["pro_type"][p]], dist[l, p])
        assert E[k] == pytest.approx(0.5 * tot, rel=1e-12, abs=1e-12)


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def test_joint_rigid_motion_invariance():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(5)
    D = _as64(synth.make_deck(12, 10, 300, 8, 24))
    E0 = oracle.energies(D, D["poses"])
    assert np.count_nonzero(E0) > 0
    for trial in range(3):
        Q = _random_rotation(rng)
        c = rng.uniform(-10, 10, size=3)
        moved = dict(D)
        moved["pro_xyz"] = D["pro_xyz"] @ Q.T + c
        P = D["poses"].copy()
        for k in range(P.shape[1]):
            R = oracle.rotation(*P[:3, k])
            P[:3, k] = Rot.from_matrix(Q @ R).as_euler("xyz")
            P[3:, k] = Q @ P[3:, k] + c
        E1 = oracle.energies(moved, P)
        np.testing.assert_allclose(E1, E0, rtol=1e-9, atol=1e-9)


def test_permutation_invariance():
    rng = np.random.default_rng(6)
    D = _as64(synth.make_deck(13, 12, 200, 6, 16))
    E0 = oracle.energies(D, D["poses"])
    pl, pp = rng.permutation(12), rng.permutation(200)
    Dp = dict(D, lig_xyz=D["lig_xyz"][pl], lig_type=D["lig_type"][pl],
              pro_xyz=D["pro_xyz"][pp], pro_type=D["pro_type"][pp])
    np.testing.assert_allclose(oracle.energies(Dp, D["poses"]), E0, rtol=1e-12, atol=1e-12)


def test_type_relabelling_invariance():
    rng = np.random.default_rng(7)
    D = _as64(synth.make_deck(14, 12, 200, 9, 16))
    E0 = oracle.energies(D, D["poses"])
    perm = rng.permutation(9)          # new id of old type t is perm[t]
    inv = np.argsort(perm)
    Dr = dict(D, lig_type=perm[D["lig_type"]].astype(np.int32),
              pro_type=perm[D["pro_type"]].astype(np.int32),
              radius=D["radius"][inv], hardness=D["hardness"][inv],
              elsc=D["elsc"][inv], hbtype=D["hbtype"][inv])
    np.testing.assert_array_equal(oracle.energies(Dr, D["poses"]), E0)


def test_translation_duality():
    """Moving the ligand by +delta equals moving the protein by -delta."""
    D = _as64(synth.make_deck(15, 10, 300, 8, 16))
    delta = np.array([0.7, -1.3, 0.4])
    P = D["poses"].copy()
    P[3:] += delta[:, None]
    Dm = dict(D, pro_xyz=D["pro_xyz"] - delta)
    np.testing.assert_allclose(oracle.energies(D, P), oracle.energies(Dm, D["poses"]),
                               rtol=1e-11, atol=1e-11)


def test_cutoff_gives_exact_zero():
    D = _as64(synth.make_deck(16, 10, 300, 8, 8))
    rmax = 2 * D["radius"].max()
    reach = np.abs(D["lig_xyz"]).max() * math.sqrt(3)
    far = 20 + rmax + 4.0 + reach + 1e-3     # protein box half-width 20
    P = D["poses"].copy()
    P[3] = far
    P[4] = 0.0
    P[5] = 0.0
    assert np.all(oracle.energies(D, P) == 0.0)
    # and a single pair just inside / just outside R + 4
    ta, tb = GOLD_TYPES["A"], GOLD_TYPES["B"]
    assert oracle.pair_energy(ta, tb, 3.0 + 4.0) == 0.0
    assert oracle.pair_energy(ta, tb, 3.0 + 4.0 - 1e-3) != 0.0


def test_term_scaling_laws():
    D = _as64(synth.make_deck(17, 10, 300, 8, 12))
    D["hbtype"] = np.zeros_like(D["hbtype"])       # no desolvation, w = 1
    elec = dict(D, hardness=np.zeros_like(D["hardness"]))
    E1 = oracle.energies(elec, D["poses"])
    E3 = oracle.energies(dict(elec, elsc=3.0 * elec["elsc"]), D["poses"])
    np.testing.assert_allclose(E3, 9.0 * E1, rtol=1e-12, atol=1e-12)
    ster = dict(D, elsc=np.zeros_like(D["elsc"]))
    S1 = oracle.energies(ster, D["poses"])
    S2 = oracle.energies(dict(ster, hardness=2.5 * ster["hardness"]), D["poses"])
    np.testing.assert_allclose(S2, 2.5 * S1, rtol=1e-12, atol=1e-12)
    assert np.all(S1 >= 0.0)
    # the three terms add: full = steric-only + electrostatic-only (no polarity)
    np.testing.assert_allclose(oracle.energies(D, D["poses"]), S1 + E1, rtol=1e-12, atol=1e-12)


def test_desolvation_only_counts_polar_apolar_pairs():
    D = _as64(synth.make_deck(18, 10, 300, 8, 12))
    base = dict(D, hardness=np.zeros_like(D["hardness"]), elsc=np.zeros_like(D["elsc"]))
    for hb in (0, 1, 2):   # every type in one class: no polar/apolar pair
        assert np.all(oracle.energies(dict(base, hbtype=np.full(8, hb, np.int32)),
                                      D["poses"]) == 0.0)
    mixed = dict(base, hbtype=np.array([0, 1, 0, 2, 0, 1, 0, 2], np.int32))
    assert np.all(oracle.energies(mixed, D["poses"]) >= 0.0)


def test_rejects_out_of_range_types():
    D = _as64(synth.make_deck(19, 4, 10, 3, 2))
    bad = dict(D, pro_type=D["pro_type"].copy())
    bad["pro_type"][3] = 3
    with pytest.raises(ValueError):
        oracle.energies(bad, D["poses"])
    bad["pro_type"][3] = -1
    with pytest.raises(ValueError):
        oracle.energies(bad, D["poses"])


def test_empty_sizes():
    D = _as64(synth.make_deck(20, 4, 10, 3, 3))
    assert np.all(oracle.energies(dict(D, lig_xyz=np.zeros((0, 3)),
                                       lig_type=np.zeros(0, np.int32)), D["poses"]) == 0)
    assert np.all(oracle.energies(dict(D, pro_xyz=np.zeros((0, 3)),
                                       pro_type=np.zeros(0, np.int32)), D["poses"]) == 0)
    assert oracle.energies(D, np.zeros((6, 0))).shape == (0,)


def test_threads_do_not_change_results():
    D = synth.make_deck(21, 10, 200, 8, 64)
    np.testing.assert_array_equal(oracle.energies(D, D["poses"], n_threads=1),
                                  oracle.energies(D, D["poses"], n_threads=4))


# --- derivatives ----------------------------------------------------------

def test_pair_derivative_matches_finite_difference():
    h = 1e-6
    for a, b in (("A", "B"), ("A", "C"), ("A", "D"), ("E", "E")):
        ta, tb = GOLD_TYPES[a], GOLD_TYPES[b]
        R = ta[0] + tb[0]
        for d in np.linspace(0.3, R + 4.5, 41):
            if min(abs(d - R), abs(d - R - 2), abs(d - R - 4)) < 10 * h:
                continue
            fd = (oracle.pair_energy(ta, tb, d + h) - oracle.pair_energy(ta, tb, d - h)) / (2 * h)
            assert oracle.pair_denergy(ta, tb, d) == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_pose_gradient_matches_central_differences():
    D = _as64(synth.make_deck(22, 8, 120, 6, 20))
    P = D["poses"]
    E, G = oracle.pose_grad(D, P)
    np.testing.assert_allclose(E, oracle.energies(D, P), rtol=1e-13, atol=1e-13)
    h = 1e-4
    scale = np.maximum(np.abs(G).max(axis=0), 1.0)
    for j in range(6):
        Pp, Pm = P.copy(), P.copy()
        Pp[j] += h
        Pm[j] -= h
        fd = (oracle.energies(D, Pp) - oracle.energies(D, Pm)) / (2 * h)
        err = np.abs(fd - G[j]) / scale
        assert err.max() < 1e-4, (j, err.max())
        assert np.median(err) < 1e-6, (j, np.median(err))


def test_translation_gradient_is_minus_protein_force():
    """dE/dt equals -dE/d(shift of every protein atom): the duality above,
    differentiated."""
    D = _as64(synth.make_deck(23, 8, 150, 6, 10))
    _, G = oracle.pose_grad(D, D["poses"])
    h = 1e-5
    for i in range(3):
        dp = np.zeros(3)
        dp[i] = h
        Ep = oracle.energies(dict(D, pro_xyz=D["pro_xyz"] + dp), D["poses"])
        Em = oracle.energies(dict(D, pro_xyz=D["pro_xyz"] - dp), D["poses"])
        fd = (Ep - Em) / (2 * h)
        np.testing.assert_allclose(-fd, G[3 + i], rtol=1e-5, atol=1e-5)


def test_gradient_of_rotation_about_z_is_torque_component():
    """For the last angle, dE/da2 = z . sum_l (x'_l - t) x g_l, an identity of
    rotations about a fixed axis, checked through finite differences of the
    ligand coordinates (independent of the pose-gradient code)."""
    D = _as64(synth.make_deck(24, 6, 150, 6, 6))
    P = D["poses"]
    _, G = oracle.pose_grad(D, P)
    h = 1e-5
    for k in range(P.shape[1]):
        R = oracle.rotation(*P[:3, k])
        t = P[3:, k]
        xp = D["lig_xyz"] @ R.T + t
        tau = np.zeros(3)
        for l in range(xp.shape[0]):
            g = np.zeros(3)
            for i in range(3):
                # energy as a function of one posed ligand atom: identity pose,
                # ligand coordinates given directly
                lig = xp.copy()
                lig[l, i] += h
                Ep = oracle.energies(dict(D, lig_xyz=lig), np.zeros((6, 1)))[0]
                lig[l, i] -= 2 * h
                Em = oracle.energies(dict(D, lig_xyz=lig), np.zeros((6, 1)))[0]
                g[i] = (Ep - Em) / (2 * h)
            tau += np.cross(xp[l] - t, g)
        assert G[2, k] == pytest.approx(tau[2], rel=1e-5, abs=1e-5)


# --- refinement -------------------------------------------------------------

def test_refine_single_pair_reaches_the_contact_minimum():
    """Types A (donor) and B (acceptor): e = 20 (s/3)^2 [s<0] - 2 phi(s/4) has
    its minimum e = -2 at s = 0, i.e. d = R = 3, E = -1.  Starting at d = 4.5
    (E = -175/256) the refinement must approach d = 3 from above."""
    ta, tb = GOLD_TYPES["A"], GOLD_TYPES["B"]
    D = _single_pair_deck(ta, tb, 0.0)
    D["pro_xyz"] = np.array([[0.0, 0.0, 0.0]])
    P0 = np.zeros((6, 1))
    P0[3, 0] = 4.5                      # ligand atom at (4.5, 0, 0)
    P, E, alpha = oracle.refine(D, P0, steps=60, step0=0.2)
    d = np.linalg.norm(P[3:, 0])
    assert E[0] == pytest.approx(-1.0, abs=1e-3)
    assert 2.95 < d < 3.05
    # the energy never increases along the way
    prev = oracle.energies(D, P0)[0]
    for k in (1, 2, 5, 10, 30):
        _, Ek, _ = oracle.refine(D, P0, steps=k, step0=0.2)
        assert Ek[0] <= prev + 1e-15
        prev = Ek[0]


def test_refine_never_raises_energy_and_keeps_rejected_poses():
    D = _as64(synth.make_deck(25, 8, 150, 6, 12))
    E0 = oracle.energies(D, D["poses"])
    P, E, alpha = oracle.refine(D, D["poses"], steps=6, step0=0.05)
    assert np.all(E <= E0)
    np.testing.assert_allclose(oracle.energies(D, P), E, rtol=1e-12, atol=1e-12)
    # alpha is step0 times grow^a shrink^r with a + r = steps
    ratios = np.log(alpha / 0.05)
    for r in ratios:
        ok = any(abs(r - (a * np.log(1.25) + (6 - a) * np.log(0.5))) < 1e-9 for a in range(7))
        assert ok


# --- gradients with respect to ligand coordinates and forcefield ------------

def _weighted_energy(D, P, w):
    return float(np.dot(w, oracle.energies(D, P)))


def test_param_grad_ligand_coordinates_match_central_differences():
    D = _as64(synth.make_deck(30, 6, 150, 6, 10))
    w = np.random.default_rng(0).uniform(0.5, 1.5, 10)
    GL, _ = oracle.param_grad(D, D["poses"], w)
    h = 1e-5
    scale = max(np.abs(GL).max(), 1.0)
    for l in range(6):
        for i in range(3):
            Dp, Dm = dict(D), dict(D)
            Dp["lig_xyz"] = D["lig_xyz"].copy()
            Dm["lig_xyz"] = D["lig_xyz"].copy()
            Dp["lig_xyz"][l, i] += h
            Dm["lig_xyz"][l, i] -= h
            fd = (_weighted_energy(Dp, D["poses"], w) - _weighted_energy(Dm, D["poses"], w)) / (2 * h)
            assert abs(fd - GL[l, i]) <= 1e-5 * scale, (l, i, fd, GL[l, i])


@pytest.mark.parametrize("col,key", [(0, "radius"), (1, "hardness"), (2, "elsc")])
def test_param_grad_forcefield_matches_central_differences(col, key):
    D = _as64(synth.make_deck(31, 8, 200, 5, 12))
    w = np.random.default_rng(1).uniform(0.5, 1.5, 12)
    _, GF = oracle.param_grad(D, D["poses"], w)
    h = 1e-6
    scale = max(np.abs(GF[:, col]).max(), 1.0)
    for t in range(5):
        Dp, Dm = dict(D), dict(D)
        Dp[key] = D[key].copy()
        Dm[key] = D[key].copy()
        Dp[key][t] += h
        Dm[key][t] -= h
        fd = (_weighted_energy(Dp, D["poses"], w) - _weighted_energy(Dm, D["poses"], w)) / (2 * h)
        assert abs(fd - GF[t, col]) <= 1e-4 * scale, (key, t, fd, GF[t, col])


def test_param_grad_scaling_identities():
    """Energy is linear in hardness (steric) and quadratic in elsc
    (electrostatics): sum_t h_t dL/dh_t = L_steric and
    sum_t q_t dL/dq_t = 2 L_elec (Euler's theorem for homogeneous terms)."""
    D = _as64(synth.make_deck(32, 8, 200, 6, 9))
    D["hbtype"] = np.zeros_like(D["hbtype"])          # no desolvation
    P = D["poses"]
    _, GF = oracle.param_grad(D, P)
    L_ster = oracle.energies(dict(D, elsc=np.zeros_like(D["elsc"])), P).sum()
    L_elec = oracle.energies(dict(D, hardness=np.zeros_like(D["hardness"])), P).sum()
    assert np.dot(D["hardness"], GF[:, 1]) == pytest.approx(L_ster, rel=1e-10, abs=1e-10)
    assert np.dot(D["elsc"], GF[:, 2]) == pytest.approx(2 * L_elec, rel=1e-10, abs=1e-10)


# --- parity scales of the forcefield gradient ------------------------------
#
# oracle.param_grad(..., with_scale=True) also returns, per output element,
# the sum of its terms in absolute value (the bound on the rounding of any
# evaluation of that sum).  Pins: it bounds the gradient, it equals the
# gradient's magnitude where a single term makes up the element, it splits
# de/dd into its steric, electrostatic and desolvation parts, and it grows
# with |w|, not w.

def test_param_grad_scale_bounds_the_gradient():
    D = _as64(synth.make_deck(33, 7, 180, 6, 14))
    w = np.random.default_rng(5).uniform(-1.5, 1.5, 14)
    GL, GF, SL, SF = oracle.param_grad(D, D["poses"], w, with_scale=True)
    assert np.all(np.abs(GL) <= SL * (1 + 1e-12) + 1e-300)
    assert np.all(np.abs(GF) <= SF * (1 + 1e-12) + 1e-300)
    # with weights of both signs some elements cancel, so the bound is strict there
    assert np.any(SF > 1.01 * np.abs(GF))
    # the scale of w equals the scale of |w| and is linear in it
    _, _, SL2, SF2 = oracle.param_grad(D, D["poses"], np.abs(w), with_scale=True)
    np.testing.assert_allclose(SL2, SL, rtol=1e-14)
    np.testing.assert_allclose(SF2, SF, rtol=1e-14)
    _, _, SL3, SF3 = oracle.param_grad(D, D["poses"], 2.0 * w, with_scale=True)
    np.testing.assert_allclose(SL3, 2.0 * SL, rtol=1e-14)
    np.testing.assert_allclose(SF3, 2.0 * SF, rtol=1e-14)


def _pair_scale(ta, tb, d, w=None):
    D = _single_pair_deck(ta, tb, d)
    P = np.zeros((6, 1 if w is None else len(w)))
    return oracle.param_grad(D, P, w, with_scale=True)


@pytest.mark.parametrize("ta,tb,d", [
    ((1.5, 10.0, 0.0, 0), (1.5, 30.0, 0.0, 0), 2.0),    # steric only
    ((1.5, 0.0, 0.5, 1), (1.5, 0.0, -0.5, 2), 4.0),     # electrostatics only
    ((1.5, 0.0, 0.0, 1), (2.0, 0.0, 0.0, 0), 4.5),      # desolvation only
])
def test_param_grad_scale_equals_a_single_term(ta, tb, d):
    GL, GF, SL, SF = _pair_scale(ta, tb, d)
    np.testing.assert_allclose(SL, np.abs(GL), rtol=1e-14, atol=1e-300)
    np.testing.assert_allclose(SF, np.abs(GF), rtol=1e-14, atol=1e-300)
    assert SL[0, 0] > 0 and SL[0, 1] == 0 and SL[0, 2] == 0


def test_param_grad_scale_keeps_the_terms_apart():
    """Electrostatics (opposite charges) and desolvation both act at d = 4 and
    their derivatives have opposite signs: the scale is the sum of the two
    single-term magnitudes, the gradient only their difference."""
    both = ((1.5, 0.0, 0.5, 1), (1.5, 0.0, -0.5, 0))
    elec = ((1.5, 0.0, 0.5, 1), (1.5, 0.0, -0.5, 1))     # same Q w, no desolvation
    desolv = ((1.5, 0.0, 0.0, 1), (1.5, 0.0, 0.0, 0))    # same S, no charges
    d = 4.0
    de_el = oracle.pair_denergy(*elec, d)
    de_de = oracle.pair_denergy(*desolv, d)
    assert de_el > 0 > de_de
    GL, GF, SL, SF = _pair_scale(*both, d)
    assert SL[0, 0] == pytest.approx(0.5 * (abs(de_el) + abs(de_de)), rel=1e-14)
    assert abs(GL[0, 0]) == pytest.approx(0.5 * abs(de_el + de_de), rel=1e-14)
    for t in (0, 1):   # de/dR = -de/dd here (s > 0): the same two parts
        assert SF[t, 0] == pytest.approx(0.5 * (abs(de_el) + abs(de_de)), rel=1e-14)
    # de/dq_a = K_E w q_b phi(s/D_E): 4 * 1 * (-0.5) * phi(1/4) / 2, phi(1/4) = 0.84375
    assert GF[0, 2] == pytest.approx(-0.84375, rel=1e-14)
    assert SF[0, 2] == pytest.approx(0.84375, rel=1e-14)
    assert SF[1, 2] == pytest.approx(0.84375, rel=1e-14)
    assert SF[0, 1] == 0 and SF[1, 1] == 0       # no overlap: no hardness term


def test_param_grad_scale_counts_cancelling_poses():
    """The same pose twice with weights +1 and -1: the gradient cancels to 0,
    the scale is twice that of one pose."""
    ta, tb, d = (1.5, 10.0, 0.0, 0), (1.5, 30.0, 0.0, 0), 2.0
    GL1, GF1, SL1, SF1 = _pair_scale(ta, tb, d)
    GL, GF, SL, SF = _pair_scale(ta, tb, d, np.array([1.0, -1.0]))
    assert np.all(GL == 0) and np.all(GF == 0)
    np.testing.assert_allclose(SL, 2 * SL1, rtol=1e-14)
    np.testing.assert_allclose(SF, 2 * SF1, rtol=1e-14)
