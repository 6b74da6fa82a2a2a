"""Pins for the Hartree-Fock oracle: closed forms of Gaussian electrostatics,
the Boys function against quadrature, integral symmetries and the
structure of G = sum_kl D_kl [2 (ij|kl) - (ik|jl)]."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_21039_gb300 import synth


def test_boys_function_against_quadrature():
    quad = pytest.importorskip("scipy.integrate").quad
    assert oracle.boys0(0.0) == 1.0
    for t in (1e-12, 1e-6, 0.1, 1.0, 7.5, 40.0, 300.0):
        ref = quad(lambda u: math.exp(-t * u * u), 0.0, 1.0, epsabs=1e-14, epsrel=1e-13)[0]
        assert oracle.boys0(t) == pytest.approx(ref, rel=1e-11)


def test_one_centre_primitive_integral():
    # four normalised s primitives of exponent x on one centre: 2 sqrt(x/pi)
    O = np.zeros(3)
    for x in (0.3, 1.0, 6.2):
        assert oracle.prim_eri(x, O, x, O, x, O, x, O) == pytest.approx(
            2.0 * math.sqrt(x / math.pi), rel=1e-13)


def test_two_gaussian_charge_clouds_interact_as_erf_over_r():
    # |phi_a|^2 and |phi_b|^2 are unit Gaussian charges of exponents 2a, 2b:
    # their repulsion is erf(sqrt(mu) R) / R with mu = (2a)(2b)/(2a + 2b)
    A = np.zeros(3)
    for a, b, R in ((0.5, 1.3, 0.7), (2.0, 0.4, 3.0), (1.0, 1.0, 10.0)):
        B = np.array([0.0, 0.0, R])
        mu = (2 * a) * (2 * b) / (2 * a + 2 * b)
        assert oracle.prim_eri(a, A, a, A, b, B, b, B) == pytest.approx(
            math.erf(math.sqrt(mu) * R) / R, rel=1e-12)


def test_contracted_far_field_is_point_charge():
    sysm = synth.make_he_lattice(1, 2, 3)
    x, c = sysm["xpnt"], sysm["coef"]
    A = np.zeros(3)
    # normalise the contraction so that (phi|phi) = 1
    S = sum(c[a] * c[b] * (2 * math.sqrt(x[a] * x[b]) / (x[a] + x[b])) ** 1.5
            for a in range(3) for b in range(3))
    cn = c / math.sqrt(S)
    B = np.array([0.0, 0.0, 40.0])
    assert oracle.eri(x, cn, A, A, B, B) == pytest.approx(1.0 / 40.0, rel=1e-9)


def test_eightfold_symmetry():
    rng = np.random.default_rng(3)
    x, c = np.array([3.0, 0.8, 0.35]), np.array([0.2, 0.5, 0.4])
    P = rng.uniform(-1.5, 1.5, size=(4, 3))
    v = oracle.eri(x, c, P[0], P[1], P[2], P[3])
    for (a, b, cc, d) in ((1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2), (2, 3, 0, 1), (3, 2, 0, 1),
                          (2, 3, 1, 0), (3, 2, 1, 0)):
        assert oracle.eri(x, c, P[a], P[b], P[cc], P[d]) == pytest.approx(v, rel=1e-13)


def test_fock_structure():
    s = synth.make_he_lattice(2, 5, 3)
    G = oracle.hf_fock(s["geom"], s["xpnt"], s["coef"], s["dens"])
    np.testing.assert_allclose(G, G.T, rtol=1e-13, atol=1e-13)
    # linear in D
    G2 = oracle.hf_fock(s["geom"], s["xpnt"], s["coef"], 2.5 * s["dens"])
    np.testing.assert_allclose(G2, 2.5 * G, rtol=1e-13, atol=1e-13)
    assert np.all(oracle.hf_fock(s["geom"], s["xpnt"], s["coef"], 0 * s["dens"]) == 0)
    # one atom: G_11 = D_11 (2 (11|11) - (11|11))
    g1 = s["geom"][:1]
    D1 = np.array([[0.7]])
    e = oracle.eri(s["xpnt"], s["coef"], g1[0], g1[0], g1[0], g1[0])
    assert oracle.hf_fock(g1, s["xpnt"], s["coef"], D1)[0, 0] == pytest.approx(0.7 * e, rel=1e-13)


# --- parity scale of the Fock term ----------------------------------------
#
# S_ij = sum_kl |D_kl| (2 |(ij|kl)| + |(ik|jl)|) bounds |G_ij| and every
# rounding of it; pinned by closed forms on one atom and on atoms far apart.

def test_fock_scale_bounds_g():
    s = synth.make_he_lattice(4, 6, 3)
    D = s["dens"] * np.random.default_rng(1).choice([-1.0, 1.0], size=s["dens"].shape)
    D = 0.5 * (D + D.T)
    G = oracle.hf_fock(s["geom"], s["xpnt"], s["coef"], D)
    S = oracle.hf_fock_scale(s["geom"], s["xpnt"], s["coef"], D)
    assert np.all(np.abs(G) <= S * (1 + 1e-13))
    assert np.any(S > 1.5 * np.abs(G))


def test_fock_scale_one_atom_is_three_times_g():
    # one primitive on one atom: G = D (00|00) and S = 3 |D| (00|00), with
    # (00|00) = 2 sqrt(x / pi) for a normalised primitive of exponent x
    x = 0.9
    g1 = np.zeros((1, 3))
    for d in (0.7, -0.4):
        D1 = np.array([[d]])
        G = oracle.hf_fock(g1, [x], [1.0], D1)[0, 0]
        S = oracle.hf_fock_scale(g1, [x], [1.0], D1)[0, 0]
        assert G == pytest.approx(d * 2 * math.sqrt(x / math.pi), rel=1e-13)
        assert S == pytest.approx(3 * abs(d) * 2 * math.sqrt(x / math.pi), rel=1e-13)


def test_fock_scale_far_apart_exchange_term():
    """Diagonal non-negative density on atoms 60 bohr apart: the exchange
    integrals (ik|ik) vanish for i != k, so S_ii - G_ii = 2 sum_k D_kk (ik|ik)
    = 2 D_ii (ii|ii), the one-centre closed form."""
    x = 1.3
    g = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 60.0], [0.0, 60.0, 0.0]])
    D = np.diag([0.3, 0.8, 0.5])
    G = oracle.hf_fock(g, [x], [1.0], D)
    S = oracle.hf_fock_scale(g, [x], [1.0], D)
    one = 2 * math.sqrt(x / math.pi)
    for i in range(3):
        assert S[i, i] - G[i, i] == pytest.approx(2 * D[i, i] * one, rel=1e-12)
