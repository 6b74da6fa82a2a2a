"""Seeded synthetic docking inputs shaped like the miniBUDE benchmark decks.

This module only draws random numbers: it holds none of the energy
arithmetic and serves the CUDA path and the oracle alike.  The real ``bm1``
deck files are not available, so these decks stand in for them with the
shapes and distributions of the benchmark configurations:

* protein atoms uniform in [-20, 20]^3 Angstrom, ligand atoms in [-4, 4]^3,
* atom types uniform in {0, .., n_types-1},
* per type: radius U[1.4, 2.2], hardness U[0, 40], elsc U[-1, 1],
  hbtype uniform in {0 none, 1 donor, 2 acceptor},
* poses: three angles U[-pi, pi], three translations U[-5, 5].

Draw order (fixed so every consumer sees the same bits): protein xyz,
protein types, ligand xyz, ligand types, radius, hardness, elsc, hbtype,
angles, translations.  Coordinates, parameters and poses are float32, types
int32.
"""
from __future__ import annotations

import math

import numpy as np

DECK_KEYS = ("lig_xyz", "lig_type", "pro_xyz", "pro_type", "radius",
             "hardness", "elsc", "hbtype")


def make_deck(seed, n_lig: int, n_pro: int, n_types: int, n_poses: int):
    """One deck plus its poses.  ``seed`` is an int or a sequence of ints.

    Returns a dict with the eight deck arrays of ``DECK_KEYS`` and ``poses``
    (float32 [6][n_poses]: angles 0..2 then translations 0..2).
    """
    rng = np.random.default_rng(seed)
    f32 = np.float32
    pro_xyz = rng.uniform(-20.0, 20.0, size=(n_pro, 3)).astype(f32)
    pro_type = rng.integers(0, n_types, size=n_pro, dtype=np.int64).astype(np.int32)
    lig_xyz = rng.uniform(-4.0, 4.0, size=(n_lig, 3)).astype(f32)
    lig_type = rng.integers(0, n_types, size=n_lig, dtype=np.int64).astype(np.int32)
    radius = rng.uniform(1.4, 2.2, size=n_types).astype(f32)
    hardness = rng.uniform(0.0, 40.0, size=n_types).astype(f32)
    elsc = rng.uniform(-1.0, 1.0, size=n_types).astype(f32)
    hbtype = rng.integers(0, 3, size=n_types, dtype=np.int64).astype(np.int32)
    angles = rng.uniform(-math.pi, math.pi, size=(3, n_poses)).astype(f32)
    trans = rng.uniform(-5.0, 5.0, size=(3, n_poses)).astype(f32)
    poses = np.ascontiguousarray(np.concatenate([angles, trans], axis=0))
    return dict(lig_xyz=lig_xyz, lig_type=lig_type, pro_xyz=pro_xyz,
                pro_type=pro_type, radius=radius, hardness=hardness, elsc=elsc,
                hbtype=hbtype, poses=poses)


def log_uniform_int(rng, lo: int, hi: int) -> int:
    """Integer drawn log-uniformly from [lo, hi]."""
    v = math.exp(rng.uniform(math.log(lo), math.log(hi)))
    return int(min(hi, max(lo, round(v))))


def batched_shapes(seed: int, count: int, lig=(8, 128), pro=(500, 5000),
                   poses=(1024, 65536)):
    """Per-instance (n_lig, n_pro, n_poses) drawn log-uniformly, seeded."""
    rng = np.random.default_rng([seed, 0x5EED])
    out = []
    for _ in range(count):
        out.append((log_uniform_int(rng, *lig), log_uniform_int(rng, *pro),
                    log_uniform_int(rng, *poses)))
    return out


def make_batched(seed: int, count: int = 64, n_types: int = 34, **ranges):
    """``count`` uneven decks; deck i is ``make_deck((seed, i), ...)``."""
    shapes = batched_shapes(seed, count, **ranges)
    return [make_deck([seed, i], nl, npro, n_types, npose)
            for i, (nl, npro, npose) in enumerate(shapes)]


# Benchmark workloads: (n_lig, n_pro, n_types, n_poses)
SMALL = dict(n_lig=26, n_pro=938, n_types=34, n_poses=4096)      # 26 x 938 x 4096, seed 0
FULL = dict(n_lig=64, n_pro=2672, n_types=34, n_poses=65536)     # 64 x 2672 x 65536
GRAD = dict(n_lig=64, n_pro=2672, n_types=34, n_poses=16384)     # pose-gradient deck


def make_he_lattice(seed, n_atoms: int, ngauss: int = 3, spacing: float = 3.0):
    """Synthetic helium-like system for the Hartree-Fock Fock build: atoms on
    a simple cubic lattice (``spacing`` bohr, jittered by U[-0.2, 0.2]), one
    s function per atom contracted from ``ngauss`` primitives with exponents
    log-uniform in [0.3, 7] and coefficients U[0.1, 0.6], and a smooth
    symmetric density D_ij = 0.5 exp(-|R_i - R_j|^2 / 8) (float64 arrays).
    Draw order: jitter, exponents, coefficients."""
    rng = np.random.default_rng(seed)
    side = int(math.ceil(n_atoms ** (1.0 / 3.0)))
    grid = np.array([(i, j, k) for i in range(side) for j in range(side)
                     for k in range(side)][:n_atoms], np.float64) * spacing
    geom = grid + rng.uniform(-0.2, 0.2, size=grid.shape)
    xpnt = np.sort(np.exp(rng.uniform(math.log(0.3), math.log(7.0), size=ngauss)))[::-1].copy()
    coef = rng.uniform(0.1, 0.6, size=ngauss)
    d2 = ((geom[:, None, :] - geom[None, :, :]) ** 2).sum(-1)
    dens = 0.5 * np.exp(-d2 / 8.0)
    return dict(geom=geom, xpnt=xpnt, coef=coef, dens=dens)
