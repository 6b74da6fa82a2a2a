"""FP64 CPU oracle for the miniBUDE pose energy (arxiv 2509.21039, Sec. 2.2,
Listing 4, Eq. 3) -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
has no fallback to it.  The arithmetic lives in ``bude_oracle.c`` (plain C,
double precision, a triple loop over poses, ligand atoms and protein atoms);
this module only compiles it with gcc and marshals numpy arrays through
ctypes.  The pair energy it evaluates is the project's own definition (the
paper never writes the forcefield down); ``bude_oracle.c`` states it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "bude_oracle.c"), os.path.join(_HERE, "hf_oracle.c")]
_LIB = os.path.join(_HERE, "libbude_oracle.so")
_lock = threading.Lock()
_lib = None

# gcc flags: no fast-math, no contraction, no target-specific flags, so x86
# and Arm hosts round identically.
_CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile ``bude_oracle.c`` into ``libbude_oracle.so`` (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and all(os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *_CFLAGS, *_SRCS, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        i64 = ctypes.c_int64
        ci = ctypes.c_int
        cd = ctypes.c_double
        lib.oracle_pair_energy.restype = cd
        lib.oracle_pair_energy.argtypes = [cd, cd, cd, ci, cd, cd, cd, ci, cd]
        lib.oracle_pair_denergy.restype = cd
        lib.oracle_pair_denergy.argtypes = [cd, cd, cd, ci, cd, cd, cd, ci, cd]
        lib.oracle_rotation.restype = None
        lib.oracle_rotation.argtypes = [cd, cd, cd, dp]
        deck_args = [ci, dp, ip, ci, dp, ip, ci, dp, dp, dp, ip]
        lib.oracle_energies.restype = ci
        lib.oracle_energies.argtypes = deck_args + [i64, dp, dp, dp, ci]
        lib.oracle_pose_grad.restype = ci
        lib.oracle_pose_grad.argtypes = deck_args + [i64, dp, dp, dp, dp, ci]
        lib.oracle_param_grad.restype = ci
        lib.oracle_param_grad.argtypes = deck_args + [i64, dp, dp, dp, dp]
        lib.oracle_param_grad_scale.restype = ci
        lib.oracle_param_grad_scale.argtypes = deck_args + [i64, dp, dp, dp, dp]
        lib.oracle_boys0.restype = cd
        lib.oracle_boys0.argtypes = [cd]
        lib.oracle_prim_eri.restype = cd
        lib.oracle_prim_eri.argtypes = [cd, dp, cd, dp, cd, dp, cd, dp]
        lib.oracle_eri.restype = cd
        lib.oracle_eri.argtypes = [ci, dp, dp, dp, dp, dp, dp]
        lib.oracle_hf_fock_entries.restype = None
        lib.oracle_hf_fock_entries.argtypes = [ci, dp, ci, dp, dp, dp, ci, ip, ip, dp]
        lib.oracle_hf_fock_scale_entries.restype = None
        lib.oracle_hf_fock_scale_entries.argtypes = [ci, dp, ci, dp, dp, dp, ci, ip, ip, dp]
        lib.oracle_max_threads.restype = ci
        lib.oracle_max_threads.argtypes = []
        _lib = lib
        return lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def max_threads() -> int:
    """OpenMP threads the oracle uses when asked for all cores."""
    return int(_load().oracle_max_threads())


def pair_energy(ff_a, ff_b, d: float) -> float:
    """e(a, b, d) for per-type rows ``(radius, hardness, elsc, hbtype)``."""
    ra, ha, qa, hba = ff_a
    rb, hb, qb, hbb = ff_b
    return float(_load().oracle_pair_energy(ra, ha, qa, int(hba), rb, hb, qb,
                                            int(hbb), float(d)))


def pair_denergy(ff_a, ff_b, d: float) -> float:
    """de/dd for per-type rows ``(radius, hardness, elsc, hbtype)``."""
    ra, ha, qa, hba = ff_a
    rb, hb, qb, hbb = ff_b
    return float(_load().oracle_pair_denergy(ra, ha, qa, int(hba), rb, hb, qb,
                                             int(hbb), float(d)))


def rotation(a0: float, a1: float, a2: float) -> np.ndarray:
    """R = Rz(a2) Ry(a1) Rx(a0) as a 3x3 float64 array."""
    out = np.zeros(9, np.float64)
    _load().oracle_rotation(float(a0), float(a1), float(a2), _dptr(out))
    return out.reshape(3, 3)


def _deck_args(deck):
    lig = np.ascontiguousarray(deck["lig_xyz"], np.float64).reshape(-1, 3)
    pro = np.ascontiguousarray(deck["pro_xyz"], np.float64).reshape(-1, 3)
    lt = np.ascontiguousarray(deck["lig_type"], np.int32)
    pt = np.ascontiguousarray(deck["pro_type"], np.int32)
    rad = np.ascontiguousarray(deck["radius"], np.float64)
    hard = np.ascontiguousarray(deck["hardness"], np.float64)
    elsc = np.ascontiguousarray(deck["elsc"], np.float64)
    hbt = np.ascontiguousarray(deck["hbtype"], np.int32)
    keep = (lig, pro, lt, pt, rad, hard, elsc, hbt)
    args = [len(lt), _dptr(lig), _iptr(lt), len(pt), _dptr(pro), _iptr(pt),
            len(rad), _dptr(rad), _dptr(hard), _dptr(elsc), _iptr(hbt)]
    return args, keep


def energies(deck, poses, n_threads: int = 0, with_abs: bool = False):
    """Per-pose energies (float64) of ``poses`` ([6][n]) on ``deck``.

    ``deck`` is a mapping with lig_xyz, lig_type, pro_xyz, pro_type, radius,
    hardness, elsc, hbtype.  ``n_threads`` 0 runs one thread, -1 all cores.
    With ``with_abs`` also returns 0.5 * sum |e| per pose (the error scale).
    """
    lib = _load()
    args, keep = _deck_args(deck)
    P = np.ascontiguousarray(poses, np.float64).reshape(6, -1)
    n = P.shape[1]
    E = np.zeros(n, np.float64)
    A = np.zeros(n, np.float64)
    nt = lib.oracle_max_threads() if n_threads < 0 else n_threads
    rc = lib.oracle_energies(*args, n, _dptr(P), _dptr(E), _dptr(A), nt)
    del keep
    if rc != 0:
        raise ValueError("oracle_energies rejected the deck (type out of range "
                         "or negative size)")
    return (E, A) if with_abs else E


def pose_grad(deck, poses, n_threads: int = 0, with_scale: bool = False):
    """(energies [n], dE/dpose [6][n]) in float64 from the analytic chain rule.

    With ``with_scale`` also returns [2][n] error scales: 0.5 sum |e'| |r| for
    the angle rows and 0.5 sum |e'| for the translation rows.
    """
    lib = _load()
    args, keep = _deck_args(deck)
    P = np.ascontiguousarray(poses, np.float64).reshape(6, -1)
    n = P.shape[1]
    E = np.zeros(n, np.float64)
    G = np.zeros((6, n), np.float64)
    S = np.zeros((2, n), np.float64)
    nt = lib.oracle_max_threads() if n_threads < 0 else n_threads
    rc = lib.oracle_pose_grad(*args, n, _dptr(P), _dptr(E), _dptr(G), _dptr(S), nt)
    del keep
    if rc != 0:
        raise ValueError("oracle_pose_grad rejected the deck")
    return (E, G, S) if with_scale else (E, G)


def param_grad(deck, poses, weights=None, with_scale: bool = False):
    """Gradient of L = sum_k w_k E_k (float64): (dL/d ligand xyz [n_lig][3],
    dL/d (radius, hardness, elsc) [n_types][3]).  With with_scale, also the
    per-element sums of the absolute values of the terms of each output
    (oracle_param_grad_scale), same shapes: (GL, GF, SL, SF)."""
    lib = _load()
    args, keep = _deck_args(deck)
    P = np.ascontiguousarray(poses, np.float64).reshape(6, -1)
    n = P.shape[1]
    w = None if weights is None else np.ascontiguousarray(weights, np.float64)
    wp = _dptr(w) if w is not None else None
    GL = np.zeros((len(deck["lig_type"]), 3), np.float64)
    GF = np.zeros((len(deck["radius"]), 3), np.float64)
    rc = lib.oracle_param_grad(*args, n, _dptr(P), wp, _dptr(GL), _dptr(GF))
    if rc == 0 and with_scale:
        SL = np.zeros_like(GL)
        SF = np.zeros_like(GF)
        rc = lib.oracle_param_grad_scale(*args, n, _dptr(P), wp, _dptr(SL), _dptr(SF))
    del keep
    if rc != 0:
        raise ValueError("oracle_param_grad rejected the deck")
    return (GL, GF, SL, SF) if with_scale else (GL, GF)


# --- pose refinement (the docking step after scoring) ----------------------

def refine(deck, poses, steps: int, step0: float, grow: float = 1.25, shrink: float = 0.5,
           n_threads: int = 0):
    """Per-pose normalised gradient descent with an adaptive step, in FP64.

    The rule both the oracle and the CUDA path follow (this project's reading
    of the refinement that docking performs after scoring; the paper stops at
    the energy):
      start: E, g = energy and pose gradient at p; alpha = step0
      each step:  if |g| > 0:  p' = p - alpha g / |g|, else p' = p
                  E', g' at p'
                  if E' < E:  p, E, g = p', E', g';  alpha *= grow
                  else:       alpha *= shrink
    Returns (poses [6][n], energies [n], alpha [n]).
    """
    P = np.array(poses, dtype=np.float64).reshape(6, -1)
    E, G = pose_grad(deck, P, n_threads=n_threads)
    alpha = np.full(P.shape[1], float(step0))
    for _ in range(steps):
        norm = np.sqrt((G * G).sum(axis=0))
        move = norm > 0
        T = P.copy()
        T[:, move] = P[:, move] - alpha[move] * G[:, move] / norm[move]
        Et, Gt = pose_grad(deck, T, n_threads=n_threads)
        acc = Et < E
        P[:, acc] = T[:, acc]
        E[acc] = Et[acc]
        G[:, acc] = Gt[:, acc]
        alpha = np.where(acc, alpha * grow, alpha * shrink)
    return P, E, alpha


# --- Hartree-Fock two-electron Fock term (s-type Gaussians) -----------------

def boys0(t: float) -> float:
    """F0(t) = (1/2) sqrt(pi/t) erf(sqrt t), F0(0) = 1."""
    return float(_load().oracle_boys0(float(t)))


def prim_eri(xa, A, xb, B, xc, C, xd, D) -> float:
    """Normalised primitive two-electron integral (ab|cd)."""
    v = [np.ascontiguousarray(X, np.float64) for X in (A, B, C, D)]
    return float(_load().oracle_prim_eri(float(xa), _dptr(v[0]), float(xb), _dptr(v[1]),
                                         float(xc), _dptr(v[2]), float(xd), _dptr(v[3])))


def eri(xpnt, coef, A, B, C, D) -> float:
    """Contracted (ij|kl) for s functions on centres A, B, C, D."""
    x = np.ascontiguousarray(xpnt, np.float64)
    c = np.ascontiguousarray(coef, np.float64)
    v = [np.ascontiguousarray(X, np.float64) for X in (A, B, C, D)]
    return float(_load().oracle_eri(len(x), _dptr(x), _dptr(c), *[_dptr(t) for t in v]))


def hf_fock_entries(geom, xpnt, coef, dens, rows, cols):
    """G_ij = sum_kl D_kl [2 (ij|kl) - (ik|jl)] for the listed (i, j)."""
    g = np.ascontiguousarray(geom, np.float64).reshape(-1, 3)
    n = g.shape[0]
    x = np.ascontiguousarray(xpnt, np.float64)
    c = np.ascontiguousarray(coef, np.float64)
    d = np.ascontiguousarray(dens, np.float64).reshape(n, n)
    r = np.ascontiguousarray(rows, np.int32)
    k = np.ascontiguousarray(cols, np.int32)
    out = np.zeros(len(r), np.float64)
    _load().oracle_hf_fock_entries(n, _dptr(g), len(x), _dptr(x), _dptr(c), _dptr(d), len(r),
                                   _iptr(r), _iptr(k), _dptr(out))
    return out


def hf_fock_scale_entries(geom, xpnt, coef, dens, rows, cols):
    """S_ij = sum_kl |D_kl| (2 |(ij|kl)| + |(ik|jl)|) for the listed (i, j):
    the sum of G_ij's terms in absolute value."""
    g = np.ascontiguousarray(geom, np.float64).reshape(-1, 3)
    n = g.shape[0]
    x = np.ascontiguousarray(xpnt, np.float64)
    c = np.ascontiguousarray(coef, np.float64)
    d = np.ascontiguousarray(dens, np.float64).reshape(n, n)
    r = np.ascontiguousarray(rows, np.int32)
    k = np.ascontiguousarray(cols, np.int32)
    out = np.zeros(len(r), np.float64)
    _load().oracle_hf_fock_scale_entries(n, _dptr(g), len(x), _dptr(x), _dptr(c), _dptr(d),
                                         len(r), _iptr(r), _iptr(k), _dptr(out))
    return out


def hf_fock_scale(geom, xpnt, coef, dens):
    """The full S matrix of hf_fock_scale_entries (small systems)."""
    n = np.asarray(geom).reshape(-1, 3).shape[0]
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return hf_fock_scale_entries(geom, xpnt, coef, dens, ii.ravel(), jj.ravel()).reshape(n, n)


def hf_fock(geom, xpnt, coef, dens):
    """The full G matrix by the plain definition (small systems)."""
    n = np.asarray(geom).reshape(-1, 3).shape[0]
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return hf_fock_entries(geom, xpnt, coef, dens, ii.ravel(), jj.ravel()).reshape(n, n)
