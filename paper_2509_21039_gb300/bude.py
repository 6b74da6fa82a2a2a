"""ctypes binding of libbude.so (C ABI in include/bude.h).

Argument marshalling only: tensors are checked for device, dtype, shape and
contiguity and their pointers handed to the library, which runs every step
of the energy evaluation in its own CUDA kernels.  PyTorch supplies device
memory and streams.  There is no fallback: if ``libbude.so`` is missing or a
call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbude.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "bude.h")

OK = 0
ERR_INVALID_ARG = -1
ERR_CUDA = -2
ERR_OOM = -3
ERR_UNSUPPORTED = -4
ERR_DEVICE_FLAG = -5

FP32_IEEE = 0
FP32_FAST = 1
FP32_COMP = 2
FP64 = 3
VARIANTS = {"ieee": FP32_IEEE, "fast": FP32_FAST, "comp": FP32_COMP, "fp64": FP64}
MAX_TYPES = 1024


class BudeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} ({code})")
        self.code = code


class DeckDesc(ctypes.Structure):
    _fields_ = [("n_lig", ctypes.c_int32), ("n_pro", ctypes.c_int32),
                ("n_types", ctypes.c_int32), ("lig_xyzt", ctypes.c_void_p),
                ("pro_xyzt", ctypes.c_void_p), ("ff", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("ppwi", ctypes.c_int32),
                ("block", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("cull", ctypes.c_int32)]


_lib = None


def load(path: str | None = None):
    """Load libbude.so (raises if it has not been built).  The environment
    variable BUDE_LIB selects another build of it, e.g. libbude_debug.so."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = os.environ.get("BUDE_LIB", LIB_PATH)
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    ci = ctypes.c_int
    sig = {
        "bude_create_deck": (ci, [ctypes.POINTER(DeckDesc), vp, ctypes.POINTER(vp)]),
        "bude_destroy_deck": (ci, [vp]),
        "bude_deck_info": (ci, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "bude_energies": (ci, [vp, vp, i64, vp, ctypes.POINTER(Options), vp]),
        "bude_energies_noalloc": (ci, [vp, vp, i64, vp, ctypes.POINTER(Options), vp]),
        "bude_energies_host": (ci, [vp, vp, i64, vp, ctypes.POINTER(Options), vp]),
        "bude_energies_batched": (ci, [ctypes.POINTER(vp), ctypes.POINTER(vp),
                                       ctypes.POINTER(i64), ctypes.POINTER(vp), i32,
                                       ctypes.POINTER(Options), vp]),
        "bude_pose_grad": (ci, [vp, vp, i64, vp, vp, ctypes.POINTER(Options), vp]),
        "bude_refine": (ci, [vp, vp, i64, i32, ctypes.c_float, vp, ctypes.POINTER(Options), vp]),
        "bude_param_grad": (ci, [vp, vp, i64, vp, vp, vp, ctypes.POINTER(Options), vp]),
        "bude_stream": (ci, [i32, i32, vp, vp, vp, ctypes.c_double, i64, vp, vp]),
        "bude_hf_create": (ci, [i32, vp, i32, vp, vp, vp, ctypes.POINTER(vp)]),
        "bude_hf_fock": (ci, [vp, vp, vp, ctypes.c_double, i32, vp]),
        "bude_hf_destroy": (ci, [vp]),
        "bude_hf_quartets": (ci, [vp, ctypes.c_double, ctypes.POINTER(i64), vp]),
        "bude_laplacian": (ci, [i32, vp, vp, i32, i32, i32, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, vp]),
        "bude_laplacian_path": (ci, [i32, vp, i32, i32, i32]),
        "bude_wait_timeouts": (ci, [ctypes.POINTER(ctypes.c_uint32), vp]),
        "bude_debug_stall_next_stencil": (ci, []),
        "bude_get_default_options": (ci, [i32, ctypes.POINTER(Options)]),
        "bude_set_default_options": (ci, [ctypes.POINTER(Options)]),
        "bude_last_launch_count": (i64, []),
        "bude_selfcheck_sqrt": (ci, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32), vp]),
        "bude_status_string": (ctypes.c_char_p, [ci]),
        "bude_last_error": (ctypes.c_char_p, []),
        "bude_debug_fail_alloc": (ci, [i32]),
        "bude_debug_pending_fail_alloc": (i32, []),
        "bude_debug_partition": (ci, [i32, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                      ctypes.POINTER(i32), i32, ctypes.POINTER(i32),
                                      ctypes.POINTER(i64), ctypes.POINTER(i64),
                                      ctypes.POINTER(i32)]),
        "bude_debug_cached_plans": (ci, [ctypes.POINTER(i32), ctypes.POINTER(i32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def header_functions(path: str = HEADER):
    """Names of the functions include/bude.h declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bude_[a-z_0-9]+)\s*\(", text)))


def _check(rc: int):
    if rc != OK:
        lib = load()
        raise BudeError(rc, f"{lib.bude_status_string(rc).decode()}: "
                            f"{lib.bude_last_error().decode()}")


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def selfcheck_sqrt(stream=None):
    """(mismatches, first mismatching bits) of the IEEE kernels' square root
    against sqrt.rn over every normal float."""
    n = ctypes.c_uint64()
    first = ctypes.c_uint32()
    _check(load().bude_selfcheck_sqrt(ctypes.byref(n), ctypes.byref(first), _stream_ptr(stream)))
    return n.value, first.value


def debug_fail_alloc(n: int) -> None:
    """Make the n-th device allocation of the library from now on fail with
    BUDE_ERR_OOM (host-side fault injection for tests; 0 disarms)."""
    _check(load().bude_debug_fail_alloc(int(n)))


def debug_pending_fail_alloc() -> int:
    """Allocations left before the injected failure (0 when disarmed)."""
    return int(load().bude_debug_pending_fail_alloc())


def debug_partition(K, nt, w, grid: int, with_owner: bool = True):
    """The kernel's split of a launch over its CTAs (bude_debug_partition):
    (CTAs used, range starts, owning CTA of every flat unit or None, CTAs
    expected per tile), all computed on the host."""
    lib = load()
    K = np.ascontiguousarray(K, np.int64)
    nt = np.ascontiguousarray(nt, np.int64)
    w = np.ascontiguousarray(w, np.int32)
    g = ctypes.c_int32()
    begin = np.zeros(int(grid) + 1, np.int64)
    owner = np.zeros(int((K * nt).sum()), np.int64) if with_owner else None
    cover = np.zeros(int(nt.sum()), np.int32)
    P = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t)) if a is not None else None  # noqa: E731
    _check(lib.bude_debug_partition(len(K), P(K, ctypes.c_int64), P(nt, ctypes.c_int64),
                                    P(w, ctypes.c_int32), int(grid), ctypes.byref(g),
                                    P(begin, ctypes.c_int64), P(owner, ctypes.c_int64),
                                    P(cover, ctypes.c_int32)))
    return g.value, begin[:g.value + 1].copy(), owner, cover


def debug_cached_plans() -> tuple[int, int]:
    """(batched, refine): captured plans the library holds (at most 64 each)."""
    b, r = ctypes.c_int32(), ctypes.c_int32()
    _check(load().bude_debug_cached_plans(ctypes.byref(b), ctypes.byref(r)))
    return b.value, r.value


def launch_count() -> int:
    """Kernels the last compute call on this thread enqueued."""
    return int(load().bude_last_launch_count())


@dataclass
class LaunchOptions:
    variant: int = FP32_IEEE
    ppwi: int = 0
    block: int = 0
    tile: int = 0
    ctas_per_sm: int = 0
    cull: int = 0

    def c(self) -> Options:
        v = VARIANTS[self.variant] if isinstance(self.variant, str) else self.variant
        return Options(v, self.ppwi, self.block, self.tile, self.ctas_per_sm, self.cull)


def _opts(opts=None, **kw) -> Options:
    if opts is None:
        opts = LaunchOptions(**kw)
    elif kw:
        raise TypeError("pass either opts or keyword options")
    return opts.c() if isinstance(opts, LaunchOptions) else opts


def default_options(variant) -> LaunchOptions:
    v = VARIANTS[variant] if isinstance(variant, str) else variant
    o = Options()
    _check(load().bude_get_default_options(v, ctypes.byref(o)))
    return LaunchOptions(o.variant, o.ppwi, o.block, o.tile, o.ctas_per_sm, o.cull)


def set_default_options(opts: LaunchOptions):
    o = opts.c()
    _check(load().bude_set_default_options(ctypes.byref(o)))


def pack_atoms(xyz, types) -> np.ndarray:
    """[n][4] float32 records: x, y, z and the int32 type in the fourth word."""
    xyz = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
    t = np.ascontiguousarray(types, np.int32).reshape(-1)
    out = np.empty((xyz.shape[0], 4), np.float32)
    out[:, :3] = xyz
    out[:, 3] = t.view(np.float32)
    return out


def pack_forcefield(radius, hardness, elsc, hbtype) -> np.ndarray:
    """[n_types][4] float32 rows: radius, hardness, elsc, hbtype (int32 bits)."""
    n = len(radius)
    out = np.empty((n, 4), np.float32)
    out[:, 0] = radius
    out[:, 1] = hardness
    out[:, 2] = elsc
    out[:, 3] = np.ascontiguousarray(hbtype, np.int32).view(np.float32)
    return out


def _cuda_device(device=None) -> torch.device:
    """A CUDA device with its index ("cuda" and None: the current device), so
    that it compares equal to the device of the tensors made on it."""
    dev = torch.device(device) if device is not None else torch.device("cuda")
    if dev.type != "cuda":
        raise ValueError(f"a CUDA device, got {dev}")
    return dev if dev.index is not None else torch.device("cuda", torch.cuda.current_device())


class Deck:
    """A deck on the current CUDA device (owns the library's deck handle)."""

    def __init__(self, deck: dict, device=None, stream=None):
        lib = load()
        dev = _cuda_device(device)
        lig = torch.from_numpy(pack_atoms(deck["lig_xyz"], deck["lig_type"])).to(dev)
        pro = torch.from_numpy(pack_atoms(deck["pro_xyz"], deck["pro_type"])).to(dev)
        ff = torch.from_numpy(pack_forcefield(deck["radius"], deck["hardness"], deck["elsc"],
                                              deck["hbtype"])).to(dev)
        self.device = dev
        self.n_lig, self.n_pro, self.n_types = lig.shape[0], pro.shape[0], ff.shape[0]
        desc = DeckDesc(self.n_lig, self.n_pro, self.n_types,
                        lig.data_ptr() if self.n_lig else None,
                        pro.data_ptr() if self.n_pro else None, ff.data_ptr())
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            rc = lib.bude_create_deck(ctypes.byref(desc), _stream_ptr(stream), ctypes.byref(h))
        _check(rc)
        self._h = h
        rows = ctypes.c_int32()
        _check(lib.bude_deck_info(h, None, None, None, ctypes.byref(rows)))
        self.n_rows = rows.value

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("deck was closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().bude_destroy_deck(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_poses(poses: torch.Tensor, deck: Deck):
    if not isinstance(poses, torch.Tensor) or poses.dtype != torch.float32:
        raise TypeError("poses must be a float32 torch tensor")
    if poses.dim() != 2 or poses.shape[0] != 6:
        raise ValueError(f"poses must be [6, n], got {tuple(poses.shape)}")
    if poses.device != deck.device:
        raise ValueError(f"poses on {poses.device}, deck on {deck.device}")
    if not poses.is_contiguous():
        raise ValueError("poses must be contiguous")


def _check_out(out, n: int, deck: Deck, what: str = "out"):
    """A caller-supplied output: the kernels write n float32 values through
    its pointer, so it must be exactly that, on the deck's device."""
    if not isinstance(out, torch.Tensor):
        raise ValueError(f"{what} must be a torch tensor")
    if out.shape != (n,) or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError(f"{what} must be a contiguous float32 [{n}] tensor, "
                         f"got {out.dtype} {tuple(out.shape)}")
    if out.device != deck.device:
        raise ValueError(f"{what} on {out.device}, deck on {deck.device}")


def energies(deck: Deck, poses: torch.Tensor, out: torch.Tensor | None = None,
             opts=None, stream=None, **kw) -> torch.Tensor:
    """Per-pose energies (float32 [n]) of device poses [6, n]."""
    _check_poses(poses, deck)
    n = poses.shape[1]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=poses.device)
    else:
        _check_out(out, n, deck)
    o = _opts(opts, **kw)
    rc = load().bude_energies(deck.handle, ctypes.c_void_p(poses.data_ptr()), n,
                              ctypes.c_void_p(out.data_ptr()), ctypes.byref(o),
                              _stream_ptr(stream))
    _check(rc)
    return out


def energies_host(deck: Deck, poses: torch.Tensor, out: torch.Tensor | None = None,
                  opts=None, stream=None, **kw) -> torch.Tensor:
    """bude_energies_host: energies of HOST poses (CPU float32 [6][n]; pinned
    lets the copies overlap) into a host tensor.  The library does both copies
    on the stream; this returns after synchronising it."""
    if poses.device.type != "cpu" or poses.dtype != torch.float32 or poses.dim() != 2 \
            or poses.shape[0] != 6 or not poses.is_contiguous():
        raise ValueError("poses must be a contiguous CPU float32 [6, n] tensor")
    n = poses.shape[1]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, pin_memory=poses.is_pinned())
    if out.device.type != "cpu" or out.shape != (n,) or out.dtype != torch.float32 \
            or not out.is_contiguous():
        raise ValueError("out must be a contiguous CPU float32 [n] tensor")
    o = _opts(opts, **kw)
    with torch.cuda.device(deck.device):
        st = stream if stream is not None else torch.cuda.current_stream()
        rc = load().bude_energies_host(deck.handle, ctypes.c_void_p(poses.data_ptr()), n,
                                       ctypes.c_void_p(out.data_ptr()), ctypes.byref(o),
                                       ctypes.c_void_p(st.cuda_stream))
        _check(rc)
        st.synchronize()
    return out


def energies_noalloc(deck: Deck, poses: torch.Tensor, out: torch.Tensor,
                     opts=None, stream=None, **kw) -> torch.Tensor:
    """bude_energies_noalloc: energies into a caller-provided ``out`` with the
    kernel's scratch in the library's fixed device array (no allocation)."""
    _check_poses(poses, deck)
    n = poses.shape[1]
    _check_out(out, n, deck)
    o = _opts(opts, **kw)
    rc = load().bude_energies_noalloc(deck.handle, ctypes.c_void_p(poses.data_ptr()), n,
                                      ctypes.c_void_p(out.data_ptr()), ctypes.byref(o),
                                      _stream_ptr(stream))
    _check(rc)
    return out


def energies_batched(decks, poses, outs=None, opts=None, stream=None, **kw):
    """Energies of several decks in one persistent, graph-replayed launch."""
    m = len(decks)
    if len(poses) != m:
        raise ValueError("one poses tensor per deck")
    for d, p in zip(decks, poses):
        _check_poses(p, d)
    if outs is None:
        outs = [torch.empty(p.shape[1], dtype=torch.float32, device=p.device) for p in poses]
    else:
        outs = list(outs)
        if len(outs) != m:
            raise ValueError(f"{len(outs)} outputs for {m} decks")
        for i, (d, p, o) in enumerate(zip(decks, poses, outs)):
            _check_out(o, p.shape[1], d, f"outs[{i}]")
    VP = ctypes.c_void_p * m
    hd = VP(*[d.handle.value for d in decks])
    hp = VP(*[p.data_ptr() for p in poses])
    ho = VP(*[o.data_ptr() for o in outs])
    hn = (ctypes.c_int64 * m)(*[p.shape[1] for p in poses])
    o = _opts(opts, **kw)
    rc = load().bude_energies_batched(hd, hp, hn, ho, m, ctypes.byref(o), _stream_ptr(stream))
    _check(rc)
    return outs


def pose_grad(deck: Deck, poses: torch.Tensor, want_energy: bool = True, opts=None,
              stream=None, **kw):
    """(energies [n] or None, d energy / d pose [6, n]) from the adjoint kernel."""
    _check_poses(poses, deck)
    n = poses.shape[1]
    E = torch.empty(n, dtype=torch.float32, device=poses.device) if want_energy else None
    G = torch.empty((6, n), dtype=torch.float32, device=poses.device)
    o = _opts(opts, **kw)
    rc = load().bude_pose_grad(deck.handle, ctypes.c_void_p(poses.data_ptr()), n,
                               ctypes.c_void_p(E.data_ptr()) if E is not None else None,
                               ctypes.c_void_p(G.data_ptr()), ctypes.byref(o),
                               _stream_ptr(stream))
    _check(rc)
    return E, G


def refine_device(deck: Deck, poses: torch.Tensor, steps: int = 10, step0: float = 0.1,
                  energies: torch.Tensor | None = None, opts=None, stream=None, **kw):
    """bude_refine: ``steps`` iterations of per-pose adaptive gradient descent
    on the GPU, one CUDA-graph replay; ``poses`` is updated in place.  Returns
    the final energies."""
    _check_poses(poses, deck)
    n = poses.shape[1]
    if energies is None:
        energies = torch.empty(n, dtype=torch.float32, device=poses.device)
    else:
        _check_out(energies, n, deck, "energies")
    o = _opts(opts, **kw)
    rc = load().bude_refine(deck.handle, ctypes.c_void_p(poses.data_ptr()), n, int(steps),
                            float(step0), ctypes.c_void_p(energies.data_ptr()), ctypes.byref(o),
                            _stream_ptr(stream))
    _check(rc)
    return energies


def param_grad(deck: Deck, poses: torch.Tensor, weights: torch.Tensor | None = None,
               opts=None, stream=None, **kw):
    """bude_param_grad: (dL/d ligand xyz [n_lig, 3], dL/d (radius, hardness,
    elsc) [n_types, 3]) for L = sum_k w_k E_k."""
    _check_poses(poses, deck)
    n = poses.shape[1]
    if weights is not None:
        if weights.shape != (n,) or weights.dtype != torch.float32 or weights.device != poses.device:
            raise ValueError("weights must be a float32 [n] tensor on the poses' device")
        weights = weights.contiguous()
    gl = torch.empty((deck.n_lig, 3), dtype=torch.float32, device=poses.device)
    gf = torch.empty((deck.n_types, 3), dtype=torch.float32, device=poses.device)
    o = _opts(opts, **kw)
    rc = load().bude_param_grad(deck.handle, ctypes.c_void_p(poses.data_ptr()), n,
                                ctypes.c_void_p(weights.data_ptr()) if weights is not None else None,
                                ctypes.c_void_p(gl.data_ptr()) if deck.n_lig else None,
                                ctypes.c_void_p(gf.data_ptr()), ctypes.byref(o),
                                _stream_ptr(stream))
    _check(rc)
    return gl, gf


STREAM_OPS = {"copy": 0, "mul": 1, "add": 2, "triad": 3, "dot": 4}


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return 0
    if t.dtype == torch.float64:
        return 1
    raise TypeError("float32 or float64 tensors only")


def _check_cuda(ts, what: str):
    """The kernels read and write these tensors through raw pointers: every
    one must be a CUDA tensor, all on one device."""
    for t in ts:
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
            raise ValueError(f"{what} must be CUDA tensors")
        if t.device != ts[0].device:
            raise ValueError(f"{what} on {t.device} and {ts[0].device}")


def stream_op(op: str, a=None, b=None, c=None, scalar: float = 0.4, dot_out=None, stream=None):
    """One BabelStream operation (copy c=a, mul b=s c, add c=a+b, triad
    a=b+s c, dot) on equal-length contiguous device tensors."""
    code = STREAM_OPS[op]
    given = {"a": a, "b": b, "c": c}
    need = {0: "ac", 1: "bc", 2: "abc", 3: "abc", 4: "ab"}[code]
    if any(given[k] is None for k in need):
        raise ValueError(f"{op} needs the arrays {', '.join(need)}")
    ts = [given[k] for k in need]
    _check_cuda(ts, "the arrays")
    if any((not t.is_contiguous()) or t.dtype != ts[0].dtype or t.numel() != ts[0].numel()
           for t in ts):
        raise ValueError("contiguous tensors of one dtype and length")
    a, b, c = (given[k] if k in need else None for k in "abc")
    if code == 4:
        if dot_out is None:
            dot_out = torch.empty((), dtype=torch.float64, device=ts[0].device)
        elif not isinstance(dot_out, torch.Tensor) or dot_out.dtype != torch.float64 \
                or dot_out.numel() != 1 or dot_out.device != ts[0].device:
            raise ValueError("dot_out must be a one-element float64 tensor on the arrays' device")
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    rc = load().bude_stream(code, _dtype_code(ts[0]), ptr(a), ptr(b), ptr(c), float(scalar),
                            ts[0].numel(), ptr(dot_out), _stream_ptr(stream))
    _check(rc)
    return dot_out


def laplacian(u: torch.Tensor, f: torch.Tensor, invhx2=1.0, invhy2=1.0, invhz2=1.0,
              invhxyz2=-6.0, stream=None):
    """Seven-point stencil of Listing 2 on [nx, ny, nz] tensors (interior of f)."""
    if u.shape != f.shape or u.dim() != 3 or u.dtype != f.dtype:
        raise ValueError("u and f: same [nx, ny, nz] shape and dtype")
    if not (u.is_contiguous() and f.is_contiguous()):
        raise ValueError("contiguous tensors")
    _check_cuda([u, f], "u and f")
    nx, ny, nz = u.shape
    rc = load().bude_laplacian(_dtype_code(u), ctypes.c_void_p(u.data_ptr()),
                               ctypes.c_void_p(f.data_ptr()), nx, ny, nz, float(invhx2),
                               float(invhy2), float(invhz2), float(invhxyz2), _stream_ptr(stream))
    _check(rc)
    return f


def laplacian_path(u: torch.Tensor) -> str:
    """"tma" or "register": the kernel bude_laplacian takes for u."""
    if u.dim() != 3:
        raise ValueError("u: [nx, ny, nz]")
    rc = load().bude_laplacian_path(_dtype_code(u), ctypes.c_void_p(u.data_ptr()), *u.shape)
    if rc < 0:
        _check(rc)
    return "tma" if rc == 1 else "register"


def wait_timeouts(stream=None) -> int:
    """Synchronise and return (and clear) the count of stencil CTAs whose
    bounded wait for a staged plane gave up."""
    n = ctypes.c_uint32(0)
    _check(load().bude_wait_timeouts(ctypes.byref(n), _stream_ptr(stream)))
    return int(n.value)


def debug_stall_next_stencil() -> None:
    """Test hook: the next TMA stencil launch has its first CTA time out."""
    _check(load().bude_debug_stall_next_stencil())


class HartreeFock:
    """Two-electron Fock term G_ij = sum_kl D_kl [2 (ij|kl) - (ik|jl)] over
    one contracted s function per atom (bude_hf_create / bude_hf_fock)."""

    def __init__(self, geom, xpnt, coef, device=None, stream=None):
        lib = load()
        g = np.ascontiguousarray(geom, np.float64).reshape(-1, 3)
        x = np.ascontiguousarray(xpnt, np.float64)
        c = np.ascontiguousarray(coef, np.float64)
        self.n = g.shape[0]
        self.device = _cuda_device(device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib.bude_hf_create(self.n, g.ctypes.data_as(ctypes.c_void_p), len(x),
                                    x.ctypes.data_as(ctypes.c_void_p),
                                    c.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream),
                                    ctypes.byref(h))
        _check(rc)
        self._h = h

    def fock(self, dens: torch.Tensor, tol: float = 1e-12, variant="fp64", out=None, stream=None):
        for t, what in ((dens, "dens"), (out, "out")):
            if t is None:
                continue
            if not isinstance(t, torch.Tensor) or t.shape != (self.n, self.n) \
                    or t.dtype != torch.float64 or not t.is_contiguous():
                raise ValueError(f"{what} must be a contiguous float64 [n, n] tensor")
            if t.device != self.device:
                raise ValueError(f"{what} on {t.device}, the basis on {self.device}")
        out = torch.empty_like(dens) if out is None else out
        v = VARIANTS[variant] if isinstance(variant, str) else variant
        rc = load().bude_hf_fock(self._h, ctypes.c_void_p(dens.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), float(tol), v,
                                 _stream_ptr(stream))
        _check(rc)
        return out

    def quartets(self, tol: float = 1e-12, stream=None) -> int:
        """Unique quartets that survive the Schwarz threshold ``tol``."""
        c = ctypes.c_int64()
        _check(load().bude_hf_quartets(self._h, float(tol), ctypes.byref(c), _stream_ptr(stream)))
        return int(c.value)

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().bude_hf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PoseEnergy(torch.autograd.Function):
    """energies = PoseEnergy.apply(poses, deck, opts); backward uses the adjoint kernel."""

    @staticmethod
    def forward(ctx, poses, deck, opts=None):
        p = poses.detach().contiguous()
        E, G = pose_grad(deck, p, want_energy=True, opts=opts)
        ctx.save_for_backward(G)
        return E

    @staticmethod
    def backward(ctx, grad_out):
        (G,) = ctx.saved_tensors
        return G * grad_out.unsqueeze(0), None, None

