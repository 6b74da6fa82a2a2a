"""Autotuner for the persistent pose kernel's launch shape.

Searches poses per thread (P), threads per CTA, resident CTAs per SM and the
protein chunk length by timing real launches through the C ABI with CUDA
events, and keeps the fastest shape per (GPU, variant, workload bucket) in a
JSON table.  The committed table ``tuned.json`` holds the shapes found on
GB300; ``apply()`` installs them as the library defaults.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import statistics

import torch

from . import bude

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")

SPACE = {
    "ppwi": [1, 2, 4, 8, 16],
    "block": [64, 128, 256, 384, 512, 768, 1024],
    "ctas_per_sm": [1, 2, 3, 4],
    "tile": [0],
}
# Protein-tile lengths (atoms staged per shared-memory chunk; 0 = as many as
# fit) tried in a second stage on the best shapes of the first.
TILES = [256, 512, 1024, 2048]
TILE_STAGE_TOP = 3


def _with_tile(o, t):
    return bude.LaunchOptions(variant=o.variant, ppwi=o.ppwi, block=o.block,
                              ctas_per_sm=o.ctas_per_sm, tile=t, cull=o.cull)


def bucket(n_lig: int, n_pro: int, n_poses: int) -> str:
    """Workload bucket: log2 of the pose count and of the pair count."""
    lp = max(0, math.ceil(math.log2(max(n_poses, 1))))
    lk = max(0, math.ceil(math.log2(max(n_lig * n_pro, 1))))
    return f"p{lp}_k{lk}"


def gpu_name() -> str:
    return torch.cuda.get_device_name().replace(" ", "_")


def key(variant: str, b: str, mode: str = "plain") -> str:
    return f"{gpu_name()}|{variant}|{mode}|{b}"


def load_table(path: str = TABLE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_table(table: dict, path: str = TABLE):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_call(fn, reps: int = 5, warmup: int = 1) -> float:
    """Median milliseconds of fn() on the current stream."""
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    ms = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def candidates(variant: str, space=None, grad: bool = False, cull: int = 0):
    sp = dict(SPACE if space is None else space)
    ps = sp["ppwi"]
    if variant == "fp64":
        ps = [p for p in ps if p <= 4]
    if grad:
        ps = [p for p in ps if p <= 8]
    if cull:
        ps = [p for p in ps if p % 2 == 0]   # culling is built for even P
    for p, b, c, t in itertools.product(ps, sp["block"], sp["ctas_per_sm"], sp["tile"]):
        yield bude.LaunchOptions(variant=variant, ppwi=p, block=b, ctas_per_sm=c, tile=t,
                                 cull=cull)


def tune_plain(deck, poses, variant: str, space=None, reps: int = 5, grad: bool = False,
               log=None, cull: int = 0, param: bool = False):
    """Fastest launch shape of bude_energies (or bude_pose_grad, or with param
    bude_param_grad) on this input."""
    out = torch.empty(poses.shape[1], dtype=torch.float32, device=poses.device)
    results = []
    for o in candidates(variant, space, grad or param, cull):
        if param:
            fn = lambda: bude.param_grad(deck, poses, opts=o)  # noqa: E731
        elif grad:
            fn = lambda: bude.pose_grad(deck, poses, want_energy=True, opts=o)  # noqa: E731
        else:
            fn = lambda: bude.energies(deck, poses, out=out, opts=o)  # noqa: E731
        try:
            ms = time_call(fn, reps)
        except bude.BudeError as e:
            if e.code != bude.ERR_UNSUPPORTED:
                raise
            continue
        results.append((ms, o))
        if log:
            log(f"{variant} P={o.ppwi:2d} block={o.block:4d} cps={o.ctas_per_sm} "
                f"tile={o.tile} cull={o.cull}: {ms:.3f} ms")
    results.sort(key=lambda r: r[0])
    return _tile_stage(results, fn_of=lambda o: (lambda: (
        bude.param_grad(deck, poses, opts=o) if param else
        bude.pose_grad(deck, poses, want_energy=True, opts=o) if grad else
        bude.energies(deck, poses, out=out, opts=o))), reps=reps, log=log, tag=variant)


def _tile_stage(results, fn_of, reps, log, tag):
    """Second stage: the best shapes again with each protein-tile length."""
    extra = []
    for _, o in results[:TILE_STAGE_TOP]:
        for t in TILES:
            ot = _with_tile(o, t)
            try:
                ms = time_call(fn_of(ot), reps)
            except bude.BudeError as e:
                if e.code != bude.ERR_UNSUPPORTED:
                    raise
                continue
            extra.append((ms, ot))
            if log:
                log(f"{tag} P={ot.ppwi:2d} block={ot.block:4d} cps={ot.ctas_per_sm} "
                    f"tile={ot.tile} cull={ot.cull}: {ms:.3f} ms")
    out = results + extra
    out.sort(key=lambda r: r[0])
    return out


def tune_batched(decks, poses, variant: str, space=None, reps: int = 5, log=None):
    outs = [torch.empty(p.shape[1], dtype=torch.float32, device=p.device) for p in poses]
    results = []
    for o in candidates(variant, space):
        try:
            ms = time_call(lambda: bude.energies_batched(decks, poses, outs, opts=o), reps)
        except bude.BudeError as e:
            if e.code != bude.ERR_UNSUPPORTED:
                raise
            continue
        results.append((ms, o))
        if log:
            log(f"batched {variant} P={o.ppwi:2d} block={o.block:4d} cps={o.ctas_per_sm}: "
                f"{ms:.3f} ms")
    results.sort(key=lambda r: r[0])
    return _tile_stage(results, fn_of=lambda o: (lambda: bude.energies_batched(
        decks, poses, outs, opts=o)), reps=reps, log=log, tag=f"batched {variant}")


def tune_plain_group(decks, poses, variant: str, space=None, reps: int = 5, log=None):
    """Fastest launch shape for plain bude_energies calls over several decks
    of one workload bucket: each candidate is timed over one call per deck,
    so the shape that wins is the best for the bucket as a whole."""
    outs = [torch.empty(p.shape[1], dtype=torch.float32, device=p.device) for p in poses]

    def run(o):
        for d, p, out in zip(decks, poses, outs):
            bude.energies(d, p, out=out, opts=o)

    results = []
    for o in candidates(variant, space):
        try:
            ms = time_call(lambda: run(o), reps)
        except bude.BudeError as e:
            if e.code != bude.ERR_UNSUPPORTED:
                raise
            continue
        results.append((ms, o))
        if log:
            log(f"group {variant} P={o.ppwi:2d} block={o.block:4d} cps={o.ctas_per_sm}: "
                f"{ms:.3f} ms")
    results.sort(key=lambda r: r[0])
    return _tile_stage(results, fn_of=lambda o: (lambda: run(o)), reps=reps, log=log,
                       tag=f"group {variant}")


def record(table: dict, k: str, ms: float, o) -> None:
    table[k] = {"ppwi": o.ppwi, "block": o.block, "ctas_per_sm": o.ctas_per_sm,
                "tile": o.tile, "ms": round(ms, 4)}
    if o.cull:
        table[k]["cull"] = o.cull


def lookup(variant: str, n_lig: int, n_pro: int, n_poses: int, mode: str = "plain",
           table: dict | None = None):
    """Tuned LaunchOptions for this workload, or None when the table has none."""
    t = load_table() if table is None else table
    e = t.get(key(variant, bucket(n_lig, n_pro, n_poses), mode))
    if e is None:
        return None
    return bude.LaunchOptions(variant=variant, ppwi=e["ppwi"], block=e["block"],
                              ctas_per_sm=e["ctas_per_sm"], tile=e["tile"],
                              cull=e.get("cull", 0))


def apply(variants=("ieee", "fast", "comp", "fp64"), n_lig=64, n_pro=2672, n_poses=65536):
    """Install the tuned shapes for a workload as the library's defaults."""
    t = load_table()
    for v in variants:
        o = lookup(v, n_lig, n_pro, n_poses, table=t)
        if o is not None:
            bude.set_default_options(o)


def _workloads(which):
    from . import synth
    if "small" in which:
        yield "small", [synth.make_deck(0, **synth.SMALL)]
    if "full" in which:
        yield "full", [synth.make_deck(1, **synth.FULL)]
    if "full_fp64" in which:
        # FP64 is ~100x slower than FP32 on GB300: its shape for the full deck is
        # tuned on the deck's first 4096 poses (the persistent kernel's choice
        # depends on the pair loop, not on the pose count once the grid is full)
        d = synth.make_deck(1, **synth.FULL)
        d["poses"] = d["poses"][:, :4096].copy()
        yield "full_fp64", [d]
    if "cull" in which:
        yield "cull", [synth.make_deck(1, **synth.FULL)]
    if "grad" in which:
        yield "grad", [synth.make_deck(4, **synth.GRAD)]
    if "grad_cull" in which:
        yield "grad_cull", [synth.make_deck(4, **synth.GRAD)]
    if "param" in which:
        yield "param", [synth.make_deck(4, **synth.GRAD)]
    if "batched" in which:
        yield "batched", synth.make_batched(3, 64)
    if "batched_plain" in which:
        # the plain launches the batched launch is compared with: one shape per
        # workload bucket of the 64 decks
        yield "batched_plain", synth.make_batched(3, 64)


def main(argv=None):
    import argparse
    from . import synth
    ap = argparse.ArgumentParser(description="tune launch shapes and write tuned.json")
    ap.add_argument("--workloads", default="small,full,grad,batched")
    ap.add_argument("--variants", default="fast,ieee,comp,fp64")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--log", default=None)
    a = ap.parse_args(argv)
    table = load_table(a.out)
    logf = open(a.log, "w") if a.log else None

    def log(msg):
        if logf:
            logf.write(msg + "\n")
            logf.flush()

    dev = torch.device("cuda", torch.cuda.current_device())
    variants = a.variants.split(",")
    for name, decks_np in _workloads(a.workloads.split(",")):
        decks = [bude.Deck(d, device=dev) for d in decks_np]
        poses = [torch.from_numpy(d["poses"]).to(dev) for d in decks_np]
        for v in variants:
            space = None
            if v == "fp64":
                if name not in ("small", "full_fp64"):
                    continue   # FP64 runs ~100x slower: the small deck and 4096 full-deck poses
                space = {"ppwi": [1, 2, 4], "block": [128, 192, 256, 384, 512],
                         "ctas_per_sm": [1, 2, 3], "tile": [0]}
            elif name == "full_fp64":
                continue
            if name == "batched_plain":
                if v not in ("fast", "ieee"):
                    continue
                groups: dict = {}
                for i, d in enumerate(decks_np):
                    b = bucket(len(d["lig_type"]), len(d["pro_type"]), d["poses"].shape[1])
                    groups.setdefault(b, []).append(i)
                for b, idx in sorted(groups.items()):
                    k = key(v, b)
                    if k in table:
                        continue   # tuned on its own workload already
                    res = tune_plain_group([decks[i] for i in idx], [poses[i] for i in idx], v,
                                           space, a.reps, log)
                    if res:
                        record(table, k, res[0][0], res[0][1])
                        table[k]["decks"] = len(idx)
                        print(f"{k}: {len(idx)} decks, P{res[0][1].ppwi}/b{res[0][1].block}/"
                              f"c{res[0][1].ctas_per_sm}/t{res[0][1].tile}:{res[0][0]:.3f}",
                              flush=True)
                continue
            if name == "batched":
                if v not in ("fast", "ieee"):
                    continue
                res = tune_batched(decks, poses, v, space, a.reps, log)
                b = "x".join(str(len(decks_np)) for _ in [0])
                k = key(v, f"n{b}", "batched")
            elif name == "cull":
                if v == "fp64":
                    continue
                d = decks_np[0]
                res = tune_plain(decks[0], poses[0], v, space, a.reps, log=log, cull=1)
                k = key(v, bucket(len(d["lig_type"]), len(d["pro_type"]), d["poses"].shape[1]),
                        "cull")
            elif name == "param":
                if v not in ("fast", "ieee"):
                    continue
                d = decks_np[0]
                res = tune_plain(decks[0], poses[0], v, space, a.reps, log=log, param=True)
                k = key(v, bucket(len(d["lig_type"]), len(d["pro_type"]), d["poses"].shape[1]),
                        "param")
            elif name in ("grad", "grad_cull"):
                if v not in ("fast", "ieee"):
                    continue
                d = decks_np[0]
                res = tune_plain(decks[0], poses[0], v, space, a.reps, grad=True, log=log,
                                 cull=int(name == "grad_cull"))
                k = key(v, bucket(len(d["lig_type"]), len(d["pro_type"]), d["poses"].shape[1]),
                        name)
            else:
                d = decks_np[0]
                res = tune_plain(decks[0], poses[0], v, space, a.reps, log=log)
                n_poses = synth.FULL["n_poses"] if name == "full_fp64" else d["poses"].shape[1]
                k = key(v, bucket(len(d["lig_type"]), len(d["pro_type"]), n_poses))
            if res:
                record(table, k, res[0][0], res[0][1])
                top = ", ".join(f"P{o.ppwi}/b{o.block}/c{o.ctas_per_sm}/t{o.tile}:{ms:.3f}"
                                for ms, o in res[:5])
                print(f"{k}: {top}", flush=True)
        for d in decks:
            d.close()
    save_table(table, a.out)
    print(f"wrote {a.out}")


if __name__ == "__main__":
    main()
