"""Throughput of the pose-energy hot path on GB300 (one JSON line on stdout).

A step is one bude_energies call over the full-size synthetic deck: 64
ligand atoms x 2672 protein atoms x 65536 poses (pose transform, pair loop,
per-pose reduction, output), inputs resident in HBM.  L2 is flushed (a
256 MiB write) before every timed step; each step is timed with CUDA events
on the launching stream.  ``value`` is poses per second over all ranks;
``e2e`` repeats the step through the C ABI's host-buffer call
(bude_energies_host) from pinned host buffers, host<->device copies included.  ``roofline`` rates the kernel against the
FP32 CUDA-core peak (152 SMs x 128 lanes x 2 FLOP x 2.07 GHz); FLOPs per
step follow Eq. 3 of the paper.  ``cpu_baseline`` times the FP64 oracle on
a bounded sample of the same workload on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--variant fast]
  python bench.py --impl reference     # the oracle arm on the host cores
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FULL = dict(n_lig=64, n_pro=2672, n_types=34, n_poses=65536)
SMALL = dict(n_lig=26, n_pro=938, n_types=34, n_poses=4096)
METRIC = "pose energies/s"
SM_MAX_MHZ = 2070.0
FP32_LANES_PER_SM = 128


# DRAM traffic of one full-size FAST launch, from one ncu capture of this
# kernel and shape (dram__bytes_read.sum + dram__bytes_write.sum, mean of 9
# launches).  Reported only while the kernel source and the launch shape are
# the ones that were measured; otherwise the line says why it is missing.
MEASURED_TRAFFIC = {"kernel_sha256_16": "bbb752c7b8eccbe4", "variant": "fast", "ppwi": 16,
                    "block": 384, "bytes": 1879438.0}

# FP32 FLOPs the kernel executes per pose-pair on the full deck, from ncu's
# per-opcode thread-instruction counters of the same launch (FADD, FMUL 1;
# FFMA, FADD2, FMUL2 2; FFMA2 4), per variant, for the kernel source with
# this hash.  Fewer than Eq. 3's 30: zero desolvation runs are skipped, and
# FAST takes the steric term as sign(H) z^2 with one fewer operation.
MEASURED_EXECUTED = {"kernel_sha256_16": "bbb752c7b8eccbe4",
                     "flop_per_pair": {"fast": 22.24, "ieee": 29.25, "comp": 29.24}}

# The same count for the FAST adjoint (energies and pose gradients) at P = 8
# on the 64 x 2672 x 16384 workload: the force and torque sums add the
# reciprocal root's products and three FFMA2 per pose pair to the energy work.
MEASURED_EXECUTED_ADJOINT = {"kernel_sha256_16": "bbb752c7b8eccbe4", "variant": "fast", "ppwi": 8,
                             "flop_per_pair": 36.77}

# The same count for the FAST forcefield-gradient kernel (param_kernel) at
# P = 8 on the 64 x 2672 x 16384 workload; the hash covers both of its
# source files.
MEASURED_EXECUTED_PARAM = {"kernel_sha256_16": "836eeb0553732cf7", "variant": "fast", "ppwi": 8,
                           "flop_per_pair": 39.12}


# FP64-pipe thread instructions per pose-pair of the FP64 energy kernel (DFMA,
# DMUL, DADD and the conversions that share the pipe), from ncu's
# smsp__inst_executed_pipe_fp64 of one launch on the full deck's first 4096
# poses, for the kernel source with this hash.  GB300's nominal FP64 rate of
# 1.25 TFLOP/s is 6.25e11 such instructions per second.
MEASURED_FP64_PIPE = {"kernel_sha256_16": "bbb752c7b8eccbe4", "ppwi": 4, "ops_per_pair": 19.88}
NOMINAL_FP64_INST_PER_S = 6.25e11

# The same count for the all-FP64 Fock build, per primitive integral, on the
# 128-atom lattice (3 primitives per atom) where it was taken: the share of
# primitives past the erf table's end, which take a reciprocal root instead,
# depends on the lattice, so the count is used for that size only.
MEASURED_HF64_PIPE = {"kernel_sha256_16": "92c2d732541e61f9", "atoms": 128, "ops_per_primitive": 30.47}


def kernel_sha(files=("bude_kernels.cuh",)):
    """First 16 hex digits of the sha256 of the kernel sources (csrc/) with
    comments and whitespace removed, so that edits to comments keep the
    measurements."""
    import hashlib
    import re
    texts = []
    for name in files:
        try:
            text = open(os.path.join(ROOT, "paper_2509_21039_gb300", "csrc", name)).read()
        except OSError:
            return None
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        texts.append(" ".join(text.split()))
    return hashlib.sha256("\n".join(texts).encode()).hexdigest()[:16]


def measured_executed(variant):
    """Executed FLOP per pose-pair of the current kernel, or None if unmeasured."""
    m = MEASURED_EXECUTED
    if kernel_sha() != m["kernel_sha256_16"]:
        return None
    return m["flop_per_pair"].get(variant)


def executed_source(variant):
    """Where roofline.executed_* come from, or why they are absent."""
    sha = kernel_sha()
    if sha != MEASURED_EXECUTED["kernel_sha256_16"]:
        return (f"absent: the ncu opcode counts were taken on kernel source "
                f"{MEASURED_EXECUTED['kernel_sha256_16']}, this is {sha}")
    if variant not in MEASURED_EXECUTED["flop_per_pair"]:
        return f"absent: no opcode count for variant {variant}"
    return f"ncu opcode counters of kernel source {sha}, full deck"


def measured_traffic(variant, ppwi, block, n_poses):
    sha = kernel_sha()
    if sha is None:
        return None
    m = MEASURED_TRAFFIC
    if (sha, variant, ppwi, block, n_poses) != (m["kernel_sha256_16"], m["variant"], m["ppwi"],
                                                 m["block"], FULL["n_poses"]):
        return None
    return m["bytes"]


def traffic_source(variant, ppwi, block, n_poses):
    """Where roofline.traffic comes from, or why it is null."""
    m = MEASURED_TRAFFIC
    sha = kernel_sha()
    if sha != m["kernel_sha256_16"]:
        return (f"null: DRAM bytes were captured on kernel source {m['kernel_sha256_16']}, "
                f"this is {sha}")
    if (variant, ppwi, block, n_poses) != (m["variant"], m["ppwi"], m["block"], FULL["n_poses"]):
        return (f"null: DRAM bytes were captured for {m['variant']} P={m['ppwi']} "
                f"block={m['block']} on {FULL['n_poses']} poses")
    return f"ncu dram__bytes_read.sum + dram__bytes_write.sum of kernel source {sha}"


def fp64_pipe_fraction(ppwi, pairs_per_s):
    """(FP64-pipe instructions per second, fraction of the nominal FP64 rate)
    of the FP64 energy kernel, or (None, None) when the counts do not belong
    to this kernel source and shape."""
    m = MEASURED_FP64_PIPE
    if m["ops_per_pair"] is None or (kernel_sha(), ppwi) != (m["kernel_sha256_16"], m["ppwi"]):
        return None, None
    ips = m["ops_per_pair"] * pairs_per_s
    return ips, ips / NOMINAL_FP64_INST_PER_S


def fp64_throughput(bude, synth, dev, timed):
    """The FP64 variant on the full deck's first 4096 poses (it runs about 80x
    slower than FAST on GB300, whose FP64 units are a small fraction of its
    FP32 ones), in the library's default (tuned) shape."""
    import torch
    D = synth.make_deck(1, **FULL)
    deck = bude.Deck(D, device=dev)
    P = torch.from_numpy(D["poses"][:, :4096].copy()).to(dev)
    out = torch.empty(P.shape[1], dtype=torch.float32, device=dev)
    o = bude.default_options("fp64")
    ms, _ = timed(lambda: bude.energies(deck, P, out=out, opts=o), 3, 1)
    deck.close()
    t = statistics.mean(ms) / 1e3
    ips, frac = fp64_pipe_fraction(o.ppwi, FULL["n_lig"] * FULL["n_pro"] * P.shape[1] / t)
    return {"workload": "64 lig x 2672 pro, first 4096 of the 65536 poses, seed 1",
            "ms": t * 1e3, "poses_per_s": P.shape[1] / t,
            "opts": {"ppwi": o.ppwi, "block": o.block, "ctas_per_sm": o.ctas_per_sm},
            "fp64_pipe_instructions_per_s": ips, "frac_of_nominal_fp64_rate": frac}


def eq3_flops(n_lig, n_pro, n_poses, ppwi):
    """Eq. 3: per work-item 28 P + nlig (2 + 18 P + npro (10 + 30 P)), x poses / P."""
    per_item = 28 * ppwi + n_lig * (2 + 18 * ppwi + n_pro * (10 + 30 * ppwi))
    return per_item * (n_poses / ppwi)


def algorithmic_flops(n_lig, n_pro, n_poses):
    """Eq. 3 in its many-poses-per-item limit: 28 + nlig (18 + 30 npro) per pose."""
    return n_poses * (28 + n_lig * (18 + 30 * n_pro))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def smi_id(local):
    """nvidia-smi's name for CUDA device `local`: its UUID, which stays right
    when CUDA_VISIBLE_DEVICES renumbers the devices; the index otherwise."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(local).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    return str(local)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0, path=None):
        self.index = index
        self.path = path
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.5)   # let nvidia-smi start before the warm-up steps
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]
            if self.path:
                with open(self.path, "w") as f:
                    f.write(self.Q + "\n" + "\n".join(self.lines) + "\n")

    def summary(self):
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "power_w_max": max(power) if power else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline_leg(deck, n_poses_total, budget_s=12.0, threads=-1):
    """The FP64 oracle, as it stands, on a bounded sample of the workload's
    poses (about budget_s of host CPU time per run, best of three runs).
    Returns (poses/s, sample size, best seconds, threads, sample energies,
    sample absolute-term sums)."""
    import oracle
    oracle.build()
    cores = oracle.max_threads() if threads < 0 else threads
    k = max(cores, 8)
    t0 = time.perf_counter()
    oracle.energies(deck, deck["poses"][:, :k], n_threads=threads)
    dt = time.perf_counter() - t0
    n = int(min(n_poses_total, max(k, k * budget_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    E, A = oracle.energies(deck, deck["poses"][:, :n], n_threads=threads, with_abs=True)
    dt = time.perf_counter() - t0
    # best of three, the first run included (the sample's energies come from it)
    for _ in range(2):
        t0 = time.perf_counter()
        oracle.energies(deck, deck["poses"][:, :n], n_threads=threads)
        dt = min(dt, time.perf_counter() - t0)
    return n / dt, n, dt, cores, E, A


def cpu_single_thread(deck, budget_s=3.0):
    """The oracle on one host core: poses/s on a sample of ~budget_s."""
    import oracle
    t0 = time.perf_counter()
    oracle.energies(deck, deck["poses"][:, :2], n_threads=0)
    dt = time.perf_counter() - t0
    k = max(2, int(2 * budget_s / max(dt, 1e-3)))
    best = float("inf")
    for _ in range(3):   # best of three
        t0 = time.perf_counter()
        oracle.energies(deck, deck["poses"][:, :k], n_threads=0)
        best = min(best, time.perf_counter() - t0)
    return k / best, k


def batched_vs_plain(bude, synth, tune, dev, timed, variant="fast", count=64, seed=3):
    """64 uneven decks: one persistent graph-replayed launch vs 64 plain launches."""
    import torch
    decks_np = synth.make_batched(seed, count)
    decks = [bude.Deck(d, device=dev) for d in decks_np]
    poses = [torch.from_numpy(d["poses"]).to(dev) for d in decks_np]
    outs_b = [torch.empty(p.shape[1], dtype=torch.float32, device=dev) for p in poses]
    outs_p = [torch.empty(p.shape[1], dtype=torch.float32, device=dev) for p in poses]
    t = tune.load_table()
    e = t.get(tune.key(variant, f"n{count}", "batched"))
    if e:
        ob = bude.LaunchOptions(variant=variant, ppwi=e["ppwi"], block=e["block"],
                                ctas_per_sm=e["ctas_per_sm"], tile=e["tile"])
    else:
        ob = bude.default_options(variant)
    # each plain launch takes the shape tuned for its own workload bucket
    # (the default when the table has none for that bucket)
    tbl = tune.load_table()
    ops = []
    for d in decks_np:
        o = tune.lookup(variant, len(d["lig_type"]), len(d["pro_type"]), d["poses"].shape[1],
                        table=tbl)
        ops.append(o)
    plain_tuned = sum(o is not None for o in ops)
    ops = [o if o is not None else bude.default_options(variant) for o in ops]

    def run_batched():
        bude.energies_batched(decks, poses, outs_b, opts=ob)

    def run_plain():
        n = 0
        for d, p, o, op in zip(decks, poses, outs_p, ops):
            bude.energies(d, p, out=o, opts=op)
            n += bude.launch_count()
        plain_launches[0] = n

    plain_launches = [0]

    ms_b, lb = timed(run_batched, 10, 3)
    ms_p, lp = timed(run_plain, 10, 3)
    # the batched launch with cutoff culling (opt-in) in the culled kernel's
    # tuned shape, checked bit for bit against the unculled kernel of that shape
    oc = tune.lookup(variant, 64, 2672, 65536, mode="cull") or \
        bude.LaunchOptions(variant=variant, ppwi=8, block=256)
    ob_c = bude.LaunchOptions(variant=variant, ppwi=oc.ppwi, block=oc.block,
                              ctas_per_sm=oc.ctas_per_sm, tile=oc.tile, cull=1)
    ob_u = bude.LaunchOptions(variant=variant, ppwi=oc.ppwi, block=oc.block,
                              ctas_per_sm=oc.ctas_per_sm, tile=oc.tile, cull=0)
    outs_c = [torch.empty_like(o) for o in outs_b]
    outs_u = [torch.empty_like(o) for o in outs_b]
    ms_c, _ = timed(lambda: bude.energies_batched(decks, poses, outs_c, opts=ob_c), 10, 3)
    bude.energies_batched(decks, poses, outs_u, opts=ob_u)
    torch.cuda.synchronize()
    cull_same = all(bool(torch.equal(a, c)) for a, c in zip(outs_u, outs_c))
    pairs = sum(len(d["lig_type"]) * len(d["pro_type"]) * d["poses"].shape[1] for d in decks_np)
    n = sum(d["poses"].shape[1] for d in decks_np)
    diff = max(float(((a - b).abs() / b.abs().clamp_min(1.0)).max()) for a, b in zip(outs_b, outs_p))
    # energies of both arms at 16 poses per deck (the last one included), for
    # the oracle comparison of the CPU-baseline leg
    samples = []
    for d, a, b in zip(decks_np, outs_b, outs_p):
        m = d["poses"].shape[1]
        idx = np.unique(np.linspace(0, m - 1, 16).round().astype(np.int64))
        samples.append((idx, a.cpu().numpy()[idx], b.cpu().numpy()[idx]))
    for d in decks:
        d.close()
    tb, tp = statistics.mean(ms_b), statistics.mean(ms_p)
    # Eq. 3 in the many-poses limit, summed over the decks, against the FP32 peak
    alg = sum(algorithmic_flops(len(d["lig_type"]), len(d["pro_type"]), d["poses"].shape[1])
              for d in decks_np)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    return {"workload": f"{count} decks, log-uniform lig 8-128, pro 500-5000, poses 1024-65536, seed {seed}",
            "variant": variant, "poses": n, "pair_evaluations": pairs,
            "batched_ms": tb, "plain_ms": tp, "speedup": tp / tb,
            "batched_eq3_frac_fp32_peak": alg / (tb / 1e3) / 1e12 / peak,
            "plain_eq3_frac_fp32_peak": alg / (tp / 1e3) / 1e12 / peak,
            "batched_poses_per_s": n / (tb / 1e3), "plain_poses_per_s": n / (tp / 1e3),
            "batched_launches": lb // 10, "plain_launches": plain_launches[0],
            "batched_opts": {"ppwi": ob.ppwi, "block": ob.block, "ctas_per_sm": ob.ctas_per_sm},
            "plain_opts": f"tuned per workload bucket for {plain_tuned} of {count} decks, "
                          f"the library default for the rest",
            "plain_tuned_decks": plain_tuned,
            "max_rel_diff_batched_vs_plain": diff,
            "batched_cull_ms": statistics.mean(ms_c), "batched_cull_bit_identical": cull_same,
            "batched_cull_opts": {"ppwi": ob_c.ppwi, "block": ob_c.block,
                                  "ctas_per_sm": ob_c.ctas_per_sm},
            "_samples": samples, "_decks": decks_np}


def adjoint_throughput(bude, synth, tune, dev, timed, variant="fast"):
    """Energies + pose gradients of 16384 poses on the 64 x 2672 deck."""
    import torch
    D = synth.make_deck(4, **synth.GRAD)
    deck = bude.Deck(D, device=dev)
    P = torch.from_numpy(D["poses"]).to(dev)
    o = tune.lookup(variant, 64, 2672, D["poses"].shape[1], mode="grad") or \
        bude.LaunchOptions(variant=variant)
    ms, _ = timed(lambda: bude.pose_grad(deck, P, opts=o), 10, 3)
    oc = tune.lookup(variant, 64, 2672, D["poses"].shape[1], mode="grad_cull") or \
        bude.LaunchOptions(variant=variant, ppwi=o.ppwi, block=o.block,
                           ctas_per_sm=o.ctas_per_sm, tile=o.tile)
    oc.cull = 1
    ms_c, _ = timed(lambda: bude.pose_grad(deck, P, opts=oc), 10, 3)
    # bit-identity against the unculled kernel of the culled launch's shape
    e1, g1 = bude.pose_grad(deck, P, opts=oc)
    ou = bude.LaunchOptions(variant=oc.variant, ppwi=oc.ppwi, block=oc.block,
                            ctas_per_sm=oc.ctas_per_sm, tile=oc.tile, cull=0)
    e2, g2 = bude.pose_grad(deck, P, opts=ou)
    same = bool(torch.equal(e1, e2) and torch.equal(g1, g2))
    deck.close()
    t = statistics.mean(ms)
    m = MEASURED_EXECUTED_ADJOINT
    executed = None
    if (kernel_sha(), variant, o.ppwi) == (m["kernel_sha256_16"], m["variant"], m["ppwi"]):
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
        tf = m["flop_per_pair"] * 64 * 2672 * P.shape[1] / (t / 1e3) / 1e12
        executed = {"flop_per_pair": m["flop_per_pair"], "tflops": tf, "frac_fp32_peak": tf / peak,
                    "source": "ncu opcode counters of the same kernel source and shape"}
    return {"workload": "64 lig x 2672 pro x 16384 poses, seed 4", "variant": variant,
            "ms": t, "poses_per_s": P.shape[1] / (t / 1e3), "executed": executed,
            "opts": {"ppwi": o.ppwi, "block": o.block, "ctas_per_sm": o.ctas_per_sm},
            "cull_ms": statistics.mean(ms_c), "cull_bit_identical": same,
            "cull_opts": {"ppwi": oc.ppwi, "block": oc.block, "ctas_per_sm": oc.ctas_per_sm}}


def refine_throughput(bude, synth, tune, dev, timed, variant="fast", steps=10):
    """Ten refinement steps on 16384 poses of the 64 x 2672 deck, one graph."""
    import torch
    D = synth.make_deck(4, **synth.GRAD)
    deck = bude.Deck(D, device=dev)
    P0 = torch.from_numpy(D["poses"]).to(dev)
    P = P0.clone()
    E = torch.empty(P.shape[1], device=dev)
    o = tune.lookup(variant, 64, 2672, D["poses"].shape[1], mode="grad") or \
        bude.LaunchOptions(variant=variant)
    e0 = bude.energies(deck, P0).mean().item()

    def step():
        P.copy_(P0)
        bude.refine_device(deck, P, steps=steps, step0=0.05, energies=E, opts=o)

    ms, launches = timed(step, 5, 2)
    Pa, Ea = P.clone(), E.clone()
    oc = bude.LaunchOptions(variant=o.variant, ppwi=o.ppwi, block=o.block,
                            ctas_per_sm=o.ctas_per_sm, tile=o.tile, cull=1)

    def step_c():
        P.copy_(P0)
        bude.refine_device(deck, P, steps=steps, step0=0.05, energies=E, opts=oc)

    ms_c, _ = timed(step_c, 5, 2)
    same = bool(torch.equal(Pa, P) and torch.equal(Ea, E))
    deck.close()
    t = statistics.mean(ms)
    # the graph evaluates the adjoint steps + 1 times (the start and each
    # trial); the two element-wise kernels per step are negligible beside it
    m = MEASURED_EXECUTED_ADJOINT
    executed = None
    if (kernel_sha(), variant, o.ppwi) == (m["kernel_sha256_16"], m["variant"], m["ppwi"]):
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
        tf = m["flop_per_pair"] * 64 * 2672 * P.shape[1] * (steps + 1) / (t / 1e3) / 1e12
        executed = {"adjoint_evaluations": steps + 1, "flop_per_pair": m["flop_per_pair"],
                    "tflops": tf, "frac_fp32_peak": tf / peak,
                    "source": "the adjoint's ncu opcode counters; time of the whole graph"}
    return {"workload": f"{steps} steps x 16384 poses, 64 lig x 2672 pro, seed 4",
            "variant": variant, "ms": t, "pose_steps_per_s": steps * P.shape[1] / (t / 1e3),
            "executed": executed,
            "graph_launches_per_call": 1, "kernels_per_call": launches // 5,
            "mean_energy_before": e0, "mean_energy_after": Ea.mean().item(),
            "cull_ms": statistics.mean(ms_c), "cull_bit_identical": same}


def cull_throughput(bude, tune, deck, poses, out, ms_brute, timed, variant="fast"):
    """The headline deck with cutoff culling on: warps skip protein atoms that
    are beyond the cutoff for all their poses.  Reported beside, never as, the
    headline: it evaluates fewer pairs than Eq. 3 counts.  The energies must
    be bit-identical to the brute-force kernel of the same launch shape."""
    import torch
    o = tune.lookup(variant, 64, 2672, poses.shape[1], mode="cull") or \
        bude.LaunchOptions(variant=variant, ppwi=8, block=256, cull=1)
    o.cull = 1
    ms, _ = timed(lambda: bude.energies(deck, poses, out=out, opts=o), 20, 3)
    culled = out.clone()
    plain = bude.LaunchOptions(variant=variant, ppwi=o.ppwi, block=o.block,
                               ctas_per_sm=o.ctas_per_sm, tile=o.tile, cull=0)
    bude.energies(deck, poses, out=out, opts=plain)
    torch.cuda.synchronize()
    t = statistics.mean(ms)
    return {"workload": "the headline deck, 64 lig x 2672 pro x 65536 poses", "variant": variant,
            "ms": t, "poses_per_s": poses.shape[1] / (t / 1e3),
            "speedup_vs_headline": ms_brute / t,
            "bit_identical_to_unculled": bool(torch.equal(culled, out)),
            "opts": {"ppwi": o.ppwi, "block": o.block, "ctas_per_sm": o.ctas_per_sm},
            "note": "pairs beyond R + 4 A are skipped warp-wide; not an Eq. 3 FLOP rate"}


def param_grad_throughput(bude, synth, tune, dev, timed, variant="fast"):
    """Gradient of the pose-energy sum w.r.t. ligand coordinates and forcefield
    parameters over 16384 poses of the 64 x 2672 deck."""
    import torch
    D = synth.make_deck(4, **synth.GRAD)
    deck = bude.Deck(D, device=dev)
    P = torch.from_numpy(D["poses"]).to(dev)
    o = tune.lookup(variant, 64, 2672, D["poses"].shape[1], mode="param") or \
        bude.LaunchOptions(variant=variant, ppwi=8, block=384)
    ms, launches = timed(lambda: bude.param_grad(deck, P, opts=o), 5, 2)
    deck.close()
    t = statistics.mean(ms)
    m = MEASURED_EXECUTED_PARAM
    executed = None
    if (kernel_sha(("bude_kernels.cuh", "bude_param.cu")), variant, o.ppwi) == \
            (m["kernel_sha256_16"], m["variant"], m["ppwi"]):
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
        tf = m["flop_per_pair"] * 64 * 2672 * P.shape[1] / (t / 1e3) / 1e12
        executed = {"flop_per_pair": m["flop_per_pair"], "tflops": tf, "frac_fp32_peak": tf / peak,
                    "source": "ncu opcode counters of param_kernel; time of the whole call "
                              "(three kernels)"}
    return {"workload": "dL/d(ligand xyz, radius, hardness, elsc), L = sum of 16384 pose "
                        "energies, 64 lig x 2672 pro, seed 4",
            "variant": variant, "ms": t, "poses_per_s": P.shape[1] / (t / 1e3),
            "executed": executed,
            "kernels_per_call": launches // 5,
            "opts": {"ppwi": o.ppwi, "block": o.block, "ctas_per_sm": o.ctas_per_sm}}


def hbm_calibration(bude, dev, timed, peak_gbs, stencil_l=1024, stream_sizes=(1 << 25, 1 << 28)):
    """The paper's memory-bound kernels on this GPU: GB/s by Eq. 2 (BabelStream,
    2^25 and 2^28 elements) and Eq. 1 (seven-point stencil, FP32 L=1024, FP64
    L=512), against the measured copy bandwidth."""
    import torch
    out = {}
    for dtype, name in ((torch.float32, "f32"), (torch.float64, "f64")):
        item = torch.tensor([], dtype=dtype).element_size()
        for n in stream_sizes:
            a = torch.full((n,), 0.1, dtype=dtype, device=dev)
            b = torch.full((n,), 0.2, dtype=dtype, device=dev)
            c = torch.zeros(n, dtype=dtype, device=dev)
            d = torch.empty((), dtype=torch.float64, device=dev)
            ops = {"copy": (lambda: bude.stream_op("copy", a=a, c=c), 2),
                   "mul": (lambda: bude.stream_op("mul", b=b, c=c, scalar=0.4), 2),
                   "add": (lambda: bude.stream_op("add", a=a, b=b, c=c), 3),
                   "triad": (lambda: bude.stream_op("triad", a=a, b=b, c=c, scalar=0.4), 3),
                   "dot": (lambda: bude.stream_op("dot", a=a, b=b, dot_out=d), 2)}
            for op, (fn, arrays) in ops.items():
                ms, _ = timed(fn, 20, 3)
                gbs = arrays * n * item / (statistics.median(ms) / 1e3) / 1e9
                out[f"{op}_{name}_2^{n.bit_length() - 1}"] = {
                    "gb_s": gbs, "frac_of_measured_copy": gbs / peak_gbs}
            del a, b, c
            torch.cuda.empty_cache()
        L = stencil_l if name == "f32" else stencil_l // 2
        u = torch.rand((L, L, L), dtype=dtype, device=dev)
        f = torch.zeros_like(u)
        ms, _ = timed(lambda: bude.laplacian(u, f, 1.0, 1.0, 1.0, -6.0), 10, 3)
        fetch = L ** 3 - 8 - 12 * (L - 2)
        write = (L - 2) ** 3
        gbs = (fetch + write) * item / (statistics.median(ms) / 1e3) / 1e9
        out[f"stencil_{name}_L{L}"] = {"gb_s": gbs, "frac_of_measured_copy": gbs / peak_gbs,
                                        "ms": statistics.median(ms)}
        if name == "f64":
            # 7 FP64 instructions per interior point (3 sums, 1 product, 3 FMAs)
            # against GB300's nominal FP64 rate of 1.25 TFLOP/s, i.e. 6.25e11
            # FMA instructions/s: the bound of this kernel on this GPU
            ips = 7.0 * (L - 2) ** 3 / (statistics.median(ms) / 1e3)
            out[f"stencil_{name}_L{L}"].update({
                "fp64_instructions_per_s": ips, "frac_of_nominal_fp64_rate": ips / 6.25e11})
        del u, f
        torch.cuda.empty_cache()
    return out


def hartree_fock(bude, synth, dev, timed, sizes=(64, 128, 256), variants=("ieee", "fp64")):
    """Two-electron Fock build for synthetic helium lattices of 64, 128 and 256
    atoms with 3 primitives per atom (the paper's Table 4 sizes), FP32
    integrals with FP64 accumulation and all-FP64, Schwarz threshold 1e-12."""
    import torch
    out = {}
    for n in sizes:
        s = synth.make_he_lattice(11, n, 3)
        hf = bude.HartreeFock(s["geom"], s["xpnt"], s["coef"], device=dev)
        D = torch.from_numpy(s["dens"]).to(dev)
        row = {}
        for v in variants:
            reps = 1 if (v == "fp64" and n == 256) else 5
            ms, _ = timed(lambda: hf.fock(D, tol=1e-12, variant=v), reps, 1)
            row["fp32_integrals_ms" if v == "ieee" else "fp64_ms"] = statistics.median(ms)
        if len(variants) < 2:
            out[f"a={n} ngauss=3"] = row
            hf.close()
            continue
        G64 = hf.fock(D, tol=1e-12, variant="fp64")
        G32 = hf.fock(D, tol=1e-12, variant="ieee")
        row["fp32_vs_fp64_max_rel"] = ((G32 - G64).abs().max() / G64.abs().max()).item()
        # surviving quartets and primitive integrals per second (ngauss^4 each)
        q = hf.quartets(1e-12)
        row["quartets"] = q
        row["fp32_primitive_integrals_per_s"] = q * 81 / (row["fp32_integrals_ms"] / 1e3)
        row["fp64_primitive_integrals_per_s"] = q * 81 / (row["fp64_ms"] / 1e3)
        m = MEASURED_HF64_PIPE
        if (kernel_sha(("bude_hf.cu",)), n) == (m["kernel_sha256_16"], m["atoms"]):
            ips = m["ops_per_primitive"] * row["fp64_primitive_integrals_per_s"]
            row["fp64_pipe_instructions_per_s"] = ips
            row["fp64_frac_of_nominal_fp64_rate"] = ips / NOMINAL_FP64_INST_PER_S
        out[f"a={n} ngauss=3"] = row
        hf.close()
    return out


def arm_config(shard, shape, world, variant, ppwi, block, ctas_per_sm, flush_mb):
    """config of the JSON line: the workload and the GPU launch it is timed
    in.  The reference arm reports the same dict for the same run."""
    return {"workload": workload_name(shard, shape, world),
            "variant": variant, "ppwi": ppwi, "block": block, "ctas_per_sm": ctas_per_sm,
            "l2": f"flushed ({flush_mb} MiB write) before every timed step",
            "parallelism": {"decks": f"independent decks per GPU x{world}",
                            "poses": f"one deck's poses split over {world} GPUs",
                            "batch": f"64-deck batch split over {world} GPUs"}[shard],
            "shard": shard}


def default_launch(variant):
    """(ppwi, block, ctas_per_sm) the GPU arm takes for the full deck: the
    tuned entry for this GPU (any GB300 entry when no GPU is visible), else
    the library's compiled-in default shape."""
    from paper_2509_21039_gb300 import tune
    table = tune.load_table()
    suffix = f"|{variant}|plain|{tune.bucket(FULL['n_lig'], FULL['n_pro'], FULL['n_poses'])}"
    keys = [k for k in table if k.endswith(suffix)]
    try:
        import torch
        if torch.cuda.is_available():
            keys = [k for k in keys if k.startswith(tune.gpu_name() + "|")] or keys
    except Exception:
        pass
    if keys:
        e = table[sorted(keys)[0]]
        return e["ppwi"], e["block"], e["ctas_per_sm"]
    return 8, 256, 1


def workload_name(shard, shape, world):
    """config.workload for a shard mode."""
    deck = (f"{shape['n_lig']} lig x {shape['n_pro']} pro x {shape['n_poses']} poses, "
            f"34 types")
    if shard == "decks":
        return f"deck {deck}, seed 1+rank (one deck per GPU)"
    if shard == "poses":
        return f"deck {deck}, seed 1, poses split over {world} GPUs"
    return ("64 decks, log-uniform lig 8-128, pro 500-5000, poses 1024-65536, 34 types, "
            f"seed 3, split over {world} GPUs")


def batched_oracle_errors(decks_np, samples):
    """Largest scaled error |E - E_ref| / max(A_ref, 1) of the batched and the
    plain arm over the sampled poses of every deck (the oracle's energies and
    absolute-term sums at those poses)."""
    import oracle
    eb = ep = 0.0
    for d, (idx, a, b) in zip(decks_np, samples):
        ref, A = oracle.energies(d, np.ascontiguousarray(d["poses"][:, idx]), n_threads=-1,
                                 with_abs=True)
        sc = np.maximum(A, 1.0)
        eb = max(eb, float((np.abs(a.astype(np.float64) - ref) / sc).max()))
        ep = max(ep, float((np.abs(b.astype(np.float64) - ref) / sc).max()))
    return eb, ep


def _r(x, digits=4):
    """x rounded to a few significant digits (None stays None)."""
    if x is None:
        return None
    if isinstance(x, bool) or not isinstance(x, (int, float)):
        return x
    return float(f"{x:.{digits}g}")


def summary(line):
    """The figures a reader looks for first, rounded, as the line's last key
    (a consumer that keeps only the end of the line still sees them)."""
    rf = line["roofline"]
    out = {"headline": {"variant": line["config"]["variant"], "poses_s": _r(line["value"]),
                        "ms": _r(line["ms_per_step"]), "eq3_frac": _r(rf["frac"]),
                        "exec_frac": _r(rf.get("executed_frac")),
                        "e2e_poses_s": _r(line["e2e"]["value"])}}
    for v, row in line.get("variants", {}).items():
        out[v] = {"poses_s": _r(row["poses_per_s"]), "eq3_frac": _r(row["frac_fp32_peak"]),
                  "err": _r(row["scaled_err_max"], 2)}
        if row.get("frac_of_nominal_fp64_rate") is not None:
            out[v]["fp64_rate_frac"] = _r(row["frac_of_nominal_fp64_rate"])
    b = line.get("batched")
    if b:
        out["batched"] = {"ms": _r(b["batched_ms"]), "plain_ms": _r(b["plain_ms"]),
                          "speedup": _r(b["speedup"]),
                          "eq3_frac": _r(b["batched_eq3_frac_fp32_peak"]),
                          "plain_tuned": f"{b['plain_tuned_decks']}/64",
                          "err_b": _r(b.get("scaled_err_max_batched"), 2),
                          "err_p": _r(b.get("scaled_err_max_plain"), 2)}
    a = line.get("adjoint")
    if a:
        out["adjoint"] = {"ms": _r(a["ms"]),
                          "exec_frac": _r((a.get("executed") or {}).get("frac_fp32_peak"))}
    if line.get("refine"):
        out["refine_ms"] = _r(line["refine"]["ms"])
    if line.get("param_grad"):
        out["param_grad_ms"] = _r(line["param_grad"]["ms"])
    if line.get("cull"):
        out["cull"] = {"ms": _r(line["cull"]["ms"]),
                       "same": line["cull"]["bit_identical_to_unculled"]}
    if line.get("cpu_baseline"):
        out["oracle_poses_s"] = _r(line["cpu_baseline"]["value"])
    return out


def reference_arm(args):
    """The FP64 oracle as it stands, timed on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2509_21039_gb300 import synth
    import oracle
    oracle.build()
    D = synth.make_deck(1, **FULL)
    cores = oracle.max_threads()
    # per step: a bounded sample of the poses, sized from a calibration call so
    # that warm-up plus timed steps take about a minute in all
    k = max(4 * cores, 64)
    t0 = time.perf_counter()
    oracle.energies(D, D["poses"][:, :k], n_threads=-1)
    rate = k / max(time.perf_counter() - t0, 1e-6)
    budget = min(0.5, 60.0 / max(args.steps + args.warmup, 1))
    per_step = int(min(FULL["n_poses"] // 2, max(k, rate * budget)))
    for _ in range(args.warmup):
        oracle.energies(D, D["poses"][:, :per_step], n_threads=-1)
    times = []
    for s in range(args.steps):
        lo = (s * per_step) % (FULL["n_poses"] - per_step)
        t0 = time.perf_counter()
        oracle.energies(D, D["poses"][:, lo:lo + per_step], n_threads=-1)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    val = per_step / (ms / 1e3)
    sample = f"{per_step} poses per step of the 64x2672x65536 deck, FP64, {cores} threads"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "poses/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            # the GPU arm's config for the same run; the oracle itself runs on the
            # host (FP64, no L2 flush): its sample is described in cpu_baseline
            "config": arm_config(args.shard, dict(FULL), args.gpus, args.variant,
                                 *default_launch(args.variant), args.flush_mb),
            "cpu_baseline": {"value": val, "unit": "poses/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "poses/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default="fast", choices=["ieee", "fast", "comp"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the variant table and the batched comparison")
    ap.add_argument("--small", action="store_true", help="26x938x4096 deck")
    ap.add_argument("--poses", type=int, default=0, help="override the pose count (profiling)")
    ap.add_argument("--flush-mb", type=int, default=256, help="L2 flush buffer, MiB")
    ap.add_argument("--clocks-csv", default=None,
                    help="also write the clock samples of the timed region to this CSV file")
    ap.add_argument("--hbm-only", action="store_true",
                    help="only the memory-bound calibration kernels (profiling)")
    ap.add_argument("--stencil-l", type=int, default=1024,
                    help="FP32 stencil grid side with --hbm-only (FP64: half)")
    ap.add_argument("--stream-log2", default="25",
                    help="BabelStream sizes with --hbm-only, as log2 of the element count")
    ap.add_argument("--param-only", action="store_true",
                    help="only the forcefield-gradient extra (profiling)")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="only the pose-gradient (adjoint) extra (profiling)")
    ap.add_argument("--refine-only", action="store_true",
                    help="only the refinement extra (profiling)")
    ap.add_argument("--fp64-only", action="store_true",
                    help="only the FP64 variant on the full deck's first 4096 poses (profiling)")
    ap.add_argument("--hf-only", type=int, default=0, metavar="ATOMS",
                    help="only the Fock build on this many atoms (profiling)")
    ap.add_argument("--hf-variant", default="ieee", choices=["ieee", "fp64"],
                    help="with --hf-only: FP32 integrals (ieee) or all FP64")
    ap.add_argument("--shard", default="decks", choices=["decks", "poses", "batch"],
                    help="decks: one deck per rank (weak scaling, the default); poses: one "
                         "full-size deck's poses split over the ranks; batch: the 64-deck "
                         "uneven batch split over the ranks (both strong scaling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    import torch.distributed as dist
    from paper_2509_21039_gb300 import bude, synth, tune

    from paper_2509_21039_gb300 import dist as bdist
    rank, local, world = bdist.world()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    # collectives run while every rank is in the timed part; once the other
    # ranks have left, rank 0 times alone
    together = [world > 1]

    def barrier():
        if together[0]:
            dist.barrier()

    shape = dict(SMALL if args.small else FULL)
    if args.poses:
        shape["n_poses"] = args.poses
    # The work of this rank (dist.shard_pieces; no data-path collective):
    #   decks  its own deck, seed 1 + rank (independent problems, weak scaling)
    #   poses  a contiguous slice of the poses of the seed-1 deck (strong)
    #   batch  its pieces of the 64-deck uneven batch (strong)
    shard = args.shard
    batch_np = None
    if shard == "batch":
        batch_np = synth.make_batched(3, 64)
        shapes_b = [(len(d["lig_type"]), len(d["pro_type"]), d["poses"].shape[1])
                    for d in batch_np]
        pieces, total_units, scaling = bdist.shard_pieces("batch", rank, world,
                                                          batch_shapes=shapes_b)
        total_alg = sum(algorithmic_flops(*sh) for sh in shapes_b)
    else:
        pieces, total_units, scaling = bdist.shard_pieces(shard, rank, world,
                                                          n_poses=shape["n_poses"])
        total_alg = algorithmic_flops(shape["n_lig"], shape["n_pro"], total_units)
    flush = torch.empty(max(args.flush_mb, 1) << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    # launch shapes found by the autotuner on GB300 (tuned.json), else defaults
    tune.apply(n_lig=FULL["n_lig"], n_pro=FULL["n_pro"], n_poses=FULL["n_poses"])
    resolved = bude.default_options(args.variant)
    opts = resolved

    if shard != "batch":
        (_, lo, hi), = pieces
        D = synth.make_deck(bdist.rank_seed(1, rank) if shard == "decks" else 1, **shape)
        if (lo, hi) != (0, shape["n_poses"]):
            D["poses"] = np.ascontiguousarray(D["poses"][:, lo:hi])
        deck = bude.Deck(D, device=dev)
        poses = torch.from_numpy(D["poses"]).to(dev)
        n = poses.shape[1]
        out = torch.empty(n, dtype=torch.float32, device=dev)

        def step():
            bude.energies(deck, poses, out=out, opts=opts)
    else:
        # one batched launch over this rank's pieces, in the batch's tuned shape
        D = None
        e = tune.load_table().get(tune.key(args.variant, "n64", "batched"))
        bopts = (bude.LaunchOptions(variant=args.variant, ppwi=e["ppwi"], block=e["block"],
                                    ctas_per_sm=e["ctas_per_sm"], tile=e["tile"])
                 if e else opts)
        deck_of = {i: bude.Deck(batch_np[i], device=dev) for i in sorted({p[0] for p in pieces})}
        b_decks = [deck_of[i] for i, _, _ in pieces]
        b_host = [torch.from_numpy(np.ascontiguousarray(batch_np[i]["poses"][:, a:b]))
                  for i, a, b in pieces]
        b_poses = [h.to(dev) for h in b_host]
        b_outs = [torch.empty(h.shape[1], dtype=torch.float32, device=dev) for h in b_host]
        n = sum(h.shape[1] for h in b_host)

        def step():
            if b_decks:
                bude.energies_batched(b_decks, b_poses, b_outs, opts=bopts)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            flush.zero_()
            fn()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        evs = []
        launches = 0
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            launches += bude.launch_count()
            evs.append((a, b))
        torch.cuda.synchronize()
        barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms, launches

    if args.param_only:
        res = param_grad_throughput(bude, synth, tune, dev, timed, variant=args.variant)
        if rank == 0:
            print(json.dumps({"param_grad": res}), flush=True)
        return

    if args.adjoint_only:
        res = adjoint_throughput(bude, synth, tune, dev, timed, variant=args.variant)
        if rank == 0:
            print(json.dumps({"adjoint": res}), flush=True)
        return

    if args.refine_only:
        res = refine_throughput(bude, synth, tune, dev, timed, variant=args.variant)
        if rank == 0:
            print(json.dumps({"refine": res}), flush=True)
        return

    if args.fp64_only:
        res = fp64_throughput(bude, synth, dev, timed)
        if rank == 0:
            print(json.dumps({"fp64": res}), flush=True)
        return

    if args.hf_only:
        res = hartree_fock(bude, synth, dev, timed, sizes=(args.hf_only,),
                           variants=(args.hf_variant,))
        if rank == 0:
            print(json.dumps({"hartree_fock": res}), flush=True)
        return

    if args.hbm_only:
        # profiling entry: the stencil and BabelStream at the given sizes
        sizes = tuple(1 << int(x) for x in args.stream_log2.split(","))
        res = hbm_calibration(bude, dev, timed, measured_peaks().get("hbm_gbs", 6800.0),
                              stencil_l=args.stencil_l, stream_sizes=sizes)
        if rank == 0:
            print(json.dumps({"hbm_calibration": res}), flush=True)
        return

    with ClockSampler(smi_id(local), args.clocks_csv) as clk:
        ms, launches = timed(step, args.steps, args.warmup)
    ms_mean = bdist.max_over_ranks(statistics.mean(ms), dev)
    value = total_units / (ms_mean / 1e3)

    if shard != "batch":
        # end to end through the C ABI's host-buffer call: pinned host poses in,
        # host energies out, both copies made by the library on the stream
        host_poses = torch.from_numpy(D["poses"]).pin_memory()
        host_out = torch.empty(n, dtype=torch.float32).pin_memory()
        h2d, d2h = host_poses.numel() * 4, host_out.numel() * 4

        def e2e_step():
            bude.energies_host(deck, host_poses, out=host_out, opts=opts)
    else:
        # the batched call a user makes from host buffers: pinned poses copied
        # in, one batched launch, energies copied back
        pin_in = [h.pin_memory() for h in b_host]
        pin_out = [torch.empty(h.shape[1], dtype=torch.float32).pin_memory() for h in b_host]
        h2d = sum(h.numel() * 4 for h in pin_in)
        d2h = sum(h.numel() * 4 for h in pin_out)

        def e2e_step():
            for h, d in zip(pin_in, b_poses):
                d.copy_(h, non_blocking=True)
            step()
            for o, h in zip(b_outs, pin_out):
                h.copy_(o, non_blocking=True)
            stream.synchronize()

    e2e_ms, _ = timed(e2e_step, max(3, args.steps // 2), 2)
    e2e_mean = bdist.max_over_ranks(statistics.mean(e2e_ms), dev)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    together[0] = False
    if world > 1:
        # the single-GPU extras and the host-side oracle belong to the N = 1 line
        args.no_extras = True
        args.no_cpu_baseline = True

    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clocks = clk.summary()
    peak_max = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    # per GPU: the FLOPs of all ranks' launches over the slowest rank's time,
    # shared out over the GPUs
    achieved = total_alg / world / (ms_mean / 1e3) / 1e12
    ppwi = resolved.ppwi
    if shard == "batch":
        ppwi = bopts.ppwi
    if shard == "batch":
        sh = [(len(batch_np[i]["lig_type"]), len(batch_np[i]["pro_type"]), b - a)
              for i, a, b in pieces]
        kernel = f"pose_kernel<{args.variant}, P={ppwi}>, one batched launch"
        block = bopts.block
    else:
        sh = [(shape["n_lig"], shape["n_pro"], n)]
        kernel = f"pose_kernel<{args.variant}, P={ppwi}>"
        block = resolved.block
    alg_rank = sum(algorithmic_flops(*x) for x in sh)
    roofline = {
        "bound": "alu", "achieved": achieved, "peak": peak_max, "unit": "TFLOP/s",
        "frac": achieved / peak_max,
        "traffic": measured_traffic(args.variant, ppwi, block, n) if shard != "batch" else None,
        "traffic_source": (traffic_source(args.variant, ppwi, block, n) if shard != "batch"
                           else "null: DRAM bytes were captured for the single-deck launch"),
        "algorithmic_bytes": int(sum(x[2] * 28 + 4 * (x[0] + x[1]) * 4 for x in sh)),
        "kernel": kernel,
        "flops_per_launch": alg_rank,
        "flop_count": "Eq. 3 in the many-poses limit: 28 + nlig (18 + 30 npro) per pose",
        "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {SM_MAX_MHZ:.0f} MHz",
        "eq3_tflops_at_ppwi": sum(eq3_flops(*x, ppwi) for x in sh) / (ms_mean / 1e3) / 1e12,
    }
    xf = measured_executed(args.variant)
    roofline["executed_source"] = executed_source(args.variant)
    if xf is not None and shard != "batch":
        # FLOPs the kernel executes (ncu opcode counters), not Eq. 3's count,
        # per GPU as achieved above
        pairs = shape["n_lig"] * shape["n_pro"] * total_units / world
        roofline["executed_flop_per_pair"] = xf
        roofline["executed_tflops"] = xf * pairs / (ms_mean / 1e3) / 1e12
        roofline["executed_frac"] = roofline["executed_tflops"] / peak_max
    if clocks:
        clk_peak = sms * FP32_LANES_PER_SM * 2 * clocks["sm_mhz"] * 1e6 / 1e12
        roofline["frac_at_measured_clock"] = achieved / clk_peak

    line = {
        "metric": METRIC, "value": value, "unit": "poses/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_mean,
        "ms_per_step_median": statistics.median(ms), "ms_per_step_best": min(ms),
        "higher_is_better": True, "scaling": scaling, "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": arm_config(shard, shape, world, args.variant, ppwi, block,
                             (bopts if shard == "batch" else resolved).ctas_per_sm,
                             args.flush_mb),
        "gpu_launches": int(launches),
        "e2e": {"value": total_units / (e2e_mean / 1e3), "unit": "poses/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "roofline": roofline,
        "clocks": clocks,
    }

    batched_private = {}
    if shard != "decks":
        # the extras and the variant table belong to the single-deck workload
        args.no_extras = True
        if not args.no_cpu_baseline:
            D = synth.make_deck(1, **FULL)
    if not args.no_extras:
        line["hbm_calibration"] = hbm_calibration(bude, dev, timed,
                                                  peaks.get("hbm_gbs", 6800.0))
        line["hartree_fock"] = hartree_fock(bude, synth, dev, timed)
        line["cull"] = cull_throughput(bude, tune, deck, poses, out, ms_mean, timed)
        line["batched"] = batched_vs_plain(bude, synth, tune, dev, timed)
        batched_private = {k: line["batched"].pop(k) for k in ("_samples", "_decks")}
        line["adjoint"] = adjoint_throughput(bude, synth, tune, dev, timed)
        line["refine"] = refine_throughput(bude, synth, tune, dev, timed)
        line["param_grad"] = param_grad_throughput(bude, synth, tune, dev, timed)

    # CPU-baseline leg: the FP64 oracle on a bounded sample of the same poses.
    # Its sample energies also give each variant's error on that sample.
    if not args.no_cpu_baseline:
        v, k, dt, cores, ref, A = cpu_baseline_leg(D, D["poses"].shape[1])
        v1, k1 = cpu_single_thread(D)
        line["cpu_baseline"] = {"value": v, "unit": "poses/s", "cores": cores, "kind": "oracle",
                                "sample": f"first {k} poses of the same deck, FP64, best of 3 "
                                          f"runs ({dt:.1f} s)",
                                "single_thread_value": v1,
                                "single_thread_sample": f"first {k1} poses, 1 thread, best of 3"}
        if not args.no_extras:
            variants = {}
            # FP64 runs ~60x slower on GB300: time it on the first 4096 poses
            n64 = min(k, 4096)
            poses64 = poses[:, :n64].contiguous()
            out64 = torch.empty(n64, dtype=torch.float32, device=dev)
            for vname in ("ieee", "fast", "comp", "fp64"):
                o = bude.LaunchOptions(variant=vname)
                if vname == "fp64":
                    vms, _ = timed(lambda: bude.energies(deck, poses64, out=out64, opts=o), 2, 1)
                    E = out64.cpu().numpy().astype(np.float64)
                    npos, rf, Af = n64, ref[:n64], A[:n64]
                else:
                    vms, _ = timed(lambda: bude.energies(deck, poses, out=out, opts=o), 5, 2)
                    E = out[:k].cpu().numpy().astype(np.float64)
                    npos, rf, Af = n, ref, A
                ab = np.abs(E - rf)
                err = ab / np.maximum(Af, 1.0)
                rel = ab / np.maximum(np.abs(rf), 1e-30)
                t = statistics.mean(vms) / 1e3
                variants[vname] = {"poses_per_s": npos / t,
                                   "frac_fp32_peak": (alg_rank * npos / n) / t / 1e12 / peak_max,
                                   "scaled_err_max": float(err.max()),
                                   "abs_err_median": float(np.median(ab)),
                                   "abs_err_max": float(ab.max()),
                                   "rel_err_median": float(np.median(rel)),
                                   "rel_err_p99": float(np.percentile(rel, 99)),
                                   "rel_err_max": float(rel.max()),
                                   "error_sample_poses": int(len(rf)),
                                   "timed_poses": int(npos)}
                if vname == "fp64":
                    ips, frac = fp64_pipe_fraction(o.ppwi if o.ppwi else
                                                   bude.default_options("fp64").ppwi,
                                                   shape["n_lig"] * shape["n_pro"] * npos / t)
                    if frac is not None:
                        variants[vname]["fp64_pipe_instructions_per_s"] = ips
                        variants[vname]["frac_of_nominal_fp64_rate"] = frac
                xv = measured_executed(vname)
                if xv is not None:
                    variants[vname]["executed_frac"] = (xv * shape["n_lig"] * shape["n_pro"] * npos
                                                        / t / 1e12 / peak_max)
            line["variants"] = variants
            if batched_private:
                # both batched-comparison arms against the oracle at the sampled poses
                eb, ep = batched_oracle_errors(batched_private["_decks"],
                                               batched_private["_samples"])
                line["batched"]["scaled_err_max_batched"] = eb
                line["batched"]["scaled_err_max_plain"] = ep
                line["batched"]["error_sample"] = "16 poses per deck (the last included), FP64 oracle"
    line["summary"] = summary(line)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
