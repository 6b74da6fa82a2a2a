"""Host-side logic that needs no GPU: the Eq. 3 FLOP count and the roofline
bookkeeping of bench.py, the autotuner's table and search space, the seeded
input generators and the options struct of the binding."""
import ctypes
import importlib.util
import math
import os

import numpy as np
import pytest

from paper_2509_21039_gb300 import bude, synth, tune

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_eq3_counts_one_work_item_by_hand(bench):
    # Eq. 3 for one work-item of P poses: 28 P + nlig (2 + 18 P + npro (10 + 30 P))
    # 2 ligand atoms, 3 protein atoms, P = 4: 112 + 2 (2 + 72 + 3 * 130) = 1040 per item,
    # and 8 poses are two items
    assert bench.eq3_flops(2, 3, 8, 4) == 2080
    # P = 1: 28 + 2 (2 + 18 + 3 * 40) = 308 per pose
    assert bench.eq3_flops(2, 3, 5, 1) == 5 * 308


def test_eq3_many_pose_limit_is_the_algorithmic_count(bench):
    # the per-pose Eq. 3 count falls towards 28 + nlig (18 + 30 npro) as P grows;
    # the pose-independent 2 + 10 npro per ligand atom is spread over P poses
    n_lig, n_pro, n = 64, 2672, 65536
    alg = bench.algorithmic_flops(n_lig, n_pro, n)
    assert alg == n * (28 + n_lig * (18 + 30 * n_pro))
    prev = None
    for p in (1, 2, 4, 8, 16, 1024):
        e = bench.eq3_flops(n_lig, n_pro, n, p)
        assert e > alg
        assert prev is None or e < prev
        assert e - alg == pytest.approx(n * n_lig * (2 + 10 * n_pro) / p)
        prev = e
    # the full-size config: 3.363e11 FLOP per launch
    assert alg == pytest.approx(3.363e11, rel=1e-3)


def test_measured_constants_are_gated_by_source_and_shape(bench):
    m = bench.MEASURED_TRAFFIC
    sha = bench.kernel_sha()
    assert len(sha) == 16
    hit = bench.measured_traffic(m["variant"], m["ppwi"], m["block"], bench.FULL["n_poses"])
    assert hit == (m["bytes"] if sha == m["kernel_sha256_16"] else None)
    # any other shape or workload is never reported
    assert bench.measured_traffic(m["variant"], m["ppwi"] * 2, m["block"], bench.FULL["n_poses"]) is None
    assert bench.measured_traffic(m["variant"], m["ppwi"], m["block"], 4096) is None
    assert bench.measured_traffic("ieee", m["ppwi"], m["block"], bench.FULL["n_poses"]) is None
    x = bench.measured_executed("fast")
    assert x is None or 10.0 < x <= 30.0


def test_tuner_buckets_and_keys():
    assert tune.bucket(64, 2672, 65536) == "p16_k18"
    assert tune.bucket(26, 938, 4096) == "p12_k15"
    assert tune.bucket(0, 0, 0) == "p0_k0"
    b = tune.bucket(64, 2672, 16384)
    assert b == "p14_k18"


def test_tuner_search_space_respects_what_is_built():
    ps = {o.ppwi for o in tune.candidates("fp64")}
    assert ps == {1, 2, 4}
    ps = {o.ppwi for o in tune.candidates("ieee", grad=True)}
    assert ps == {1, 2, 4, 8}
    cs = list(tune.candidates("fast", cull=1))
    assert {o.ppwi for o in cs} == {2, 4, 8, 16} and all(o.cull == 1 for o in cs)
    n = len(list(tune.candidates("fast")))
    assert n == 5 * 7 * 4


def test_tuned_table_record_and_lookup_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "gpu_name", lambda: "TEST_GPU")
    t = {}
    o = bude.LaunchOptions(variant="fast", ppwi=16, block=384, ctas_per_sm=2, tile=0, cull=1)
    tune.record(t, tune.key("fast", "p16_k18", "cull"), 2.5, o)
    tune.record(t, tune.key("fast", "p16_k18"), 4.8,
                bude.LaunchOptions(variant="fast", ppwi=8, block=512, ctas_per_sm=1))
    path = str(tmp_path / "t.json")
    tune.save_table(t, path)
    t2 = tune.load_table(path)
    assert t2 == t
    got = tune.lookup("fast", 64, 2672, 65536, mode="cull", table=t2)
    assert (got.ppwi, got.block, got.ctas_per_sm, got.cull) == (16, 384, 2, 1)
    got = tune.lookup("fast", 64, 2672, 65536, table=t2)
    assert (got.ppwi, got.block, got.cull) == (8, 512, 0)
    assert tune.lookup("ieee", 64, 2672, 65536, table=t2) is None
    assert tune.load_table(str(tmp_path / "missing.json")) == {}


def test_committed_tuned_table_is_well_formed():
    t = tune.load_table()
    assert t, "tuned.json is committed"
    for k, e in t.items():
        gpu, variant, mode, b = k.split("|")
        assert variant in ("fast", "ieee", "comp", "fp64")
        assert mode in ("plain", "grad", "batched", "cull", "grad_cull", "param")
        assert e["ppwi"] in (1, 2, 4, 8, 16)
        assert 64 <= e["block"] <= 1024 and e["block"] % 32 == 0
        assert 1 <= e["ctas_per_sm"] <= 4 and e["ms"] > 0
        if mode.startswith("grad") or mode == "param":
            assert e["ppwi"] <= 8
        if e.get("cull"):
            assert e["ppwi"] % 2 == 0
    full = [k for k in t if k.endswith("|fast|plain|p16_k18")]
    assert full, "the headline workload has a tuned FAST shape"


def test_options_struct_matches_the_header():
    # six int32 fields in the order of include/bude.h
    assert ctypes.sizeof(bude.Options) == 6 * 4
    names = [f[0] for f in bude.Options._fields_]
    assert names == ["variant", "ppwi", "block", "tile", "ctas_per_sm", "cull"]
    text = open(os.path.join(ROOT, "include", "bude.h")).read()
    body = text[text.index("typedef struct {\n    int32_t variant;"):]
    body = body[:body.index("} bude_options;")]
    assert [line.split()[1].rstrip(";") for line in body.splitlines()[1:]] == names


def test_synthetic_decks_are_seeded_and_in_range():
    a = synth.make_deck(3, 20, 100, 34, 50)
    b = synth.make_deck(3, 20, 100, 34, 50)
    c = synth.make_deck(4, 20, 100, 34, 50)
    for k in synth.DECK_KEYS + ("poses",):
        np.testing.assert_array_equal(a[k], b[k])
    assert not np.array_equal(a["pro_xyz"], c["pro_xyz"])
    assert a["pro_xyz"].shape == (100, 3) and a["lig_xyz"].shape == (20, 3)
    assert a["poses"].shape == (6, 50) and a["poses"].dtype == np.float32
    assert np.all(np.abs(a["pro_xyz"]) <= 20) and np.all(np.abs(a["lig_xyz"]) <= 4)
    assert a["pro_type"].min() >= 0 and a["pro_type"].max() < 34
    assert np.all((a["radius"] >= 1.4) & (a["radius"] <= 2.2))
    assert np.all((a["hardness"] >= 0) & (a["hardness"] <= 40))
    assert set(np.unique(a["hbtype"])) <= {0, 1, 2}
    assert np.all(np.abs(a["poses"][:3]) <= math.pi) and np.all(np.abs(a["poses"][3:]) <= 5)


def test_batched_shapes_are_log_uniform_in_range():
    shapes = synth.batched_shapes(3, 64)
    assert len(shapes) == 64 and shapes == synth.batched_shapes(3, 64)
    nl, npro, npo = (np.array(x) for x in zip(*shapes))
    assert nl.min() >= 8 and nl.max() <= 128
    assert npro.min() >= 500 and npro.max() <= 5000
    assert npo.min() >= 1024 and npo.max() <= 65536
    # log-uniform: the median sits near the geometric mean of the range (8192 poses,
    # about 1581 protein atoms), not near the arithmetic mean
    assert 2048 < np.median(npo) < 32768
    assert 700 < np.median(npro) < 3500


def test_he_lattice_is_seeded_and_symmetric():
    s = synth.make_he_lattice(5, 27)
    assert s["geom"].shape == (27, 3)
    np.testing.assert_array_equal(s["dens"], s["dens"].T)
    assert np.all(np.diff(s["xpnt"]) < 0)   # exponents sorted, largest first


# --- caller-supplied outputs are checked before anything is launched --------
#
# The kernels write n float32 values through each output pointer, so a short,
# mistyped, strided or host-side output (or a missing one in a batch) must be
# refused by the binding.  A stub deck on the "meta" device stands in for a
# GPU deck: every check below raises before the library is reached.

class _StubDeck:
    device = __import__("torch").device("meta")
    n_lig, n_pro, n_types, n_rows = 4, 10, 3, 2

    @property
    def handle(self):
        raise AssertionError("the library was reached")


def _meta(*shape, dtype=None):
    import torch
    return torch.empty(*shape, dtype=dtype or torch.float32, device="meta")


@pytest.mark.parametrize("bad", ["short", "long", "dtype", "strided", "cpu", "2d"])
def test_bad_out_is_refused_before_any_launch(bad):
    import torch
    deck, P = _StubDeck(), _meta(6, 8)
    out = {"short": _meta(7), "long": _meta(9), "dtype": _meta(8, dtype=torch.float64),
           "strided": _meta(16)[::2], "cpu": torch.empty(8), "2d": _meta(8, 1)}[bad]
    for call in (lambda: bude.energies(deck, P, out=out),
                 lambda: bude.energies_noalloc(deck, P, out),
                 lambda: bude.refine_device(deck, P, energies=out)):
        with pytest.raises(ValueError):
            call()


def test_batched_outputs_are_checked_per_deck():
    import torch
    decks = [_StubDeck(), _StubDeck()]
    poses = [_meta(6, 8), _meta(6, 5)]
    with pytest.raises(ValueError, match="outputs for 2 decks"):
        bude.energies_batched(decks, poses, outs=[_meta(8)])
    with pytest.raises(ValueError, match="outs\\[1\\]"):
        bude.energies_batched(decks, poses, outs=[_meta(8), _meta(8)])
    with pytest.raises(ValueError, match="outs\\[0\\]"):
        bude.energies_batched(decks, poses, outs=[torch.empty(8), _meta(5)])
    with pytest.raises(ValueError, match="outs\\[1\\]"):
        bude.energies_batched(decks, poses, outs=[_meta(8), _meta(5, dtype=torch.float16)])


def test_no_plans_are_cached_before_any_call():
    assert bude.debug_cached_plans() == (0, 0)


def test_stream_stencil_and_fock_refuse_bad_tensors_before_any_launch():
    # host tensors reach a kernel as host pointers; missing arrays as nulls
    import torch
    x = torch.zeros(64)
    with pytest.raises(ValueError, match="CUDA"):
        bude.stream_op("copy", a=x, c=x.clone())
    with pytest.raises(ValueError, match="needs the arrays a, b"):
        bude.stream_op("dot", a=x)
    with pytest.raises(ValueError, match="needs the arrays b, c"):
        bude.stream_op("mul", c=x)
    with pytest.raises(ValueError, match="CUDA"):
        bude.laplacian(torch.zeros(4, 4, 4), torch.zeros(4, 4, 4))
    hf = bude.HartreeFock.__new__(bude.HartreeFock)
    hf.n, hf.device, hf._h = 4, torch.device("cuda", 0), None
    with pytest.raises(ValueError, match="dens on cpu"):
        hf.fock(torch.zeros(4, 4, dtype=torch.float64))
    hf.device = torch.device("meta")
    with pytest.raises(ValueError, match="dens must be"):
        hf.fock(torch.zeros(4, 5, dtype=torch.float64, device="meta"))
    with pytest.raises(ValueError, match="out must be"):
        hf.fock(torch.zeros(4, 4, dtype=torch.float64, device="meta"),
                out=torch.zeros(4, 4, device="meta"))
    with pytest.raises(ValueError, match="a CUDA device"):
        bude._cuda_device("cpu")
    assert bude._cuda_device("cuda:1") == torch.device("cuda", 1)


def test_bench_summary_is_compact_and_last(bench):
    """The bench line ends with a rounded summary short enough that a reader
    keeping only the last 1500 characters of the line still sees all of it."""
    import json
    row = {"poses_per_s": 1.2345678e7, "frac_fp32_peak": 0.86912345, "scaled_err_max": 1.5e-6}
    line = {"value": 13636442.36, "ms_per_step": 4.806123, "e2e": {"value": 1.353e7},
            "config": {"variant": "fast"},
            "roofline": {"frac": 0.8687, "executed_frac": 0.61523},
            "variants": {v: dict(row) for v in ("ieee", "fast", "comp", "fp64")},
            "batched": {"batched_ms": 24.58, "plain_ms": 27.6, "speedup": 1.1229,
                        "batched_eq3_frac_fp32_peak": 0.8351, "plain_tuned_decks": 63,
                        "scaled_err_max_batched": 1.234e-6, "scaled_err_max_plain": 2.2e-6},
            "adjoint": {"ms": 2.19, "executed": {"frac_fp32_peak": 0.5851}},
            "refine": {"ms": 24.1}, "param_grad": {"ms": 2.26},
            "cull": {"ms": 2.91, "bit_identical_to_unculled": True},
            "cpu_baseline": {"value": 19125.7}}
    line["summary"] = bench.summary(line)
    text = json.dumps(line)
    tail = text[-1500:]
    assert json.dumps(line["summary"]) in tail
    assert line["summary"]["batched"]["speedup"] == 1.123
    assert line["summary"]["headline"]["eq3_frac"] == 0.8687


# --- the persistent kernel's work split (computed on the host by the same
# functions the kernel uses, through bude_debug_partition) -------------------

def _check_partition(K, nt, w, grid, with_owner=True):
    g, begin, owner, cover = bude.debug_partition(K, nt, w, grid, with_owner)
    N = int(sum(int(k) * int(t) for k, t in zip(K, nt)))
    assert 1 <= g <= grid and g <= N
    # the CTAs' ranges tile the flat space in order, and none is empty
    assert begin[0] == 0 and begin[-1] == N
    assert np.all(np.diff(begin) >= 1)
    # each tile expects exactly the CTAs whose ranges meet it (ranges are
    # contiguous and non-empty, so those are the owners of its first and last
    # unit and every CTA between them)
    starts = np.cumsum([0] + [int(k) * int(t) for k, t in zip(K, nt)])
    t_global = 0
    for (k, t), s0 in zip(zip(K, nt), starts):
        for j in range(int(t)):
            k0, k1 = s0 + j * int(k), s0 + (j + 1) * int(k)
            first = np.searchsorted(begin, k0, side="right") - 1
            last = np.searchsorted(begin, k1 - 1, side="right") - 1
            assert cover[t_global] == last - first + 1
            t_global += 1
    if owner is not None:
        # every unit's owner is the CTA whose range holds it
        np.testing.assert_array_equal(owner, np.repeat(np.arange(g), np.diff(begin)))
        # partial slots (CTA + tile) of split tiles are unique and in range
        slots = set()
        t_global = 0
        for (k, t), s0 in zip(zip(K, nt), starts):
            for j in range(int(t)):
                cov = np.unique(owner[s0 + j * int(k):s0 + (j + 1) * int(k)])
                if len(cov) > 1:
                    for c in cov:
                        sl = int(c) + t_global
                        assert sl < g + len(cover) and sl not in slots
                        slots.add(sl)
                t_global += 1
    return g


def test_work_split_random_launches():
    rng = np.random.default_rng(21)
    for trial in range(600):
        n = int(rng.integers(1, 7))
        K = rng.integers(1, 60, n)
        nt = rng.integers(1, 6, n)
        w = rng.integers(50, 170, n)
        _check_partition(K, nt, w, int(rng.integers(1, 80)))


def test_work_split_where_a_unit_outweighs_a_cta_share():
    """Few units, one dearer than a CTA's share of the total: the grid shrinks
    until every CTA's range holds a unit (a CTA without units inside a tile
    would be counted among the tile's arrivals and never arrive, leaving the
    tile unwritten)."""
    for K, nt, w, grid in (([5, 20], [1, 1], [140, 158], 29), ([1, 3], [2, 6], [124, 70], 27),
                           ([5, 20], [1, 1], [100, 120], 152)):
        g = _check_partition(K, nt, w, grid)
        assert g < min(grid, sum(k * t for k, t in zip(K, nt)))


def test_work_split_of_the_batched_workload():
    """The 64-deck batch on one CTA per SM of a GB300: all 152 CTAs, every
    range non-empty, every tile's expected arrivals equal to the CTAs that
    meet it."""
    shapes = synth.batched_shapes(3, 64)
    K = [nl * npro for nl, npro, _ in shapes]
    nt = [-(-n // 512) for _, _, n in shapes]
    w = [100 + (17 * i) % 40 for i in range(64)]
    assert _check_partition(K, nt, w, 152, with_owner=False) == 152


def test_reference_arm_line_and_other_ranks(tmp_path):
    # the reference arm times the oracle on the host: one JSON line on rank 0
    # with the keys the bench contract names; any other rank prints nothing
    import json
    import subprocess
    import sys
    env = dict(os.environ, RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                         env=env, cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "poses/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["higher_is_better"] is True
    assert line["config"]["workload"].startswith("deck 64 lig x 2672 pro x 65536 poses")
    env["RANK"] = "1"
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                         env=env, cwd=ROOT, timeout=600)
    assert out.returncode == 0 and out.stdout.strip() == ""
