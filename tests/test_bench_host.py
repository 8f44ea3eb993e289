"""Host logic of bench.py (no GPU): the reference arm's JSON line, the
comment-insensitive source hashes that decide whether a committed ncu
traffic figure still describes a kernel, the traffic table itself, and the
roofline and replica arithmetic."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_line():
    """`bench.py --impl reference` times the oracle on the headline workload
    and prints one JSON line in the contract's shape."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "MLUPS" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "ST D2Q9 8192x8192" in line["config"]["workload"]


def test_source_hash_ignores_comments(tmp_path, monkeypatch):
    src = tmp_path / "paper_1505_03271_gb300" / "csrc"
    src.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (src / "k.cu").write_text("int f(int a) { return a + 1; }  // one\n")
    h0 = bench.source_hash(["k.cu"])
    (src / "k.cu").write_text("/* a block\n comment */\nint f(int a) {\n    return a + 1;   // two\n}\n")
    assert bench.source_hash(["k.cu"]) == h0
    (src / "k.cu").write_text("int f(int a) { return a + 2; }\n")
    assert bench.source_hash(["k.cu"]) != h0


def test_traffic_table_well_formed():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        table = json.load(fh)
    entries = {k: v for k, v in table.items() if not k.startswith("_")}
    assert entries
    for key, e in entries.items():
        schedule, case = key.split("|")
        assert schedule and case
        assert isinstance(e["bytes"], int) and e["bytes"] > 0
        assert len(e["sources"]) == 16 and e["files"]
        for f in e["files"]:
            assert os.path.exists(os.path.join(ROOT, "paper_1505_03271_gb300", "csrc", f)), f
        assert os.path.exists(os.path.join(ROOT, e["profile"])), e["profile"]
        # the lookup returns the bytes exactly when the kernel's code is unchanged
        expect = e["bytes"] if bench.source_hash(e["files"]) == e["sources"] else None
        assert bench.measured_traffic(schedule, case) == expect
    assert bench.measured_traffic("no such schedule", "channel") is None


def test_roofline_arithmetic():
    r = bench.roofline(72 * 131072, 0.0144, 6680.2, "measured", traffic=4805120)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] == 4805120
    assert r["achieved"] == pytest.approx(72 * 131072 / 14.4e-6 / 1e9, abs=0.05)
    assert r["frac"] == pytest.approx(r["achieved"] / 6680.2, abs=1e-4)


def test_single_rank_aggregate():
    t, mlups = bench.aggregate(0.5, 131072, 1000, 1)
    assert t == 0.5 and mlups == pytest.approx(131072 * 1000 / 0.5 / 1e6)


def test_reference_arm_other_ranks_do_no_work():
    """Under torchrun only rank 0 times the oracle; the other ranks exit 0
    without output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_oracle_sample_threads_and_cpu_model():
    """The CPU legs of the bench: a bounded oracle sample on the requested
    thread count, and the host's CPU model for the JSON line."""
    from paper_1505_03271_gb300 import configs as cfg
    w = cfg.channel(nx=16, ny=32)
    r, done, el, thr = bench.oracle_sample(w, budget_s=0.05, threads=1)
    assert thr == 1 and done >= 1 and el > 0
    _, ux, _, _ = r.moments()
    assert ux.shape == (32, 16) and np.isfinite(ux).all()
    model = bench.cpu_model()
    assert isinstance(model, str) and model


def test_st_schedule_names_follow_the_dispatch():
    """The bench names an ST line by the kernel the library dispatches
    (lb_step_st: the four-cell kernels on x-periodic flow grids with nx a
    multiple of 4, FP32 or 16-bit; the pair kernels elsewhere), and the
    committed traffic entries of the ST lines carry those names."""
    import types
    import paper_1505_03271_gb300 as lb

    def grid(store, nx, bcx=lb.LB_BC_PERIODIC, thermal=False):
        return types.SimpleNamespace(store=store, nx=nx, thermal=thermal, desc=types.SimpleNamespace(bcx=bcx))

    quad32 = "st quad (128-bit words, f32x2), four cells per thread"
    quad16 = "st quad (64-bit words, f32x2), four cells of two rows per thread"
    assert bench.schedule_name(lb, grid(lb.LB_STORE_F32, 8192), "st") == quad32
    assert bench.schedule_name(lb, grid(lb.LB_STORE_F32, 8190), "st") == "st pair (f32x2), two cells per thread"
    assert bench.schedule_name(lb, grid(lb.LB_STORE_F32, 8192, bcx=lb.LB_BC_WALLS), "st") != quad32
    assert bench.schedule_name(lb, grid(lb.LB_STORE_F32, 8192, thermal=True), "st") != quad32
    for store in (lb.LB_STORE_F16DEV, lb.LB_STORE_BF16DEV):
        assert bench.schedule_name(lb, grid(store, 8192), "st") == quad16
        assert bench.schedule_name(lb, grid(store, 8190), "st") == "st pair (f32x2), two cells of two rows per thread"
    assert bench.schedule_name(lb, grid(lb.LB_STORE_F64, 64), "st") == "st push, one thread per cell"
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        keys = set(json.load(fh))
    assert quad32 + "|st4096" in keys
    assert quad16 + "|st4096_f16dev" in keys and quad16 + "|st4096_bf16dev" in keys
