"""Host-side checks of the benchmark's measurement bookkeeping.

The roofline's DRAM traffic comes from a committed ncu capture and may only be
reported while the kernel that was captured is the kernel that runs: the same
sources and the same launch configuration. These tests pin that guard on a
scratch copy of the bookkeeping, and that the committed record names the
sources and launch fields the benchmark checks.
"""
import json
import os

import pytest

import bench
from paper_2501_18977_gb300.binding import blowchoc_tuning


def _scratch_root(tmp_path, text="kernel v1"):
    csrc = tmp_path / "paper_2501_18977_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text(text)
    (tmp_path / "profiles").mkdir()
    return csrc


def _tuning(**kw):
    t = blowchoc_tuning()
    for k, v in dict(lanes_choose=2, ctas_per_sm=8, keys_per_cta=128, persistent=1, set_mode=0,
                     lanes_query=1, query_early=1).items():
        setattr(t, k, kw.get(k, v))
    return t


@pytest.fixture
def scratch(tmp_path, monkeypatch):
    csrc = _scratch_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.KERNEL_SOURCES, "persistent_insert_kernel", ["k.cu"])
    record = {"kernels": {"persistent_insert_kernel": {
        "dram_bytes_per_launch": 123456789,
        "launch": bench.launch_config(_tuning(), "persistent_insert_kernel"),
        "sources": ["k.cu"],
        "sources_sha256": bench.sources_sha256(["k.cu"]),
    }}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(record))
    return csrc


def test_traffic_reported_for_the_captured_kernel(scratch):
    assert bench.ncu_traffic("persistent_insert_kernel", _tuning()) == 123456789


def test_traffic_dropped_when_a_source_changes(scratch):
    (scratch / "k.cu").write_text("kernel v2")
    assert bench.ncu_traffic("persistent_insert_kernel", _tuning()) is None


@pytest.mark.parametrize("field,value", [("lanes_choose", 4), ("keys_per_cta", 64), ("set_mode", 1),
                                         ("persistent", 0), ("ctas_per_sm", 4)])
def test_traffic_dropped_when_the_launch_differs(scratch, field, value):
    assert bench.ncu_traffic("persistent_insert_kernel", _tuning(**{field: value})) is None


def test_traffic_absent_for_an_uncaptured_kernel(scratch):
    assert bench.ncu_traffic("query_kernel", _tuning()) is None


def test_committed_record_matches_the_guard():
    path = os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.json")
    with open(path) as fh:
        kernels = json.load(fh)["kernels"]
    for name, entry in kernels.items():
        assert entry["sources"] == bench.KERNEL_SOURCES[name]
        assert sorted(entry["launch"]) == sorted(bench.KERNEL_LAUNCH_FIELDS[name])
        assert entry["dram_bytes_per_launch"] > 0
        for field in entry["launch"]:
            assert hasattr(blowchoc_tuning(), field)


def test_bench_lines_are_strict_json():
    """A measurement that was not taken (a gather ceiling skipped by
    --no-extra-records) is printed as null, never as NaN or Infinity."""
    import json
    import bench
    rec = {"frac_of_gather_ceiling": bench.ratio(3519.4, None),
           "gather_ceiling_gbs": {"filter_footprint_128MiB": bench.rounded(None, 1), "hbm_4GiB": float("nan")},
           "list": [1.5, float("inf"), -float("inf")], "ok": 0.52}
    text = json.dumps(bench.finite(rec), allow_nan=False)
    back = json.loads(text)
    assert back["frac_of_gather_ceiling"] is None
    assert back["gather_ceiling_gbs"] == {"filter_footprint_128MiB": None, "hbm_4GiB": None}
    assert back["list"] == [1.5, None, None] and back["ok"] == 0.52
    assert bench.ratio(3519.4, 8300.0) == round(3519.4 / 8300.0, 4)


def test_clock_record_is_the_median_under_load():
    """The clock record's sm_mhz is the median over samples with the GPU busy
    (utilization >= 50%); idle samples at idle clocks do not pull it down.
    Throttle reasons are collected from every sample."""
    import bench

    class Done:  # a finished sampler process
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c = bench.ClockSampler(0)
    with open(c.path, "w") as fh:
        fh.write("0, 120, 2070, 150.1, 0x0, Not Active, Not Active, Not Active, Not Active, 0\n" * 5)
        fh.write("0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Active, 97\n" * 3)
        fh.write("garbage line\n")
    c.proc, c.fh = Done(), open(os.devnull, "w")
    rec = c.stop()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_mhz_all_samples"] == 120.0
    assert (rec["samples"], rec["samples_busy"]) == (8, 3)
    assert rec["reasons"] == ["sw_power_cap"] and rec["sm_max_mhz"] == 2070.0
    assert rec["sm_mhz_basis"] == "median of busy samples"
    # no busy sample at all: the highest clock seen, and the record says so
    c = bench.ClockSampler(0)
    with open(c.path, "w") as fh:
        fh.write("0, 120, 2070, 150.1, 0x0, Not Active, Not Active, Not Active, Not Active, 0\n" * 4)
        fh.write("0, 1980, 2070, 400.0, 0x0, Not Active, Not Active, Not Active, Not Active, 12\n")
    c.proc, c.fh = Done(), open(os.devnull, "w")
    rec = c.stop()
    assert rec["sm_mhz"] == 1980.0 and rec["samples_busy"] == 0
    assert rec["sm_mhz_basis"] == "highest sample (no busy sample)"


def _run_bench(args, env_extra=None, timeout=300):
    import subprocess
    import sys
    env = dict(os.environ)
    env.update(env_extra or {})
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    return subprocess.run([sys.executable, os.path.join(root, "bench.py")] + args, cwd=root, env=env,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_strict_json_line():
    """The reference arm (the oracle on the host, a bounded sample per step)
    prints exactly one JSON line with the benchmark's metric and unit, its
    own cpu_baseline and e2e blocks, and no NaN."""
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0], parse_constant=lambda c: (_ for _ in ()).throw(ValueError(c)))
    assert d["impl"] == "reference" and d["unit"] == "Mkeys/s" and d["higher_is_better"] is True
    assert d["metric"] == "insert+query throughput (DNA 31-mers, c=3, k=16, cost^LA)"
    assert d["steps"] == 1 and d["warmup"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] == 1
    assert d["e2e"] == {"value": d["value"], "unit": "Mkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "dna_kmer_31_c3_la"


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the reference arm; another rank exits
    0 at once and prints nothing."""
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "1", "--gpus", "2"],
                   env_extra={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]
