"""Host checks of the benchmark's reporting: the roofline entry's arithmetic,
the lookup of ncu DRAM traffic (used only while the kernel sources still
hash to the profiled ones), and the commands the ncu summaries under
profiles/ give (each names committed files and flags that bench.py still
accepts); also the host-only checkpoint-sharing block."""
import json
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PROFILES = os.path.join(ROOT, "profiles")


def test_roofline_pair_reports_the_binding_roof():
    # 3000 GB/s of 6000 (0.5) against 10 of 40 T ops/s (0.25): HBM binds
    r = bench.roofline_pair(3000.0, 6000.0, "measured", 10e12 * 2e-3, 2.0, "c128df", 1.5e9, 4, "32 B")
    assert r["bound"] == "hbm" and r["frac"] == pytest.approx(0.5)
    assert r["other_roof"]["bound"] == "alu"
    assert r["other_roof"]["frac"] == pytest.approx(10.0 / bench.FP32_PEAK_TOPS)
    assert r["traffic"] == 1.5e9 and r["kernel_launches"] == 4
    # the other way round: 30 T ops/s in 1 ms binds against 1000 GB/s
    r = bench.roofline_pair(1000.0, 6000.0, "measured", 30e12 * 1e-3, 1.0, "c64", None, 1, "16 B")
    assert r["bound"] == "alu" and r["frac"] == pytest.approx(30.0 / bench.FP32_PEAK_TOPS)
    assert r["other_roof"]["frac"] == pytest.approx(1000.0 / 6000.0)
    assert r["traffic"] is None


def test_alu_peak_is_unit_counts_times_clock():
    assert bench.FP32_PEAK_TOPS == pytest.approx(152 * 128 * 2.07e9 / 1e12)


@pytest.mark.parametrize("name", ["k_pass_df_traffic.json", "k_pass_c64_traffic.json"])
def test_traffic_is_used_only_for_the_profiled_kernel_source(name):
    with open(os.path.join(PROFILES, name)) as f:
        d = json.load(f)
    # the summary it was taken from is committed beside it
    assert os.path.exists(os.path.join(PROFILES, d["source"]))
    # a DRAM figure per amplitude-pass near the algorithmic read + write
    per_amp = 32.0 if "df" in name else 16.0
    assert 0.5 * per_amp < d["dram_bytes_per_amp_pass"] <= 1.2 * per_amp
    assert bench.profiled_traffic("0" * 16, name) is None
    got = bench.profiled_traffic(d["kernel_source_hash"], name)
    assert got is not None and got["dram_bytes_per_amp_pass"] == d["dram_bytes_per_amp_pass"]


def _bench_flags():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True,
                         text=True, check=True, cwd=ROOT).stdout
    return set(re.findall(r"(--[a-z0-9][a-z0-9-]*)", out))


def test_profile_commands_run_committed_files_with_current_flags():
    flags = _bench_flags()
    seen = 0
    for fn in sorted(os.listdir(PROFILES)):
        if not fn.endswith(".md"):
            continue
        text = open(os.path.join(PROFILES, fn)).read()
        cmds = [ln.strip() for ln in text.splitlines() if ln.strip().startswith("ncu ")]
        assert cmds, f"{fn} gives no command"
        for cmd in cmds:
            assert "--clock-control none" in cmd, fn
            assert "_work" not in cmd and "/root/" not in cmd, fn
            prog = cmd.split(" python ", 1)[1]
            assert prog.startswith("bench.py"), fn
            for flag in re.findall(r"\s(--[a-z0-9-]+)", " " + prog):
                assert flag in flags, (fn, flag)
            seen += 1
    assert seen >= 4


def test_checkpoint_sharing_block_runs_on_the_host():
    """configs.checkpoint_sharing plans dry runs only (no GPU): the shared
    fraction of each spacing is a fraction, and small on these circuits
    (every uncontrolled gate touches every partition)."""
    from paper_2210_01076_gb300 import binding as B
    from paper_2210_01076_gb300 import build as qbuild
    from paper_2210_01076_gb300 import workloads as W
    qbuild.build()
    B.load()
    levels, _, _, _ = bench.make_workload(bench.rank_seed(0), 2)
    out = bench.sharing_block(B, W, levels)
    for key in ("incremental_n24", "qft_like_n30"):
        rows = out[key]
        assert [r["levels_per_checkpoint"] for r in rows][0] == 1
        for r in rows:
            assert r["segments"] >= 1
            assert 0.0 <= r["unchanged_partition_fraction"] <= 0.05
        # one level per checkpoint shares at least as much as longer segments
        assert rows[0]["unchanged_partition_fraction"] >= rows[-1]["unchanged_partition_fraction"]
