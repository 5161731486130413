"""Host logic of bench.py (CPU): the algorithmic-bytes formula of the roofline, the rule that ties
ncu traffic to the kernel sources it was measured on, and the bench line's argument handling."""
from __future__ import annotations

import os

import bench


def _stats(reached, examined, live, samples):
    z = [0, 0, 0, 0]
    st = {"tier_reached": list(z), "tier_examined_edges": list(z), "tier_live_edges": list(z),
          "tier_samples": list(z)}
    st["tier_reached"][3], st["tier_examined_edges"][3] = reached, examined
    st["tier_live_edges"][3], st["tier_samples"][3] = live, samples
    return st


def test_algorithmic_bytes_formula():
    # 10 samples, 3 seeds each: 8|R| + 8 E_R + 8 |R \ S|; with targets of live edges only:
    # 8|R| + 4 E_R + 4 L + 8 |R \ S|
    st = _stats(reached=500, examined=7000, live=420, samples=10)
    assert bench.algorithmic_bytes(st, 3, 3) == 8 * 500 + 8 * 7000 + 8 * (500 - 30)
    assert bench.algorithmic_bytes_live_targets(st, 3, 3) == 8 * 500 + 4 * 7000 + 4 * 420 + 8 * (500 - 30)
    assert bench.algorithmic_bytes(_stats(0, 0, 0, 0), 3, 50) == 0


def test_roofline_names_its_bound():
    """HBM when the kernel's DRAM traffic is of the order of its algorithmic bytes; instruction
    issue when the graph is served from L2 (traffic far below them)."""
    prof = {k: {"launches": 0, "ms": 0.0} for k in ("sample_tier0", "sample_tier1", "sample_tier2",
                                                     "sample_cta", "select", "other")}
    prof["sample_cta"] = {"launches": 2, "ms": 4.0}
    st = _stats(reached=1000, examined=100000, live=900, samples=10)
    r = bench.roofline_of(prof, st, 3, workload="no-such-workload")
    assert r["kernel"] == "k_sample_cta" and r["bound"] == "hbm" and r["traffic"] is None
    alg = (8 * 1000 + 8 * 100000 + 8 * (1000 - 30)) / 2
    assert abs(r["achieved"] - alg / 2e-3 / 1e9) < 1e-9 and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12


def test_traffic_only_for_the_sources_it_was_measured_on(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    csrc = tmp_path / "paper_2302_13529_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        (csrc / f).write_text(f"// {f} v1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash()
    path = prof / f"k_sample_cta_{bench.WORKLOAD}.md"
    path.write_text(f"# x\nsource_hash: {h}\ndram_bytes_per_launch: 1234\n")
    assert bench.ncu_traffic("k_sample_cta") == 1234.0
    (csrc / bench.KERNEL_SOURCES[0]).write_text("// changed\n")  # the kernel changed since
    assert bench.kernel_source_hash() != h
    assert bench.ncu_traffic("k_sample_cta") is None
    assert bench.ncu_traffic("k_other") is None  # no summary at all


def test_ncu_figures_follow_the_source_hash(tmp_path, monkeypatch):
    """The summary's other header figures reach roofline.ncu, and the bound turns to "issue",
    only while the summary was taken on the current kernel sources."""
    prof_dir = tmp_path / "profiles"
    prof_dir.mkdir()
    csrc = tmp_path / "paper_2302_13529_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        (csrc / f).write_text(f"// {f} v1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash()
    (prof_dir / f"k_sample_cta_{bench.WORKLOAD}.md").write_text(
        f"# x\nsource_hash: {h}\ndram_bytes_per_launch: 100\nissue_active_pct: 58.5\n"
        "l2_hit_rate_pct: 87.6\n")
    prof = {k: {"launches": 0, "ms": 0.0} for k in ("sample_tier0", "sample_tier1", "sample_tier2",
                                                     "sample_cta", "select", "other")}
    prof["sample_cta"] = {"launches": 2, "ms": 4.0}
    st = _stats(reached=1000, examined=100000, live=900, samples=10)
    r = bench.roofline_of(prof, st, 3)
    assert r["bound"] == "issue" and r["traffic"] == 100.0
    assert r["ncu"] == {"issue_active_pct": 58.5, "l2_hit_rate_pct": 87.6}
    (csrc / bench.KERNEL_SOURCES[0]).write_text("// changed\n")
    r = bench.roofline_of(prof, st, 3)
    assert r["bound"] == "hbm" and r["traffic"] is None and "ncu" not in r


def test_committed_profiles_match_the_kernel_sources():
    """Every committed ncu summary that names a source hash was taken on the current kernel
    sources: a kernel change without a new capture would leave counters that describe other
    code (and bench.py would drop their traffic figure)."""
    prof_dir = os.path.join(bench.ROOT, "profiles")
    current = bench.kernel_source_hash()
    checked = 0
    for name in sorted(os.listdir(prof_dir)):
        for line in open(os.path.join(prof_dir, name)):
            if line.startswith("source_hash:"):
                assert line.split(":", 1)[1].strip() == current, name
                checked += 1
    assert checked >= 3


def test_committed_profile_names_its_kernel_sources():
    """The committed block-tier summary carries a source hash and a traffic figure."""
    path = os.path.join(bench.ROOT, "profiles", f"k_sample_cta_{bench.WORKLOAD}.md")
    text = open(path).read()
    assert "source_hash:" in text and "dram_bytes_per_launch:" in text


def test_default_arguments_are_the_driver_contract():
    a = bench.parse_args([])
    assert (a.gpus, a.workload, a.impl) == (1, "rmat17", "ours")
    assert a.warmup >= 3 and a.steps >= 1
    a = bench.parse_args(["--workload", "rmat22", "--b", "2", "--theta", "500"])
    assert (a.b, a.theta) == (2, 500)


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints one JSON line with the
    metric, unit and config of the GPU arm, its CPU-baseline description and a zero-copy e2e."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1", "--ref-step-seconds", "0.2"],
                         capture_output=True, text=True, timeout=600, cwd=bench.ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "samples/s" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["config"]["workload"] == bench.WORKLOAD
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert line["e2e"] == {"value": line["value"], "unit": "samples/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
