"""bench.py's reference arm on the CPU: the oracle timed on the host, one JSON
line with the GPU line's metric, unit, direction and workload config."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    sys.path.insert(0, ROOT)
    import bench
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "ba2000", "--steps", "2", "--warmup", "0", "--ref-step-seconds", "0.3"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is False and d["steps"] == 2 and d["warmup"] == 0
    assert d["config"]["workload"] == "ba2000: " + bench.WORKLOADS["ba2000"]
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_profile_traffic_needs_the_same_kernel_source(tmp_path, monkeypatch):
    """The roofline's `traffic` comes from a committed ncu summary only when it
    was captured on the kernel source the bench runs; otherwise it is null."""
    sys.path.insert(0, ROOT)
    import bench
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k_sparse_grid1024.md").write_text(
        "# summary\n\ntraffic_bytes_per_launch: 12345\n\nkernel_source_sha256: abcdef0123456789\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("k_sparse", "abcdef0123456789", "grid1024") == 12345.0
    assert bench.profile_traffic("k_sparse", "0000000000000000", "grid1024") is None
    assert bench.profile_traffic("k_sparse", "abcdef0123456789", "grid2048") is None
    assert bench.profile_traffic("k_wave_grid", "abcdef0123456789", "grid1024") is None


def test_committed_profiles_name_their_source_and_command():
    """Every DRAM-traffic summary the bench can read states the kernel source it
    was taken on, and every summary gives the command that made it."""
    pdir = os.path.join(ROOT, "profiles")
    for name in sorted(os.listdir(pdir)):
        text = open(os.path.join(pdir, name)).read()
        if "traffic_bytes_per_launch:" in text:
            assert "kernel_source_sha256:" in text, name
        assert "python bench.py" in text or "Same capture as" in text, name


def test_workload_names_resolve():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1507_01490_gb300 import graphgen
    assert set(bench.WORKLOADS) >= {"chunglu1m", "rmat20", "grid2048", "ba2000"}
    for name in ("ba2000", "grid256"):
        g = graphgen.workload(name)
        assert g.n > 0 and g.m > 0, name
    g = graphgen.workload("grid256")
    assert g.n == 65536 and int(g.degrees().max()) == 4   # a lattice: the one-source kernel's default case
