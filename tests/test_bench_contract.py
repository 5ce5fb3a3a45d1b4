"""Host-side parts of the benchmark on CPU.  The reference arm
(`bench.py --impl reference`) times the FP64 oracle on a bounded crop of the
workload and prints one JSON line with the keys of the device arm plus impl,
cpu_baseline and a zero-copy e2e; a rank other than 0 prints nothing and
exits 0.  The device arm's cpu_baseline also carries a single-thread oracle
timing (a child process with OMP_NUM_THREADS=1) and the host CPU's name."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ, **(extra_env or {}))
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "crop64",
           "--steps", "1", "--warmup", "3"]
    return subprocess.run(cmd, capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)


def test_reference_arm_line():
    r = _run()
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3 and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_do_no_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_single_thread_oracle_timing_and_cpu_name(tmp_path):
    b = _bench()
    d = b.oracle_single_thread()
    assert d["cores"] == 1 and d["value"] > 0 and d["unit"] == "MLUPS" and "16x16x32" in d["sample"]
    arm = tmp_path / "cpuinfo"
    arm.write_text("processor\t: 0\nBogoMIPS\t: 2000.00\nCPU implementer\t: 0x41\nCPU part\t: 0xd4f\n")
    assert b.cpu_model(str(arm)).endswith("implementer 0x41, part 0xd4f")
    x86 = tmp_path / "cpuinfo_x86"
    x86.write_text("processor\t: 0\nmodel name\t: Some CPU @ 2.0GHz\n")
    assert b.cpu_model(str(x86)) == "Some CPU @ 2.0GHz"


def test_d2q9_oracle_sample():
    b = _bench()
    v, secs, n, cores = b.oracle2d_sample(n=(64, 16), steps=3)
    assert v > 0 and secs > 0 and n == (64, 16) and cores >= 1
    ch, tau, F = b.d2q9_channel((4096, 1024))
    assert tau == 0.8 and abs(F - 8.0 * 0.1 * 0.05 / 1023 ** 2) < 1e-18 and ch.J4.shape == (4, 4096 * 1024)


def test_side_report_oracle_samples():
    """The oracle timings that sit beside the lattice-gradient and
    chart-change reports of the device line (run here on the profiling
    workload's half-size crop)."""
    b = _bench()
    g, t = b.oracle_side_samples(b.workload_spec("crop64"))
    assert g["kind"] == "oracle" and g["value"] > 0 and g["unit"] == "GFLOP/s (FP64)" and "32x64x32" in g["sample"]
    assert g["mnode_per_s"] > 0
    assert t["kind"] == "oracle" and t["node_wise_ms"] > 0 and t["interp_ms"] > 0 and t["nodes"] == 32 * 64 * 32


def test_batch_oracle_sample():
    from paper_1803_07822_gb300 import inputs as I
    b = _bench()
    ws = I.batch_channels(nb=4, seed0=4100, side=(8, 12), kmax=1, lmax=1)
    d = b.oracle_batch_sample(ws, count=2, steps=2)
    assert d["kind"] == "oracle" and d["value"] > 0 and "2 smallest channels" in d["sample"]
