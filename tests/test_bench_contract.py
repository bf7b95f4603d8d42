"""The benchmark's command-line contract on CPU: the reference arm (the FP64 oracle on the
host cores) prints one JSON line with the keys and units of the device arm, alone or under
torchrun, and the warm-up floor is enforced."""
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, timeout=300):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_complete_line():
    res = _bench("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["unit"] == "snapshot updates/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["vs_baseline"] is None and d["scaling"] == "weak" and d["data"] == "synthetic"
    assert "n=393216" in d["config"]["workload"] and d["config"]["r_max"] == 40
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_warmup_below_three_is_refused():
    res = _bench("--impl", "reference", "--steps", "1", "--warmup", "2", timeout=120)
    assert res.returncode != 0
    assert "warmup" in res.stderr


def test_reference_arm_under_torchrun_prints_once():
    """Launched as the multi-rank benchmark is (torchrun, one process per rank; gloo here),
    the reference arm runs on rank 0 alone: exactly one JSON line, with n_gpus = 2, and every
    rank exits 0."""
    env = dict(os.environ, ODMD_BENCH_BACKEND="gloo", MASTER_ADDR="127.0.0.1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", "29531", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_clock_sampler_reads_median_clock_and_throttle_reasons(tmp_path, monkeypatch):
    """The clocks object of the JSON line: median SM clock under load, the maximum, and every
    throttle reason seen active (the names the rejection rule checks), over the samples taken
    while the timed regions run.  A stand-in nvidia-smi prints a sample every 20 ms from a
    state file; throttled samples printed while the sampler is paused are not counted."""
    sys.path.insert(0, ROOT)
    import bench

    state = tmp_path / "state"
    state.write_text("good")
    fake = tmp_path / "nvidia-smi"
    fake.write_text(
        "#!" + sys.executable + "\n"
        "import sys, time\n"
        "k = 0\n"
        "while True:\n"
        f"    s = open({str(state)!r}).read().strip()\n"
        "    if s == 'bad':\n"
        "        print('0, 1500, 2070, 1400.0, 0x8, Active, Not Active, Not Active, Not Active', flush=True)\n"
        "    elif k % 3 == 1:\n"
        "        print('0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active', flush=True)\n"
        "    else:\n"
        "        print('0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active', flush=True)\n"
        "    print('garbled line', flush=True)\n"
        "    k += 1\n"
        "    time.sleep(0.02)\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])

    s = bench.ClockSampler(0)
    s.start()
    assert s.rows, "start() returns once the first sample is in"
    time.sleep(0.4)
    s.pause()
    state.write_text("bad")
    time.sleep(0.3)
    state.write_text("good")
    time.sleep(0.2)
    s.resume()
    time.sleep(0.4)
    c = s.stop()
    assert c["samples"] >= 10
    assert c["sm_mhz"] in (1980.0, 2025.0, 2070.0) and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    assert any(len(f) > 1 and f[1] == "1500" for _, f in s.rows), "throttled samples were printed while paused"
    assert 0.7 < c["timed_s"] < 1.5


def test_oracle_child_times_whole_blocks_with_the_thread_count_set():
    """The CPU legs time the oracle in a child process whose BLAS thread count is set through
    the environment (one thread here), on whole blocks of the workload, and report the BLAS
    library with the threads it ran with."""
    sys.path.insert(0, ROOT)
    import bench

    d = bench.oracle_child(1, 1)
    assert d["blocks"] == 1 and d["rank"] == 40
    assert d["threads"] == 1 and d["blas"] and d["blas"] != "unknown"
    assert d["updates_per_s"] > 0 and d["states_per_s"] > 0 and d["step_s"] > 0
