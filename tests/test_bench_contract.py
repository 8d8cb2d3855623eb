"""bench.py's JSON contract on CPU: the reference arm (the oracle timed on the
host cores) prints one line with the keys the driver reads, and the
argument parser accepts the documented flags. No GPU is needed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(*args, env=None, timeout=600):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, OMP_NUM_THREADS="1")  # as a launcher sets it: the arm must still use all cores
    # a small workload keeps the CPU suite short; the default is R-MAT scale 26
    r = run("--impl", "reference", "--workload", "rmat16", "--steps", "1", "--warmup", "3", env=env)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == "triangle-count TEPS" and d["unit"] == "edges/s"
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "rmat-s16-ef16-seed1"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] == (
        len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_warmup_below_three_is_refused():
    r = run("--warmup", "2", timeout=120)
    assert r.returncode != 0 and "warmup" in (r.stderr + r.stdout)


def test_documented_flags_parse():
    r = run("--help", timeout=120)
    assert r.returncode == 0
    for flag in ("--gpus", "--steps", "--warmup", "--impl", "--workload", "--batched", "--serve-seconds",
                 "--reorder", "--ablation", "--reorder-profile", "--profile-hash-mode", "--no-cpu-baseline",
                 "--second", "--e2e-steps"):
        assert flag in r.stdout, flag


def test_default_workload_is_rmat26_with_int64_offsets():
    sys.path.insert(0, ROOT)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    w = b.WORKLOADS[b.DEFAULT_WORKLOAD]
    assert w["name"] == "rmat-s26-ef16-seed3" and w["offset_bits"] == 64
    golden = json.load(open(os.path.join(ROOT, "tests", "golden", w["golden"])))
    assert golden["workload"] == w["name"] and golden["triangles"] > 2 ** 32


def test_host_reservations_cover_the_workloads():
    # the end-to-end host buffers are mapped before the graph exists, from each
    # workload's bounds on n and nnz: the generated graphs must fit them
    sys.path.insert(0, ROOT)
    import bench
    import graphgen as G
    for key in ("rmat16", "rmat22", "rgg22"):
        spec = bench.WORKLOADS[key]
        g = G.workload(spec["graph"])
        assert g.n == spec["n"], key
        assert g.nnz <= spec["nnz_max"], key
    spec = bench.WORKLOADS["rmat26"]  # 2 * edge factor * 2^scale entries at most
    assert spec["n"] == 1 << 26 and spec["nnz_max"] >= 2 * 16 * (1 << 26)
    # a reservation is whole 2 MiB pages of touched anonymous memory
    ptr, nbytes = bench.HugePinned.reserve(3 << 20)
    try:
        assert nbytes == 4 << 20 and ptr
    finally:
        bench.HugePinned._c().munmap(ptr, nbytes)
