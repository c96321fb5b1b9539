"""The reference arm of bench.py (the FP64 oracle on the host cores): its JSON line, and
its launch under torchrun, where rank 0 alone runs and prints and the other ranks exit 0
without work.  CPU only."""
import json
import os
import socket
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(cmd, env_extra):
    env = dict(os.environ, OMP_NUM_THREADS="2", **env_extra)
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def _check_line(line, n_gpus):
    d = json.loads(line)
    assert d["impl"] == "reference" and d["n_gpus"] == n_gpus
    assert d["unit"] == "MLUPS" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "sample" in d["cpu_baseline"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_reference_arm_line_and_non_zero_ranks():
    args = [sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"]
    r0 = _run(args, {"RANK": "0", "WORLD_SIZE": "1"})
    assert r0.returncode == 0, r0.stderr[-2000:]
    lines = [ln for ln in r0.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    _check_line(lines[0], 1)
    r1 = _run(args, {"RANK": "1", "WORLD_SIZE": "2"})
    assert r1.returncode == 0 and not r1.stdout.strip()


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "2", "--warmup", "3"]
    r = _run(cmd, {})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    _check_line(lines[0], 2)


def test_traffic_record_matches_the_kernel_sources():
    """The DRAM-traffic record the bench line quotes (profiles/traffic.json) was captured on
    the kernel sources as they are, and covers the kernels the bench times at 512^3 in
    every storage mode it reports."""
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    assert rec["kernel_sources_sha256"] == bench.kernel_sources_sha()
    for prec in ("f32", "f16", "bf16"):
        for kern, algo in (("k_lb_rows", bench.kernel_bytes("lb", prec)), ("k_fv_pair", bench.kernel_bytes("fv", prec))):
            r = rec["kernels"][f"{kern}:{prec}"]
            # measured DRAM bytes at least the algorithmic bytes, and no large re-read
            assert algo <= r["bytes_per_cell"] <= 1.1 * algo, (kern, prec, r["bytes_per_cell"], algo)
            assert bench.load_traffic(prec, kern, "auto") == r["dram_bytes_per_launch_full_size"]
