"""bench.py's contract on the CPU: the reference arm (the FP64 oracle) in one process and as two
torchrun ranks over gloo (rank 0 alone runs and prints one JSON line; the other rank exits 0)."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"}


def _json_lines(text):
    return [json.loads(x) for x in text.splitlines() if x.startswith("{")]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_single_process():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", "ni147", "--steps", "3",
                          "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = _json_lines(out.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert KEYS <= set(d)
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 3 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_two_ranks_gloo():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference", "--gpus", "2",
           "--config", "ni147", "--steps", "3", "--warmup", "3"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = _json_lines(out.stdout)
    assert len(lines) == 1  # rank 0 only
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2


def test_replica_workloads_per_rank_share_the_shape_and_differ_in_seeds():
    """Under torchrun each rank runs an independent replica: the same clusters and sizes (so the work per GPU
    is fixed as N grows, weak scaling), with velocities and Langevin noise from rank-specific seeds."""
    import numpy as np
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    for name in ("ni2000", "ni147", "ni147x64"):
        w0, w1 = bench.workload(name, 0), bench.workload(name, 1)
        assert w0["sizes"] == w1["sizes"] and w0["prec"] == w1["prec"] and w0["dt"] == w1["dt"]
        assert np.array_equal(w0["pos"], w1["pos"]) and np.array_equal(w0["mass"], w1["mass"])
        assert w0["seed"] != w1["seed"]
        assert not np.allclose(w0["vel"], w1["vel"])
