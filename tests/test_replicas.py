"""The N > 1 path of bench.py on the CPU: world size 2 over gloo.

Every rank solves its own replica of the workload (the method exchanges nothing between
instances). The only coordination is a barrier around each timed region, the maximum of the
timed durations and rank 0 alone printing. The reference arm's other ranks exit at once,
without work. The ranks here run as separate processes rendezvousing on 127.0.0.1.
"""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import bench
rep = bench.Replicas("gloo")
rep.barrier()
seconds = 1.0 + 0.5 * rep.rank              # rank 1 is the slower one
smax = rep.max(seconds)
rate = bench.job_rate(rep.world, 10, smax)  # 10 solves per rank
print(json.dumps({"rank": rep.rank, "world": rep.world, "local": rep.local, "max": smax, "rate": rate}))
rep.close()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    env = dict(os.environ)
    env.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    return env


def test_two_ranks_share_the_slowest_time_and_report_the_job_rate():
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", RANK_SCRIPT, ROOT], env=_env(r, 2, port), cwd=ROOT,
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert [o["rank"] for o in outs] == [0, 1]
    assert all(o["world"] == 2 for o in outs)
    assert [o["local"] for o in outs] == [0, 1]
    assert all(o["max"] == 1.5 for o in outs)                       # every rank sees the slowest
    assert all(abs(o["rate"] - 2 * 10 / 1.5) < 1e-12 for o in outs)  # all units over that time


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    env_keep = {k: os.environ.pop(k) for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK") if k in os.environ}
    try:
        rep = bench.Replicas("gloo")
        assert (rep.rank, rep.world, rep.local) == (0, 1, 0) and rep.dist is None
        rep.barrier()
        assert rep.max(3.25) == 3.25
        rep.close()
        assert bench.job_rate(1, 20, 2.0) == 10.0
    finally:
        os.environ.update(env_keep)


def test_reference_arm_other_ranks_exit_without_work():
    # rank 1 of 2 under torchrun: exits 0 at once, prints nothing, never touches the oracle
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       env=_env(1, 2, _free_port()), cwd=ROOT, capture_output=True, text=True, timeout=180)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_prints_one_complete_line():
    # The reference arm times the oracle on the host cores: every step is one measured outer
    # FGMRES iteration of back-to-back oracle solves (here 16 steps after 2 untimed ones, so the
    # first solve of 14 iterations finishes inside the run).  Its JSON line carries the contract
    # keys, a cpu_baseline describing the run, an e2e that moves no bytes, and the same config
    # object as the GPU arm.
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "2d256_p20",
                        "--steps", "16", "--warmup", "2"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["config"]["workload"] == "2d_lognormal_256x256_l10_a1e-2_p20"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] == 1 and cb["sample"]
    assert "measured in this run" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    per = d["oracle_ms_per_iteration"]
    assert len(per) == 16
    assert abs(sum(per) / 16 - d["ms_per_step"]) <= 0.1 + 1e-6 * d["ms_per_step"]
    # value = 16 iterations / (14 iterations per solve x the timed seconds)
    assert abs(d["value"] - 16 / (14 * sum(per) / 1e3)) <= 1e-3 * d["value"]
    sys.path.insert(0, ROOT)
    import bench
    from paper_2506_03947_gb300 import inputs
    P = inputs.config_2d(n=256, ell=10, alpha=1e-2, inner_its=20, seed_field=11, seed_b=12)
    assert d["config"] == json.loads(json.dumps(bench.bench_config("2d256_p20", P, 20, 1)))


def test_oracle_rate_counts_solve_equivalents():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.oracle_rate([1.0, 1.0, 2.0], 2) == 3 / (2 * 4.0)
