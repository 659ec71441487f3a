"""The benchmark's host logic on the CPU: the replica helpers with two gloo
ranks (max over ranks, distinct images per rank, whole-job throughput), the
reference arm's JSON line, and the reference arm under two ranks (rank 0
alone prints)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    r, w, _ = bench.dist_init("gloo")
    ms = [5.0, 7.5][r]  # this rank's timed region
    ms_max = bench.max_over_ranks(ms, w, "cpu")
    seeds = [bench.replica_seed(1, r, j) for j in range(2)]
    rate = bench.job_rate(12e6, w, 10, ms_max)
    bench.dist_barrier(w)
    torch.distributed.destroy_process_group()
    q.put((r, ms_max, seeds, rate))


def test_replica_helpers_two_gloo_ranks():
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    ps = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [7.5, 7.5]              # every rank sees the slowest time
    assert not set(res[0][2]) & set(res[1][2])            # different images on every rank
    assert res[0][3] == pytest.approx(2 * 12e6 * 10 / 7.5e-3 / 1e6)  # all units / slowest time


def _run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_json_line():
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "3", "--ref-seconds", "0.2"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "MP/s"
    assert d["config"]["workload"] == "wdr-12mp-fwd"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "3", "--ref-seconds", "0.2"],
                   {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""
