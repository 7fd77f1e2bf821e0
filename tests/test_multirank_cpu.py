"""The host logic of bench.py on CPU: two gloo ranks, the slowest rank's time
sets the job time, and the whole-job value counts every rank's product
(independent replicas, weak scaling, no collective on the data path); the
reference arm (the FP64 oracle on the host cores) prints the contract's line
on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [10.0, 25.0][rank]
    m = bench.max_over_ranks(ms, world)
    v = bench.job_value(world, 1e9, 4, m)
    out.put((rank, m, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in res:
        assert m == 25.0
        assert v == pytest.approx(2 * 1e9 * 4 / 0.025 / 1e9)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_value(1, 1e9, 2, 1000.0) == pytest.approx(2.0)


def _bench(args, env_extra=None):
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py")] + args, cwd=root,
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_line_and_nonzero_ranks():
    """`bench.py --impl reference` times the oracle on the host cores and prints
    the contract's line; under several ranks only rank 0 works and prints."""
    (line,) = _bench(["--impl", "reference", "--n", "512", "--steps", "1", "--warmup", "3"])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "Gop/s"
    assert line["steps"] == 1 and line["warmup"] == 3 and line["higher_is_better"] is True
    assert line["vs_baseline"] is None and line["data"] == "synthetic"
    assert "workload" in line["config"] and line["config"]["n"] == 512
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert "entries" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "Gop/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert _bench(["--impl", "reference", "--n", "512", "--steps", "1", "--warmup", "3"],
                  {"RANK": "1", "WORLD_SIZE": "2"}) == []
