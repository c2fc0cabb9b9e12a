"""The N > 1 path of bench.py on CPU: two gloo ranks (one process each)
report the slowest rank's time and the whole-job throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slowest
    max_ms, value = bench.job_throughput(local_ms, 1000, 10, world, dist, "cpu")
    q.put((rank, max_ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, max_ms, value in res:
        assert max_ms == 150.0
        assert value == pytest.approx(1000 * 10 * 2 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    max_ms, value = bench.job_throughput(200.0, 100, 5, 1, None)
    assert max_ms == 200.0 and value == pytest.approx(2500.0)


@pytest.mark.parametrize("extra", [[], ["--mode", "train", "--workload", "product_bf16"]])
def test_reference_arm_prints_one_line(extra):
    # The reference arm times the FP64 oracle on the host cores and prints the
    # same JSON line shape as the main arm (no GPU involved).
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--ref-sample", "64"] + extra,
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["unit"] == line["e2e"]["unit"]
