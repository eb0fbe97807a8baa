"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank gets the slowest
rank's time and the whole-job rate counts every rank's frames; the reference arm runs on rank 0
only."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    e = bench.max_over_ranks(0.5 + rank, "cpu")
    q.put((rank, e, bench.whole_job_rate(world, 16, 10, e)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [1.5, 1.5]
    assert res[0][2] == pytest.approx(2 * 16 * 10 / 1.5)


def test_reference_arm_ranks_other_than_zero_do_nothing(capsys):
    import bench

    class A:
        warmup, steps, gpus = 1, 1, 2
    bench.run_reference(A, rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(capsys):
    """The reference arm as the driver launches it (rank 0 of one): the oracle times frames of
    the batched workload on the host cores and prints one JSON line with the contract's keys,
    the reference arm's own e2e (no host-device copies) and its CPU-baseline record."""
    import json

    import bench

    class A:
        warmup, steps, gpus = 1, 2, 1
    bench.run_reference(A, rank=0, world=1)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "img/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2 and d["n_gpus"] == 1
    assert d["config"]["workload"] == bench.WORKLOAD
    assert d["e2e"] == {"value": d["value"], "unit": "img/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
