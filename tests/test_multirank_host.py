"""Host logic of the multi-rank bench (N > 1), run as two gloo ranks on CPU.

With N GPUs bench.py gives every rank its own cosmology (independent
problems: no collective on the data path) and reports the job's step time as
the largest rank's, the all-reduce MAX over ranks.  Here two spawned CPU
processes on 127.0.0.1 run exactly those functions of bench.py.
"""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    from paper_1812_07437_gb300 import workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cosmo = bench.rank_cosmology(workloads.FIDUCIAL, rank)
    job = bench.job_step_ms(100.0 + 37.0 * rank, world, "cpu")
    every = [None] * world
    dist.all_gather_object(every, cosmo)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as fh:
        json.dump({"job_ms": job, "cosmologies": every}, fh)


@pytest.mark.timeout(180)
def test_two_gloo_ranks_independent_problems_and_max_time(tmp_path):
    mp.spawn(_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    # the job's step time is the slower rank's, on every rank
    assert [r["job_ms"] for r in res] == [137.0, 137.0]
    # rank 0 the fiducial, rank 1 a +1% step of one parameter: different problems
    c0, c1 = res[0]["cosmologies"]
    from paper_1812_07437_gb300 import workloads
    assert c0 == workloads.FIDUCIAL
    diff = [k for k in c0 if c0[k] != c1[k]]
    assert len(diff) == 1 and c1[diff[0]] == pytest.approx(1.01 * c0[diff[0]])


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1812_07437_gb300 import workloads
    assert bench.job_step_ms(42.0, 1, "cpu") == 42.0
    assert bench.rank_cosmology(workloads.FIDUCIAL, 0) == workloads.FIDUCIAL
    # eight ranks: eight distinct cosmologies
    cs = [tuple(sorted(bench.rank_cosmology(workloads.FIDUCIAL, r).items())) for r in range(8)]
    assert len(set(cs)) == 8
