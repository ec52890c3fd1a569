"""The multi-GPU bookkeeping of the benchmark, as two gloo ranks on the CPU:
each rank solves its own block of right-hand sides (distinct seeds, no data
exchange) and the job's throughput is the summed count over the slowest time."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_2103_07329_gb300 import multirank as MR
    from paper_2103_07329_gb300 import problems as P
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = MR.rank_env()
    B = P.rhs_uniform(1000, 4, MR.rhs_seed(r), m_draw=32)
    t_local = [0.5, 2.0][r]
    solved = [4, 3][r]
    value, t_max, total = MR.job_throughput(t_local, solved, dist, "cpu")
    out.put((r, w, local, float(B[0, 0]), value, t_max, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    assert res[0][3] != res[1][3]                      # distinct right-hand sides
    for r in res:
        assert r[5] == 2.0 and r[6] == 7                # slowest time, summed count
        assert r[4] == pytest.approx(7 / 2.0)


def test_single_process_throughput():
    from paper_2103_07329_gb300 import multirank as MR
    assert MR.job_throughput(2.0, 10, None) == (5.0, 2.0, 10)
    from paper_2103_07329_gb300 import problems as P
    b0 = P.rhs_uniform(100, 4, MR.rhs_seed(0), m_draw=32)
    assert np.array_equal(b0, P.rhs_uniform(100, 32, 0)[:, :4])
