"""Multi-process host logic of the benchmark on CPU: two gloo ranks (the GPU path runs one
independent replica per GPU, so the only cross-rank steps are the barrier, the max over
ranks of the step time and rank 0's report)."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ms_values, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(ms_values[rank], world)
        value = bench.replica_value(1.0e9, ms, world)
        buf = io.StringIO()
        with redirect_stdout(buf):
            rc = bench.run_reference(bench.parse_args_for_test()) if rank != 0 else 0
        dist.barrier()
        out_q.put((rank, ms, value, rc, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ms_values = [12.5, 17.25]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, ms_values, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, rc, out in res:
        assert ms == 17.25                                  # the slowest rank's time
        assert abs(value - 2 * 1.0e9 / 17.25e-3) < 1e-3      # both replicas' work
        assert rc == 0
        if rank != 0:
            assert out == ""                                 # only rank 0 reports
