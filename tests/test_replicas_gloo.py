"""Multi-GPU replicas on the CPU: two gloo ranks aggregate like bench.py does.

The traversal path has no collective; bench.py only combines per-rank
timings (max) and traversed edges (sum) after the timed region.  This runs
that combination with world_size 2 on the gloo backend.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, edges = bench.aggregate_ranks(10.0 + rank * 5.0, 1000 * (rank + 1), world)
    e2e = bench.combine_e2e({"value": 0.0, "unit": "GTEPS", "_ms": 20.0 + rank, "_edges": 500,
                             "h2d_bytes_per_step": 8, "d2h_bytes_per_step": 4, "steps": 4,
                             "ms_per_step": 0.0}, world)
    q.put((rank, ms, edges, bench.rank_source_offset(rank), e2e))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_aggregate_max_time_and_total_edges():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms, edges, off, e2e in res:
        assert ms == 15.0 and edges == 3000.0
        # e2e: both ranks' edges over the slower rank's region, both ranks' bytes
        assert e2e["value"] == 1000 / (21.0 / 1e3) / 1e9 and e2e["ms_per_step"] == 21.0 / 4
        assert e2e["h2d_bytes_per_step"] == 16 and e2e["d2h_bytes_per_step"] == 8
        assert "_ms" not in e2e and "_edges" not in e2e
    assert res[0][3] != res[1][3]          # replicas run different sources


def test_single_rank_needs_no_collective():
    import bench
    assert bench.aggregate_ranks(3.0, 42, 1) == (3.0, 42.0)
