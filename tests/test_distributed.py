"""The N > 1 path of the benchmark, on CPU ranks: one process per rank joins a gloo process
group through bench.py's own setup, the ranks meet at the barrier, and the timing and
throughput reductions (max over ranks of the step time, sum over ranks of the work) give
the same totals on every rank.  With one GPU per call, the multi-GPU form is replicas
(independent instances per rank, no data-path collective); these reductions are its only
exchange."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q) -> None:
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), ODMD_BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench

    try:
        r, w, local, dist = bench.dist_setup(world)
        bench.barrier(dist)
        step_ms = 10.0 + rank       # each rank's own time
        work = 50.0 * (rank + 1)    # each rank's own units
        q.put((r, w, local, bench.max_over_ranks(step_ms, dist), bench.sum_over_ranks(work, dist)))
        bench.barrier(dist)
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent
        q.put(("error", repr(e)))


def test_rank_reductions_over_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(o[0] != "error" for o in out), out
    assert sorted(o[0] for o in out) == [0, 1]
    for r, w, local, mx, sm in out:
        assert w == world and local == r
        assert mx == 11.0                 # the slowest rank sets the step time
        assert sm == 50.0 + 100.0         # the work of every replica counts
