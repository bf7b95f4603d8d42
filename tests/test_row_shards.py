"""The row-shard reduction protocol on CPU ranks (gloo): each rank holds a contiguous range
of row blocks of the basis and the snapshots, forms pass A's 2 r + 3 per-block partial sums
(Sec. 2.3's row-local products: L^T e, L^T x, e.e, e.x, x.x with e = c - L a), exchanges the
per-block partials, and adds them in block order.  Every rank must get bitwise the sums of
one process that holds every row, for 2 and 3 ranks, with blocks of unequal size."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, R, BLOCKS = 3001, 7, 13


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _data():
    rng = np.random.default_rng(7)
    L, _ = np.linalg.qr(rng.standard_normal((N, R)))
    c, x = rng.standard_normal(N), rng.standard_normal(N)
    a = L.T @ c + 1e-3 * rng.standard_normal(R)  # carried coefficients, as the update holds them
    return L, c, x, a


def _block_partials(L, c, x, a, rows, blocks):
    """Pass A's partial sums of each row block in `blocks` (row-local arithmetic only)."""
    out = []
    for b in blocks:
        s = slice(rows[b], rows[b + 1])
        e = c[s] - L[s] @ a
        out.append(np.concatenate([L[s].T @ e, L[s].T @ x[s], [e @ e, e @ x[s], x[s] @ x[s]]]))
    return np.array(out)


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    try:
        import torch
        import torch.distributed as dist

        from paper_2311_18715_gb300 import shards

        dist.init_process_group("gloo", rank=rank, world_size=world)
        L, c, x, a = _data()
        rows = shards.row_blocks(N, BLOCKS)
        first, count = shards.shard_blocks(BLOCKS, world, rank)
        # this rank holds only the rows of its blocks
        lo, hi = rows[first], rows[first + count]
        mine = _block_partials(L[lo:hi], c[lo:hi], x[lo:hi], a, [r - lo for r in rows[first:first + count + 1]],
                               range(count))
        allp = shards.exchange_partials(torch.from_numpy(mine), first, BLOCKS)
        q.put((rank, shards.fold(allp.numpy()).tobytes(), (lo, hi)))
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent
        q.put(("error", repr(e), None))


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_reduction_is_bitwise_the_unsharded_one(world):
    sys.path.insert(0, ROOT)
    from paper_2311_18715_gb300 import shards

    L, c, x, a = _data()
    rows = shards.row_blocks(N, BLOCKS)
    assert rows[0] == 0 and rows[-1] == N and all(r % 64 == 0 for r in rows[:-1])
    want = shards.fold(_block_partials(L, c, x, a, rows, range(BLOCKS)))
    e = c - L @ a  # the sums by their definition, for scale
    ref = np.concatenate([L.T @ e, L.T @ x, [e @ e, e @ x, x @ x]])
    np.testing.assert_allclose(want, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())

    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(o[0] != "error" for o in out), out
    spans = sorted(o[2] for o in out)
    assert spans[0][0] == 0 and spans[-1][1] == N and all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
    for rank, got, _ in out:
        assert np.frombuffer(got, dtype=np.float64).tobytes() == want.tobytes(), rank


def test_shard_ranges_cover_the_blocks():
    sys.path.insert(0, ROOT)
    from paper_2311_18715_gb300 import shards

    for blocks in (1, 5, 152):
        for g_count in range(1, min(blocks, 6) + 1):
            spans = [shards.shard_blocks(blocks, g_count, g) for g in range(g_count)]
            assert spans[0][0] == 0 and sum(cnt for _, cnt in spans) == blocks
            assert all(spans[g][0] + spans[g][1] == spans[g + 1][0] for g in range(g_count - 1))
            assert all(cnt >= 1 for _, cnt in spans)
    with pytest.raises(ValueError):
        shards.shard_blocks(4, 5, 0)
    with pytest.raises(ValueError):
        shards.row_blocks(100, 3)  # two 64-row tiles cannot make three blocks
