"""Host logic of bench.py with several ranks, on CPU with the gloo backend
(world size 2): max-over-ranks timing, barriers, round-robin sharding of
independent domains, and the reference arm printing on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout
from pathlib import Path
from types import SimpleNamespace

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, ws: int, port: int, q) -> None:
    try:
        os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                          MASTER_PORT=str(port))
        sys.path.insert(0, str(ROOT))
        import torch.distributed as dist
        dist.init_process_group("gloo", rank=rank, world_size=ws)
        import bench
        m = bench._max_over_ranks(ws, 10.0 + rank)
        bench._barrier(ws)
        part = bench.shard(11, rank, ws)
        out = io.StringIO()
        with redirect_stdout(out):
            rc = bench.run_reference(SimpleNamespace(gpus=ws, steps=1, warmup=0), ws, rank) if rank == 1 else 0
        dist.destroy_process_group()
        q.put((rank, m, part, rc, out.getvalue()))
    except Exception as e:  # reported to the parent
        q.put((rank, repr(e), None, None, None))


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        rank, m, part, rc, printed = res[r]
        assert m == 11.0, res[r]               # maximum over ranks
        assert part == list(range(r, 11, 2))
    assert sorted(res[0][2] + res[1][2]) == list(range(11))
    assert res[1][3] == 0 and res[1][4] == ""  # reference arm: rank 1 exits without work or output


def test_shard_covers_items_once():
    sys.path.insert(0, str(ROOT))
    import bench
    for ws in (1, 2, 3, 8):
        parts = [bench.shard(256, r, ws) for r in range(ws)]
        assert sorted(sum(parts, [])) == list(range(256))
