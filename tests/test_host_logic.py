"""Host-side checks that need no GPU: the C ABI library exports every function its
header declares, and the multi-rank timing of bench.py (gloo, world size 2) reports the
slowest rank and gives every replica its own box."""
import os
import re
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "sdot.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sdot_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    from paper_2110_08868_gb300 import build as b

    path = b.build()
    import ctypes

    lib = ctypes.CDLL(path)
    names = _declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2110_08868_gb300 import binding

    assert sorted(binding.EXPORTS) == names


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 * (rank + 1), dist)
    cfg = bench.replica_config("zeldovich-16^3-kinv-0.3a", rank, world)
    dist.destroy_process_group()
    q.put((rank, ms, cfg["seed"]))


def test_bench_replicas_gloo_world2():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [20.0, 20.0]  # both ranks see the max
    assert out[0][2] != out[1][2]                # independent boxes
