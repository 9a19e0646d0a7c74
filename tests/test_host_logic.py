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


def test_header_is_plain_c_and_links(tmp_path):
    # the C ABI is usable from C: the header compiles as C99 without warnings and a C
    # program links the library and calls host-only entry points
    import shutil
    import subprocess

    from paper_2110_08868_gb300 import build as b

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lib = b.build()
    src = tmp_path / "abi.c"
    src.write_text(r"""
#include <stdio.h>
#include "sdot.h"
int main(void) {
    sdot_options o;
    sdot_server_options so;
    double box[3] = {1.0, 1.0, 1.0};
    size_t bytes = 0;
    if (sdot_default_options(&o) != SDOT_OK || o.k != 24) return 1;
    if (sdot_server_default_options(&so) != SDOT_OK || so.max_active != 8) return 2;
    if (sdot_server_footprint(32768, box, &o, &bytes) != SDOT_OK || bytes == 0) return 3;
    if (sdot_server_footprint(1, box, &o, &bytes) != SDOT_ERR_ARG) return 4;
    printf("%zu %s\n", bytes, sdot_last_error());
    return 0;
}
""")
    exe = tmp_path / "abi"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"), str(src), lib,
                        "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert int(r.stdout.split()[0]) > 32768 * 1000


def _bench(args, env_extra=None, timeout=600):
    import json
    import subprocess

    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args,
                       capture_output=True, text=True, timeout=timeout, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_bench_reference_arm_contract():
    # the reference arm (the CPU oracle on a bounded sample) prints one JSON line with
    # the keys of the bench contract; a small box keeps it fast
    out = _bench(["--impl", "reference", "--steps", "1", "--warmup", "1",
                  "--workload", "zeldovich-16^3-kinv-0.3a"])
    assert len(out) == 1
    line = out[0]
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["config"]["workload"] == "zeldovich-16^3-kinv-0.3a"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_bench_reference_arm_other_ranks_are_silent():
    out = _bench(["--impl", "reference", "--steps", "1", "--warmup", "0",
                  "--workload", "zeldovich-16^3-kinv-0.3a"],
                 {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out == []
