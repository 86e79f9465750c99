"""The multi-process path of bench.py (one replica per rank) on CPU: the timing of a step is
the maximum over ranks, taken with a gloo all-reduce (world size 2, 127.0.0.1)."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [3.5, 7.25][rank]
    q.put((rank, bench.max_over_ranks(mine, dist), bench.max_over_ranks(mine, None)))
    dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
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
    assert res == [(0, 7.25, 3.5), (1, 7.25, 7.25)]


def test_traffic_is_reported_only_for_the_profiled_source():
    """The ncu DRAM traffic in the bench line holds while the kernel source is the one that was
    profiled; a changed source (a table entry with another hash) or an unknown configuration
    reports none."""
    sys.path.insert(0, ROOT)
    import bench
    import hashlib
    key = ("blocked", "greedy", 2500, 8, 512, 0)
    src = os.path.join(ROOT, "paper_1812_01448_gb300", "csrc", bench.NCU_TRAFFIC[key][1])
    same = hashlib.sha1(open(src, "rb").read()).hexdigest() == bench.NCU_TRAFFIC[key][2]
    nbytes, prof = bench._traffic(key)
    if same:
        assert nbytes == float(bench.NCU_TRAFFIC[key][0]) and prof.startswith("profiles/")
    else:
        assert nbytes is None and "changed" in prof
    assert bench._traffic(("plain", "rcm", 0, 0, 0, 0)) == (None, None)
    saved = bench.NCU_TRAFFIC[key]
    try:
        bench.NCU_TRAFFIC[key] = saved[:2] + ("0" * 40,) + saved[3:]
        nbytes, why = bench._traffic(key)
        assert nbytes is None and "changed" in why
    finally:
        bench.NCU_TRAFFIC[key] = saved
