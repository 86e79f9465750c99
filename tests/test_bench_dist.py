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


def test_counters_are_reported_only_for_the_profiled_sources(tmp_path, monkeypatch):
    """The ncu counters in the bench line (DRAM traffic, shared-memory wavefronts, instructions)
    hold while the kernel's sources hash as they did at the capture; changed sources or an
    uncaptured configuration report none."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    key = {"workload": "scatterer", "variant": "blocked", "tiler": "greedy", "tile_tris": 2500,
           "block_depth": 8, "threads": 512, "frame": 0, "kernel": "split"}
    rec = {"config": key, "sources_sha1": bench.sources_sha1(),
           "per_launch": {"dram_bytes": 5.0, "smem_wavefronts": 7.0, "smem_instructions": 3.5,
                          "warp_instructions": 11.0}}
    f = tmp_path / "counters.json"
    f.write_text(json.dumps({"records": [rec]}))
    monkeypatch.setattr(bench, "COUNTER_FILE", str(f))
    got, why = bench._counters(key)
    assert why is None and got["per_launch"]["dram_bytes"] == 5.0
    assert bench._counters(dict(key, tile_tris=2048)) == (None, "configuration not captured")
    f.write_text(json.dumps({"records": [dict(rec, sources_sha1="0" * 40)]}))
    got, why = bench._counters(key)
    assert got is None and "changed" in why
    # the committed file parses and every record names a configuration and a sources hash
    with open(os.path.join(ROOT, "profiles", "ncu_counters.json")) as fh:
        for r in json.load(fh)["records"]:
            assert set(r["config"]) == set(key) and len(r["sources_sha1"]) == 40


def test_onchip_roofline_from_counters(monkeypatch):
    """roofline.onchip: shared-memory wavefronts against one per SM per cycle, warp instructions
    against four per SM per cycle, and the load/store split against one wavefront per
    instruction (the cp.async writes reported apart)."""
    sys.path.insert(0, ROOT)
    import types
    import bench
    fake_props = types.SimpleNamespace(multi_processor_count=100)
    import torch
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: fake_props)
    c = {"smem_wavefronts": 2.0e6, "warp_instructions": 8.0e6, "smem_instructions": 1.0e6,
         "pipe_lsu_wavefronts_mem_shared_op_ld": 1.2e6, "pipe_lsu_wavefronts_mem_shared_op_st": 0.3e6,
         "pipe_lsu_wavefronts_mem_shared_op_misc": 0.5e6}
    r = bench.onchip_roofline(c, 0.1, 1000.0)          # 0.1 ms at 1 GHz on 100 SMs
    assert abs(r["smem"]["frac"] - 2.0e6 / (1e-4 * 100 * 1e9)) < 1e-12
    assert abs(r["issue"]["frac"] - 8.0e6 / (1e-4 * 4 * 100 * 1e9)) < 1e-12
    assert abs(r["smem"]["bank_conflict_factor"] - 1.5) < 1e-12
    assert r["smem"]["cp_async_wavefronts"] == 0.5e6
    # without the split, the factor falls back to all wavefronts over instructions
    r = bench.onchip_roofline({k: c[k] for k in ("smem_wavefronts", "warp_instructions", "smem_instructions")},
                              0.1, None)
    assert abs(r["smem"]["bank_conflict_factor"] - 2.0) < 1e-12 and r["clock_mhz"] == 2070.0
