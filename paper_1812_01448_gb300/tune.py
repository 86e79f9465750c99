"""Autotuner for batched stepping: variant, tiler and tile size, threads per tile, blocking depth.

Many independent meshes advance together (ue_batch_create).  Which launch form is fastest
depends on the meshes' sizes and on the GPU: one E and one B launch per step over the whole
batch, one cooperative persistent launch per chunk of steps, or temporal blocking (KD or
greedy tiles of at most ``tile_tris`` triangles advanced ``block_depth`` steps per launch by 512
or 1024 threads).
The tuner times each candidate on a sample of the meshes, spread over their size
distribution, as a real batch: built by the library, stepped inside its CUDA graphs, timed
with CUDA events on the launching stream.  Each mesh keeps its own source; a fixed small dt
is used because speed does not depend on it.

Only the library's calls are sequenced here; all stepping work runs in libue.so.
"""
from __future__ import annotations

import time

import numpy as np

from .api import Mesh, batch_create
from . import _native as N

# (variant, tiler, tile_tris, block_depth, tb_threads); plain and persistent use the tiled
# order too.
DEFAULT_CANDIDATES = (
    ("plain", "kd", 2048, 1, 512),
    ("persistent", "kd", 2048, 1, 512),
    ("blocked", "kd", 1024, 4, 512),
    ("blocked", "kd", 2048, 4, 512),
    ("blocked", "kd", 2048, 6, 512),
    ("blocked", "kd", 2048, 8, 512),
    ("blocked", "kd", 2048, 8, 1024),
    ("blocked", "greedy", 2500, 8, 512),
    ("blocked", "rings", 2500, 8, 512),
    ("blocked", "rings", 2500, 10, 512),
)

TILERS = {"kd": N.UE_REORDER_KD, "greedy": N.UE_REORDER_GREEDY, "rings": N.UE_REORDER_GREEDY_RINGS}

_VARIANT = {"plain": N.UE_VARIANT_PLAIN, "persistent": N.UE_VARIANT_PERSISTENT,
            "blocked": N.UE_VARIANT_BLOCKED}


def spread(sizes, k: int) -> list[int]:
    """Indices of k items evenly spaced through the items sorted by size (all if k >= n)."""
    order = np.argsort(np.asarray(sizes), kind="stable")
    n = len(order)
    if k >= n:
        return [int(i) for i in order]
    pos = np.round(np.linspace(0, n - 1, k)).astype(np.int64)
    return [int(order[p]) for p in np.unique(pos)]


def _steps_for(steps: int, depth: int) -> int:
    return max(depth, steps - steps % depth)


def time_batch(items, variant: str, tile_tris: int, block_depth: int, tb_threads: int,
               steps: int = 192, warmup: int = 48, stream=None, meshes=None, tiler: str = "kd") -> float:
    """Triangle-steps/s of one configuration on a batch of ``items`` = (MeshArrays, source
    edge ids, amplitudes, omega0).  ``meshes`` may hold already loaded Mesh objects of the same
    items, tiler and tile size (they are rebuilt for this variant)."""
    import torch
    own = meshes is None
    if own:
        meshes = [Mesh(ms.xy, ms.tris, reorder=TILERS[tiler], tile_tris=tile_tris) for ms, *_ in items]
    for m, (ms, ids, amp, w0) in zip(meshes, items):
        m.geometry_build(stream=stream, dt_mode=N.UE_DT_GIVEN, dt=1e-7, variant=_VARIANT[variant],
                         block_depth=block_depth, tb_threads=tb_threads, graph_chunk=32)
        m.set_source(ids, amp, w0, 0.1, 0.05)
    b = batch_create(meshes, stream)
    try:
        b.step_n(_steps_for(warmup, block_depth), stream)
        n = _steps_for(steps, block_depth)
        s = torch.cuda.current_stream() if stream is None else stream
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        b.step_n(n, stream)
        e1.record(s)
        torch.cuda.synchronize()
        rate = b.n_tris * n / (e0.elapsed_time(e1) * 1e-3)
    finally:
        b.close()
        if own:
            for m in meshes:
                m.close()
    return rate


def autotune_batch(items, candidates=DEFAULT_CANDIDATES, sample: int = 32, steps: int = 192,
                   stream=None):
    """Time every candidate on a spread sample of ``items``; return (best, table).  ``best``
    and each row of ``table`` are dicts with variant, tile_tris, block_depth, tb_threads and
    rate (triangle-steps/s on the sample), plus the tiler; the table also records the tuning
    time."""
    idx = spread([ms.n_tris for ms, *_ in items], sample)
    sub = [items[i] for i in idx]
    t0 = time.perf_counter()
    table = []
    by_tile: dict[tuple, list] = {}
    for c in candidates:
        by_tile.setdefault((c[1], int(c[2])), []).append(c)
    for (tiler, tile), cands in by_tile.items():
        meshes = [Mesh(ms.xy, ms.tris, reorder=TILERS[tiler], tile_tris=tile) for ms, *_ in sub]
        try:
            for variant, _, _, depth, threads in cands:
                row = dict(variant=variant, tiler=tiler, tile_tris=tile, block_depth=depth, tb_threads=threads)
                try:
                    row["rate"] = time_batch(sub, variant, tile, depth, threads, steps=steps, stream=stream,
                                             meshes=meshes, tiler=tiler)
                except N.UEError as e:
                    # a configuration the library refuses for these meshes (a tile with its halo
                    # beyond the blocked kernel's capacity): recorded, not chosen
                    if e.code != N.UE_ERR_ARG:
                        raise
                    row["rate"], row["refused"] = 0.0, str(e)
                table.append(row)
        finally:
            for m in meshes:
                m.close()
    usable = [r for r in table if "refused" not in r]
    if not usable:
        raise ValueError("autotune_batch: the library refused every candidate for these meshes")
    best = max(usable, key=lambda r: r["rate"])
    return dict(best), {"rows": table, "sample_meshes": len(sub),
                        "sample_tris": int(sum(ms.n_tris for ms, *_ in sub)),
                        "seconds": time.perf_counter() - t0}
