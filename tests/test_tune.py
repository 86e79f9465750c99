"""Batch autotuner: sampling over the size distribution (host) and a tuned batch on the GPU."""
import numpy as np
import pytest

from paper_1812_01448_gb300 import tune


def test_spread_covers_the_size_range():
    sizes = [50, 7, 300, 12, 99, 5, 1000, 64, 20, 8]
    idx = tune.spread(sizes, 4)
    assert len(idx) == 4 == len(set(idx))
    got = sorted(sizes[i] for i in idx)
    assert got[0] == min(sizes) and got[-1] == max(sizes)
    assert sorted(tune.spread(sizes, 99)) == list(range(len(sizes)))


def test_candidates_are_valid_launch_forms():
    for variant, tiler, tile, depth, threads in tune.DEFAULT_CANDIDATES:
        assert variant in ("plain", "persistent", "blocked") and tiler in tune.TILERS
        assert tile >= 256 and threads in (512, 1024)
        assert depth >= 1 and (variant == "blocked" or depth == 1)


def test_autotune_skips_a_refused_configuration(monkeypatch):
    """A candidate the library refuses with UE_ERR_ARG (a tile with its halo too large for the
    blocked kernel) is recorded as refused and never chosen; other errors propagate (host only:
    the timing is replaced by a stand-in)."""
    import meshgen
    from paper_1812_01448_gb300 import _native as N
    items = []
    for sp in meshgen.batch_specs(3, seed=78, n_min=600, n_max=1500):
        ms = meshgen.batch_mesh(sp)
        items.append((ms, None, None, sp["omega0"]))

    def fake_time(sub, variant, tile, depth, threads, **kw):
        if depth == 10:
            raise N.UEError(N.UE_ERR_ARG, "ue_geometry_build")
        return 1e9 * depth
    monkeypatch.setattr(tune, "time_batch", fake_time)
    cands = (("blocked", "rings", 300, 4, 512), ("blocked", "rings", 300, 10, 512),
             ("blocked", "rings", 300, 8, 512))
    best, table = tune.autotune_batch(items, candidates=cands, sample=3)
    assert best["block_depth"] == 8 and best["rate"] == 8e9
    refused = [r for r in table["rows"] if "refused" in r]
    assert len(refused) == 1 and refused[0]["block_depth"] == 10 and refused[0]["rate"] == 0.0

    def broken(*a, **kw):
        raise N.UEError(-5, "ue_step_n")
    monkeypatch.setattr(tune, "time_batch", broken)
    with pytest.raises(N.UEError):
        tune.autotune_batch(items, candidates=cands[:1], sample=3)


@pytest.mark.gpu
def test_autotune_picks_a_measured_candidate():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import meshgen
    from paper_1812_01448_gb300 import build
    build.build()
    items = []
    for sp in meshgen.batch_specs(5, seed=77, n_min=3000, n_max=12000):
        ms = meshgen.batch_mesh(sp)
        ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.3, ms.h)
        items.append((ms, ids, amp, sp["omega0"]))
    cands = (("plain", "kd", 512, 1, 512), ("persistent", "kd", 512, 1, 512),
             ("blocked", "kd", 512, 4, 512), ("blocked", "greedy", 600, 4, 512))
    best, table = tune.autotune_batch(items, candidates=cands, sample=3, steps=48)
    assert table["sample_meshes"] == 3 and len(table["rows"]) == 4
    assert all(r["rate"] > 0 and np.isfinite(r["rate"]) for r in table["rows"])
    assert best["rate"] == max(r["rate"] for r in table["rows"])
