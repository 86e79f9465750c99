"""The seeded workloads: meshes, initial fields, source profiles and plasma densities.

Recipes (seed = 1000 + workload number unless stated):

1. PEC cavity a=1, b=0.5: 33x17 lattice, h=1/32, +-0.2h jitter, local redraw to a 0.05h
   Delaunay margin; B(t=dt/2) = TE(1,1) = cos(pi x/a) cos(pi y/b) sampled at the circumcentres
   (the caller passes those points in), E(0) = 0.
2. Unit square, PEC walls, PEC equilateral hole of side 0.2 centred at (0.5, 0.5); spacing
   graded linearly from 2e-4 at the hole to 8e-4; about 4M triangles, jitter 0.2h; soft
   line source at x = 0.35.
3. Unit square, uniform spacing giving about 1M triangles (20k for the oracle downscale);
   Gaussian plasma density; same line source.
4. A batch of independent meshes with log-uniform sizes and random scatterers.
"""
from __future__ import annotations

import math

import numpy as np

from .core import (MeshArrays, cavity_lattice, edge_table, graded_square, polygon_ellipse,
                   polygon_rectangle, polygon_triangle)


def cavity_te11_mesh(seed: int = 1001) -> MeshArrays:
    return cavity_lattice(33, 17, 1.0, 0.5, jitter=0.2, dual_floor=0.05, seed=seed)


def te_mode_b(points: np.ndarray, m: int, n: int, a: float, b: float) -> np.ndarray:
    """TE(m,n) magnetic field cos(m pi x/a) cos(n pi y/b) at the given points."""
    return np.cos(m * np.pi * points[:, 0] / a) * np.cos(n * np.pi * points[:, 1] / b)


# linear grading slope giving ~4.0M triangles with h 2e-4 .. 8e-4 around the side-0.2 hole
SCATTERER_GRADE = 0.0105


def scatterer_mesh(seed: int = 1002, h_min: float = 2e-4, h_max: float = 8e-4,
                   grade: float = SCATTERER_GRADE, jitter: float = 0.2,
                   side: float = 0.2) -> MeshArrays:
    hole = polygon_triangle((0.5, 0.5), side)
    return graded_square(h_min, h_max, grade=grade, holes=[hole], jitter=jitter, seed=seed)


def uniform_spacing_for(n_tris: float, area: float = 1.0) -> float:
    """Spacing h of an equilateral-ish mesh with n_tris triangles over the given area."""
    return math.sqrt(4.0 * area / (math.sqrt(3.0) * n_tris))


def plasma_square_mesh(n_tris: int = 1_000_000, seed: int = 1003, jitter: float = 0.2) -> MeshArrays:
    h = uniform_spacing_for(n_tris)
    return graded_square(h, h, grade=0.0, holes=(), jitter=jitter, seed=seed)


def plasma_density_nodes(xy: np.ndarray, omega0: float = 2 * math.pi * 20, peak_frac: float = 0.8,
                         width: float = 0.15, center=(0.5, 0.5)) -> np.ndarray:
    """n(r) = (peak_frac*omega0)^2 exp(-|r-c|^2 / (2 width^2)) at the nodes."""
    r2 = (xy[:, 0] - center[0]) ** 2 + (xy[:, 1] - center[1]) ** 2
    return (peak_frac * omega0) ** 2 * np.exp(-r2 / (2 * width ** 2))


def source_line_amplitudes(xy: np.ndarray, tris: np.ndarray, x_s: float, h: float,
                           amplitude: float = 1.0, cutoff: float = 3.0):
    """Soft vertical line source: a_i = A (e_i . y) exp(-((x_mid - x_s)/(1.5 h))^2).

    Returns (edge_ids, a) in the caller edge numbering (unique (lo, hi) node pairs sorted
    lexicographically), interior edges only, Gaussian cut at ``cutoff`` widths.
    """
    edges, he_edge, _, cnt = edge_table(np.asarray(tris, np.int64), xy.shape[0])
    p0 = xy[edges[:, 0]]
    p1 = xy[edges[:, 1]]
    v = p1 - p0
    ey = v[:, 1] / np.hypot(v[:, 0], v[:, 1])
    xm = 0.5 * (p0[:, 0] + p1[:, 0])
    w = 1.5 * h
    sel = (cnt == 2) & (np.abs(xm - x_s) < cutoff * w) & (np.abs(ey) > 0)
    ids = np.nonzero(sel)[0]
    a = amplitude * ey[ids] * np.exp(-((xm[ids] - x_s) / w) ** 2)
    return ids.astype(np.int32), a.astype(np.float64)


def batch_specs(n_meshes: int = 512, seed: int = 1004, n_min: int = 5_000, n_max: int = 200_000):
    """Parameters of a batch of independent meshes: log-uniform sizes, one random scatterer
    each (triangle, ellipse or rotated rectangle of size U[0.1, 0.3]), jitter U[0, 0.3] h, and
    a source frequency omega0 = 2 pi U[10, 30].  All draws come from one seeded stream."""
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(n_meshes):
        n_t = float(math.exp(rng.uniform(math.log(n_min), math.log(n_max))))
        kind = int(rng.integers(3))
        size = float(rng.uniform(0.1, 0.3))
        ang = float(rng.uniform(0, 2 * math.pi))
        c = (0.5 + float(rng.uniform(-0.1, 0.1)), 0.5 + float(rng.uniform(-0.1, 0.1)))
        aspect = float(rng.uniform(0.5, 1.0)) if kind == 1 else float(rng.uniform(0.4, 1.0))
        jit = float(rng.uniform(0.0, 0.3))
        omega0 = 2 * math.pi * float(rng.uniform(10, 30))
        specs.append(dict(index=k, n_tris=n_t, kind=("triangle", "ellipse", "rectangle")[kind],
                          size=size, angle=ang, center=c, aspect=aspect, jitter=jit,
                          omega0=omega0, seed=int(rng.integers(1 << 31))))
    return specs


def batch_mesh(spec) -> MeshArrays:
    """Build one mesh of ``batch_specs``."""
    size, ang, c = spec["size"], spec["angle"], spec["center"]
    if spec["kind"] == "triangle":
        hole = polygon_triangle(c, size, ang)
        area = math.sqrt(3) / 4 * size ** 2
    elif spec["kind"] == "ellipse":
        ra, rb = size / 2, size / 2 * spec["aspect"]
        hole = polygon_ellipse(c, ra, rb, ang, n_vertices=48)
        area = math.pi * ra * rb
    else:
        w, hh = size, size * spec["aspect"]
        hole = polygon_rectangle(c, w, hh, ang)
        area = w * hh
    h = uniform_spacing_for(spec["n_tris"], 1.0 - area)
    return graded_square(h, h, grade=0.0, holes=[hole], jitter=spec["jitter"], seed=spec["seed"])


def batch_meshes(n_meshes: int = 512, seed: int = 1004, n_min: int = 5_000, n_max: int = 200_000):
    """Yield dict(mesh=..., **spec) for each mesh of the batch (sequentially)."""
    for spec in batch_specs(n_meshes, seed, n_min, n_max):
        yield dict(mesh=batch_mesh(spec), **spec)


def learned_specs(n_meshes: int, seed: int = 1005, n_min: int = 1_000, n_max: int = 50_000):
    """Corpus for the learned spectral-radius predictor: log-uniform sizes, jitter U[0, 0.3] h,
    grading ratio h_max/h_min U[1, 8] around one random scatterer (triangle, ellipse or rotated
    rectangle of size U[0.1, 0.3]).  All draws come from one seeded stream."""
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(n_meshes):
        n_t = float(math.exp(rng.uniform(math.log(n_min), math.log(n_max))))
        kind = int(rng.integers(3))
        size = float(rng.uniform(0.1, 0.3))
        ang = float(rng.uniform(0, 2 * math.pi))
        c = (0.5 + float(rng.uniform(-0.1, 0.1)), 0.5 + float(rng.uniform(-0.1, 0.1)))
        aspect = float(rng.uniform(0.5, 1.0)) if kind == 1 else float(rng.uniform(0.4, 1.0))
        specs.append(dict(index=k, n_tris=n_t, kind=("triangle", "ellipse", "rectangle")[kind],
                          size=size, angle=ang, center=c, aspect=aspect,
                          jitter=float(rng.uniform(0.0, 0.3)), ratio=float(rng.uniform(1.0, 8.0)),
                          omega0=2 * math.pi * 20, seed=int(rng.integers(1 << 31))))
    return specs


def learned_mesh(spec) -> MeshArrays:
    """Build one mesh of ``learned_specs``: spacing graded from h at the scatterer to ratio*h
    over a band of width 0.2, h chosen so that a uniform mesh of h_max would have n_tris / ratio
    triangles (the graded mesh then lands near n_tris)."""
    size, ang, c = spec["size"], spec["angle"], spec["center"]
    if spec["kind"] == "triangle":
        hole = polygon_triangle(c, size, ang)
    elif spec["kind"] == "ellipse":
        hole = polygon_ellipse(c, size / 2, size / 2 * spec["aspect"], ang, n_vertices=48)
    else:
        hole = polygon_rectangle(c, size, size * spec["aspect"], ang)
    ratio = spec["ratio"]
    h_max = uniform_spacing_for(spec["n_tris"] / max(1.0, ratio ** 0.5))
    h_min = h_max / ratio
    grade = (h_max - h_min) / 0.2
    return graded_square(h_min, h_max, grade=grade, holes=[hole], jitter=spec["jitter"],
                         seed=spec["seed"])


def cached(name: str, make, cache_dir: str | None = None) -> MeshArrays:
    """Return make() memoised in an .npz under $UE_MESH_CACHE (default: the system temp dir).

    Large graded meshes take tens of seconds to generate; tests and the benchmark that run in
    one session share them through this cache.  ``name`` must encode every generator argument.
    """
    import os
    import tempfile
    d = cache_dir or os.environ.get("UE_MESH_CACHE") or os.path.join(tempfile.gettempdir(), "ue_meshcache")
    os.makedirs(d, exist_ok=True)
    path = os.path.join(d, name + ".npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        return MeshArrays(z["xy"], z["tris"], float(z["h"]), z["boundary_node"], dict(cached=path))
    m = make()
    tmp = path + f".{os.getpid()}.tmp.npz"
    np.savez(tmp, xy=m.xy, tris=m.tris, h=m.h, boundary_node=m.boundary_node)
    os.replace(tmp, path)
    return m
