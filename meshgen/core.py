"""Node placement, Qhull triangulation, hole carving and seeded jitter.

Every generator takes a ``seed`` and returns a :class:`MeshArrays` with caller-order node
coordinates (float64 [n_n, 2]) and triangles (int32 [n_t, 3]).  Triangles are returned
counter-clockwise, but consumers must not rely on it (ingest re-orients).

Mesh quality is controlled by the *Delaunay margin* of each interior edge, the sum over its
two triangles of ``|e|/2 * cot(opposite angle)``.  A positive margin everywhere means the
triangulation is Delaunay; the generators redraw node jitter locally until every margin is at
least ``dual_floor * h`` (h = local target spacing), the local-redraw rule for jittered
lattices.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.spatial import Delaunay, cKDTree


@dataclasses.dataclass
class MeshArrays:
    xy: np.ndarray            # float64 [n_n, 2]
    tris: np.ndarray          # int32 [n_t, 3]
    h: float                  # nominal (finest) spacing
    boundary_node: np.ndarray  # bool [n_n]
    info: dict

    @property
    def n_nodes(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


# ----------------------------------------------------------------------------------------
# edge adjacency and the Delaunay margin
# ----------------------------------------------------------------------------------------

def edge_table(tris: np.ndarray, n_nodes: int):
    """Unique undirected edges and their incident half-edges.

    Returns (edges [n_e,2] sorted (lo,hi), half_edge_edge [3*n_t], half_edge_opp [3*n_t],
    count [n_e]).  Half-edge k = 3*j + q joins tris[j,q] -> tris[j,(q+1)%3], opposite vertex
    tris[j,(q+2)%3].
    """
    a = tris[:, [0, 1, 2]].reshape(-1).astype(np.int64)
    b = tris[:, [1, 2, 0]].reshape(-1).astype(np.int64)
    opp = tris[:, [2, 0, 1]].reshape(-1).astype(np.int64)
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    key = lo * np.int64(n_nodes) + hi
    uniq, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
    edges = np.stack([uniq // n_nodes, uniq % n_nodes], axis=1)
    return edges, inv, opp, cnt


def delaunay_margin(xy: np.ndarray, tris: np.ndarray):
    """Per interior edge: (edge index, margin, the up-to-4 quad vertices).

    margin = sum over the edge's two triangles of |e|/2 * cot(angle opposite the edge).
    """
    n_nodes = xy.shape[0]
    edges, he_edge, he_opp, cnt = edge_table(tris, n_nodes)
    pa = xy[edges[he_edge, 0]]
    pb = xy[edges[he_edge, 1]]
    po = xy[he_opp]
    u = pa - po
    v = pb - po
    dot = u[:, 0] * v[:, 0] + u[:, 1] * v[:, 1]
    crs = np.abs(u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0])
    with np.errstate(divide="ignore", invalid="ignore"):
        cot = dot / crs
    elen = np.hypot(pb[:, 0] - pa[:, 0], pb[:, 1] - pa[:, 1])
    contrib = 0.5 * elen * cot
    margin = np.zeros(edges.shape[0])
    np.add.at(margin, he_edge, contrib)
    interior = cnt == 2
    # opposite vertices per edge (first and second incident half-edge)
    order = np.argsort(he_edge, kind="stable")
    first = np.full(edges.shape[0], -1, np.int64)
    second = np.full(edges.shape[0], -1, np.int64)
    se = he_edge[order]
    starts = np.searchsorted(se, np.arange(edges.shape[0]))
    first[:] = he_opp[order[starts]]
    has2 = cnt == 2
    second[has2] = he_opp[order[starts[has2] + 1]]
    quad = np.stack([edges[:, 0], edges[:, 1], first, second], axis=1)
    return edges, margin, interior, quad


def _orient(xy, tris):
    p0 = xy[tris[:, 0]]
    p1 = xy[tris[:, 1]]
    p2 = xy[tris[:, 2]]
    return (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p1[:, 1] - p0[:, 1]) * (p2[:, 0] - p0[:, 0])


def _max_angle_cot(xy, tris):
    """cot of the largest angle of each triangle (negative when obtuse)."""
    cots = []
    for q in range(3):
        o = xy[tris[:, q]]
        u = xy[tris[:, (q + 1) % 3]] - o
        v = xy[tris[:, (q + 2) % 3]] - o
        cots.append((u[:, 0] * v[:, 0] + u[:, 1] * v[:, 1]) / np.abs(u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0]))
    return np.min(np.stack(cots), axis=0)


def _triangulate(xy: np.ndarray) -> np.ndarray:
    tri = Delaunay(xy, qhull_options="Qbb Qc Qz Q12").simplices.astype(np.int64)
    ar = _orient(xy, tri)
    scale = np.max(np.ptp(xy, axis=0)) ** 2
    keep = np.abs(ar) > 1e-13 * scale
    tri = tri[keep]
    ar = ar[keep]
    flip = ar < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return tri


# ----------------------------------------------------------------------------------------
# lattices
# ----------------------------------------------------------------------------------------

def cavity_lattice(nx: int = 33, ny: int = 17, a: float = 1.0, b: float = 0.5,
                   jitter: float = 0.2, dual_floor: float = 0.05, seed: int = 1001,
                   max_rounds: int = 5000) -> MeshArrays:
    """Jittered square lattice on [0,a]x[0,b], Delaunay-triangulated, with local redraw.

    Interior nodes move uniformly by +-jitter*h in x and y; boundary nodes stay fixed.  While
    any interior edge has Delaunay margin below dual_floor*h, the interior vertices of every
    offending edge's quad get fresh jitter from the same seeded stream and the cloud is
    re-triangulated.
    """
    hx = a / (nx - 1)
    hy = b / (ny - 1)
    h = min(hx, hy)
    X, Y = np.meshgrid(np.arange(nx) * hx, np.arange(ny) * hy, indexing="xy")
    base = np.stack([X.ravel(), Y.ravel()], axis=1)
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    bnd = ((ix == 0) | (ix == nx - 1) | (iy == 0) | (iy == ny - 1)).ravel()
    rng = np.random.default_rng(seed)
    xy = base.copy()
    free = np.nonzero(~bnd)[0]
    xy[free] += rng.uniform(-jitter * h, jitter * h, size=(free.size, 2))
    rounds = 0
    while True:
        tris = _triangulate(xy)
        edges, margin, interior, quad = delaunay_margin(xy, tris)
        bad = interior & (margin < dual_floor * h)
        if not bad.any():
            break
        rounds += 1
        if rounds > max_rounds:
            raise RuntimeError("cavity_lattice: local redraw did not converge")
        nodes = np.unique(quad[bad].reshape(-1))
        nodes = nodes[(nodes >= 0) & ~bnd[nodes]]
        xy[nodes] = base[nodes] + rng.uniform(-jitter * h, jitter * h, size=(nodes.size, 2))
    _, margin, interior, _ = delaunay_margin(xy, tris)
    info = dict(kind="cavity_lattice", a=a, b=b, nx=nx, ny=ny, jitter=jitter, seed=seed,
                redraw_rounds=rounds, min_margin_over_h=float(margin[interior].min() / h))
    return MeshArrays(xy, tris.astype(np.int32), h, bnd, info)


def right_split_lattice(nx: int, ny: int, a: float, b: float) -> MeshArrays:
    """Square lattice with every cell cut by its rising diagonal (cocircular quads)."""
    hx = a / (nx - 1)
    hy = b / (ny - 1)
    X, Y = np.meshgrid(np.arange(nx) * hx, np.arange(ny) * hy, indexing="xy")
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)
    tris = []
    for j in range(ny - 1):
        for i in range(nx - 1):
            p00 = j * nx + i
            p10 = p00 + 1
            p01 = p00 + nx
            p11 = p01 + 1
            tris.append((p00, p10, p11))
            tris.append((p00, p11, p01))
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    bnd = ((ix == 0) | (ix == nx - 1) | (iy == 0) | (iy == ny - 1)).ravel()
    return MeshArrays(xy, np.asarray(tris, np.int32), min(hx, hy), bnd,
                      dict(kind="right_split", a=a, b=b, nx=nx, ny=ny))


def equilateral_lattice(n_rows: int, h: float, jitter: float = 0.0, seed: int = 0) -> MeshArrays:
    """Rows of equilateral triangles of side h (a parallelogram strip, every row offset)."""
    rng = np.random.default_rng(seed)
    rh = h * math.sqrt(3.0) / 2.0
    ncols = n_rows
    pts = []
    for r in range(n_rows + 1):
        for c in range(ncols + 1):
            pts.append((c * h + 0.5 * h * r, r * rh))
    xy = np.asarray(pts, np.float64)
    tris = []
    W = ncols + 1
    for r in range(n_rows):
        for c in range(ncols):
            p = r * W + c
            tris.append((p, p + 1, p + W))
            tris.append((p + 1, p + W + 1, p + W))
    rr, cc = np.divmod(np.arange(xy.shape[0]), W)
    bnd = (rr == 0) | (rr == n_rows) | (cc == 0) | (cc == ncols)
    if jitter > 0:
        free = ~bnd
        xy[free] += rng.uniform(-jitter * h, jitter * h, size=(int(free.sum()), 2))
    return MeshArrays(xy, np.asarray(tris, np.int32), h, bnd,
                      dict(kind="equilateral", n_rows=n_rows, jitter=jitter, seed=seed))


def random_delaunay(n_points: int, seed: int, dual_floor: float = 0.0) -> MeshArrays:
    """Delaunay triangulation of the unit square's corners plus uniform random points."""
    rng = np.random.default_rng(seed)
    pts = np.concatenate([np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float64),
                          rng.random((n_points, 2))])
    tris = _triangulate(pts)
    h = 1.0 / math.sqrt(n_points)
    bnd = np.zeros(pts.shape[0], bool)
    bnd[:4] = True
    return MeshArrays(pts, tris.astype(np.int32), h, bnd, dict(kind="random", seed=seed))


# ----------------------------------------------------------------------------------------
# polygons (holes) and graded, conforming meshes of the unit square
# ----------------------------------------------------------------------------------------

def polygon_triangle(center, side, angle=0.0):
    """Equilateral triangle, counter-clockwise vertices."""
    R = side / math.sqrt(3.0)
    th = angle + np.pi / 2 + np.arange(3) * 2 * np.pi / 3
    return np.stack([center[0] + R * np.cos(th), center[1] + R * np.sin(th)], axis=1)


def polygon_rectangle(center, w, hgt, angle=0.0):
    c, s = math.cos(angle), math.sin(angle)
    loc = np.array([[-w / 2, -hgt / 2], [w / 2, -hgt / 2], [w / 2, hgt / 2], [-w / 2, hgt / 2]])
    rot = np.array([[c, -s], [s, c]])
    return loc @ rot.T + np.asarray(center)[None, :]


def polygon_ellipse(center, ra, rb, angle=0.0, n_vertices=64):
    t = np.arange(n_vertices) * 2 * np.pi / n_vertices
    loc = np.stack([ra * np.cos(t), rb * np.sin(t)], axis=1)
    c, s = math.cos(angle), math.sin(angle)
    rot = np.array([[c, -s], [s, c]])
    return loc @ rot.T + np.asarray(center)[None, :]


def _seg_dist(p: np.ndarray, poly: np.ndarray) -> np.ndarray:
    """Distance from points p [n,2] to the closed polygon boundary poly [m,2]."""
    d = np.full(p.shape[0], np.inf)
    m = poly.shape[0]
    for k in range(m):
        a = poly[k]
        b = poly[(k + 1) % m]
        ab = b - a
        t = np.clip(((p - a) @ ab) / (ab @ ab), 0.0, 1.0)
        q = a[None, :] + t[:, None] * ab[None, :]
        d = np.minimum(d, np.hypot(p[:, 0] - q[:, 0], p[:, 1] - q[:, 1]))
    return d


def _inside(p: np.ndarray, poly: np.ndarray) -> np.ndarray:
    """Even-odd point-in-polygon."""
    x = p[:, 0]
    y = p[:, 1]
    inside = np.zeros(p.shape[0], bool)
    m = poly.shape[0]
    for k in range(m):
        x0, y0 = poly[k]
        x1, y1 = poly[(k + 1) % m]
        cond = (y0 > y) != (y1 > y)
        with np.errstate(divide="ignore", invalid="ignore"):
            xc = x0 + (y - y0) * (x1 - x0) / (y1 - y0)
        inside ^= cond & (x < xc)
    return inside


def _seed_segment(a, b, size_fn):
    """Nodes on segment a->b (a included, b excluded) spaced by the size function."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    L = float(np.hypot(*(b - a)))
    s = [0.0]
    while True:
        p = a + (b - a) * (s[-1] / L)
        step = float(size_fn(p[None, :])[0])
        if s[-1] + 0.5 * step >= L:
            break
        s.append(s[-1] + step)
    n = len(s)
    # stretch so that the last interval ends exactly at b
    s = np.asarray(s) * (L / (s[-1] + float(size_fn(b[None, :])[0]))) if n > 1 else np.array([0.0])
    return a[None, :] + (b - a)[None, :] * (s[:, None] / L)


class _Quads:
    """Fixed connectivity of a triangulation: evaluates Delaunay margins for moving nodes."""

    def __init__(self, tris: np.ndarray, n_nodes: int):
        self.tris = tris
        edges, he_edge, he_opp, cnt = edge_table(tris, n_nodes)
        self.edges = edges
        self.he_edge = he_edge
        self.he_opp = he_opp
        self.interior = cnt == 2
        order = np.argsort(he_edge, kind="stable")
        starts = np.searchsorted(he_edge[order], np.arange(edges.shape[0]))
        self.he0 = order[starts]
        self.he1 = np.where(self.interior, order[np.minimum(starts + 1, order.size - 1)], -1)
        first = he_opp[self.he0]
        second = np.where(self.interior, he_opp[np.maximum(self.he1, 0)], -1)
        self.quad = np.stack([edges[:, 0], edges[:, 1], first, second], axis=1)
        self.ne = edges.shape[0]

    def _half(self, xy, he):
        e = self.he_edge[he]
        pa = xy[self.edges[e, 0]]
        pb = xy[self.edges[e, 1]]
        po = xy[self.he_opp[he]]
        u = pa - po
        v = pb - po
        dot = u[:, 0] * v[:, 0] + u[:, 1] * v[:, 1]
        crs = np.abs(u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0])
        elen = np.hypot(pb[:, 0] - pa[:, 0], pb[:, 1] - pa[:, 1])
        with np.errstate(divide="ignore", invalid="ignore"):
            return 0.5 * elen * dot / crs

    def margin(self, xy, eids=None):
        """Margins of the given interior edges (all edges, boundary ones included, if None)."""
        if eids is None:
            m = self._half(xy, self.he0)
            m[self.interior] += self._half(xy, self.he1[self.interior])
            return m
        return self._half(xy, self.he0[eids]) + self._half(xy, self.he1[eids])


def graded_square(h_min: float, h_max: float, grade: float = 0.0, holes=(), jitter: float = 0.2,
                  dual_floor: float = 0.005, seed: int = 0, repair_rounds: int = 200,
                  attempts: int = 8) -> MeshArrays:
    """Graded Delaunay mesh of the unit square around convex polygonal holes (see
    ``_graded_square_once``).  A draw whose repair cannot reach a positive margin everywhere is
    discarded and redrawn with the next seed (seed + 1, seed + 2, ...)."""
    last = None
    for a in range(attempts):
        try:
            m = _graded_square_once(h_min, h_max, grade, holes, jitter, dual_floor, seed + a,
                                    repair_rounds)
            m.info["attempt"] = a
            return m
        except RuntimeError as e:
            last = e
    raise last


def _graded_square_once(h_min: float, h_max: float, grade: float = 0.0, holes=(), jitter: float = 0.2,
                        dual_floor: float = 0.005, seed: int = 0, repair_rounds: int = 200) -> MeshArrays:
    """Graded Delaunay mesh of the unit square around convex polygonal holes.

    Target spacing h(x) = clip(h_min + grade * dist(x, holes), h_min, h_max) (h_max
    everywhere without holes).  Interior nodes come from randomly offset hexagonal lattices,
    one per spacing level (levels a factor 2**0.25 apart), thinned where levels meet; boundary
    nodes are seeded along the square and the hole outlines at the local spacing.  Interior
    nodes are jittered by +-jitter*h(x), the cloud is triangulated once by Qhull and the
    triangles inside holes are removed.  Then, with that connectivity held fixed, the interior
    vertices of every quad whose Delaunay margin is below dual_floor*h are moved again
    (+-0.15h around their triangulated position) until no margin is below the floor and no
    triangle is flipped.
    """
    rng = np.random.default_rng(seed)
    holes = [np.asarray(hp, np.float64) for hp in holes]
    graded = bool(holes) and grade > 0

    def hfun(p):
        if not graded:
            return np.full(p.shape[0], h_max)
        d = np.min(np.stack([_seg_dist(p, hp) for hp in holes]), axis=0)
        return np.clip(h_min + grade * d, h_min, h_max)

    H_min = h_min if graded else h_max
    H_max = h_max
    # --- interior lattice points, level by level
    ratio = 2 ** 0.25
    n_lev = max(1, int(math.ceil(math.log(H_max / H_min) / math.log(ratio) - 1e-9)) + 1)
    pts = []
    for k in range(n_lev):
        Hk = min(H_min * ratio ** k, H_max)
        rh = Hk * math.sqrt(3.0) / 2
        ox, oy = rng.uniform(0, Hk), rng.uniform(0, rh)
        ny_ = int(math.ceil(1.0 / rh)) + 2
        nx_ = int(math.ceil(1.0 / Hk)) + 2
        J, I = np.meshgrid(np.arange(-1, ny_), np.arange(-1, nx_), indexing="ij")
        P = np.stack([(I * Hk + 0.5 * Hk * (J % 2) + ox).ravel(), (J * rh + oy).ravel()], axis=1)
        P = P[(P[:, 0] > 0) & (P[:, 0] < 1) & (P[:, 1] > 0) & (P[:, 1] < 1)]
        if P.shape[0] == 0:
            continue
        if n_lev > 1:
            lv = np.clip(np.rint(np.log(hfun(P) / H_min) / math.log(ratio)), 0, n_lev - 1)
            P = P[lv.astype(int) == k]
        pts.append(P)
    P = np.concatenate(pts)
    # drop interior points inside holes or too close to any boundary
    Hp = hfun(P)
    bd = np.minimum.reduce([P[:, 0], 1 - P[:, 0], P[:, 1], 1 - P[:, 1]])
    keep = bd > 0.6 * Hp
    for hp in holes:
        keep &= ~_inside(P, hp)
        keep &= _seg_dist(P, hp) > 0.6 * Hp
    P = P[keep]
    Hp = Hp[keep]
    if n_lev > 1:
        # thin points closer than 0.7*h to an already accepted point (fine levels first)
        order = np.argsort(Hp, kind="stable")
        P = P[order]
        Hp = Hp[order]
        close = cKDTree(P).query_pairs(r=0.7 * H_max, output_type="ndarray")
        acc = np.ones(P.shape[0], bool)
        if close.size:
            i, j = close[:, 0], close[:, 1]
            lim = 0.7 * np.minimum(Hp[i], Hp[j])
            close = close[np.hypot(*(P[i] - P[j]).T) < lim]
            close.sort(axis=1)
            close = close[np.lexsort((close[:, 0], close[:, 1]))]
            ptr = np.searchsorted(close[:, 1], np.arange(P.shape[0] + 1))
            for j in np.unique(close[:, 1]):
                if acc[close[ptr[j]:ptr[j + 1], 0]].any():
                    acc[j] = False
        P = P[acc]
        Hp = Hp[acc]
    if jitter > 0:
        P = P + rng.uniform(-jitter, jitter, size=P.shape) * Hp[:, None]
    # --- boundary nodes
    corners = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float64)
    B = [_seed_segment(corners[k], corners[(k + 1) % 4], hfun) for k in range(4)]
    for hp in holes:
        for k in range(hp.shape[0]):
            B.append(_seed_segment(hp[k], hp[(k + 1) % hp.shape[0]], hfun))
    B = np.concatenate(B)
    xy = np.concatenate([B, P])
    bnd = np.zeros(xy.shape[0], bool)
    bnd[:B.shape[0]] = True
    tris = _triangulate(xy)
    c = (xy[tris[:, 0]] + xy[tris[:, 1]] + xy[tris[:, 2]]) / 3
    out = np.zeros(tris.shape[0], bool)
    for hp in holes:
        out |= _inside(c, hp)
    tris = tris[~out]
    # drop nodes no longer used (inside holes there are none, but be safe)
    used = np.zeros(xy.shape[0], bool)
    used[tris.reshape(-1)] = True
    remap = np.cumsum(used) - 1
    xy = xy[used]
    bnd = bnd[used]
    tris = remap[tris]
    # --- local repair of low-margin quads with the connectivity held fixed
    base = xy.copy()
    hb = hfun(base)
    Q = _Quads(tris, xy.shape[0])
    hmid = 0.5 * (hb[Q.edges[:, 0]] + hb[Q.edges[:, 1]])
    floor = dual_floor * hmid
    free = ~bnd

    def offenders(xy_, moved):
        em = moved[Q.quad].any(axis=1) & Q.interior
        ee = np.nonzero(em)[0]
        bad = ee[Q.margin(xy_, ee) < floor[ee]]
        tt = np.nonzero(moved[tris].any(axis=1))[0]
        inv = tt[_orient(xy_, tris[tt]) <= 0]
        nodes = np.unique(np.concatenate([Q.quad[bad].reshape(-1), tris[inv].reshape(-1)]))
        return nodes[(nodes >= 0) & free[nodes]]

    moved = np.ones(xy.shape[0], bool)
    rounds = 0
    for rounds in range(repair_rounds):
        nodes = offenders(xy, moved)
        if nodes.size == 0:
            break
        xy[nodes] = base[nodes] + rng.uniform(-0.15, 0.15, size=(nodes.size, 2)) * hb[nodes, None]
        moved = np.zeros(xy.shape[0], bool)
        moved[nodes] = True
    margin = Q.margin(xy)
    rel = margin[Q.interior] / hmid[Q.interior]
    info = dict(kind="graded_square", h_min=h_min, h_max=h_max, grade=grade, jitter=jitter,
                seed=seed, repair_rounds=rounds, dual_floor=dual_floor,
                min_margin_over_h=float(rel.min()),
                frac_below_0p05h=float(np.mean(rel < 0.05)))
    if not (_orient(xy, tris) > 0).all() or rel.min() <= 0:
        raise RuntimeError("graded_square: could not reach a positive Delaunay margin")
    return MeshArrays(xy, tris.astype(np.int32), h_min, bnd, info)
