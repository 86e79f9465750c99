"""Mesh generation: Delaunay triangulation of a node cloud and flip refinement (oracle).

Test infrastructure only.  Section 3 ("Mesh generation"): the boundary, the objects and any
paths are seeded with nodes, the area between them is seeded at the same spacing, and the
classical Delaunay method triangulates the convex hull of the cloud.  Triangles may then cross
the geometry; the paper restores it by flipping the two triangles on each edge that crosses a
geometry segment (Fig. 5a), and notes that the plain form fails where several neighbouring
triangles cross the same segment.

Readings (where the paper gives the idea but not the procedure):
* the triangulation covers the convex hull of all nodes (no node may repeat, and not all may be
  collinear);
* a geometry segment is a pair of node ids.  Its crossing edges are flipped in a queue: an edge
  whose two triangles form a strictly convex quadrilateral is flipped, and its new diagonal goes
  back on the queue if it still crosses the segment; an edge whose quadrilateral is not convex
  waits at the back of the queue until flips around it make it convex.  This queue (Sloan's
  constrained-edge recovery) always ends, which covers the case of several crossing triangles.
  A node on the open segment, or two segments that cross, is an error;
* afterwards every edge that is neither a segment nor on the hull, and is not locally Delaunay,
  is flipped (Lawson) until none is left.  The result is then the constrained Delaunay
  triangulation: unique for nodes in general position (no four cocircular);
* regions: the triangles reachable from a hole point without crossing a segment are dropped;
  with drop_exterior, so are those reachable through a hull edge that is not a segment;
* orientation and in-circle signs are exact: the determinants are evaluated over
  fractions.Fraction of the double coordinates.

Steps, in the paper's order: any triangulation of the hull (a left-to-right sweep), Lawson
flips to the Delaunay triangulation, flip refinement of the segments, Lawson flips with the
segments fixed, region removal.

Parity: pinned by tests/test_oracle_triangulate.py (the empty-circumcircle definition by brute
force over all triples, Qhull's triangulation of random clouds, a hand-worked four-node kite
with and without its long diagonal as a segment, and a checker of the constrained Delaunay
property -- every segment an edge, every other interior edge locally Delaunay, the hull or the
domain covered exactly -- that shares no code with the construction).
"""
from __future__ import annotations

from collections import deque
from fractions import Fraction

import numpy as np


class TriangulationError(ValueError):
    pass


def _F(xy):
    return [(Fraction(float(x)), Fraction(float(y))) for x, y in np.asarray(xy, np.float64)]


def orient(P, a, b, c) -> int:
    """Sign of twice the signed area of (a, b, c): +1 counter-clockwise."""
    (ax, ay), (bx, by), (cx, cy) = P[a], P[b], P[c]
    d = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
    return (d > 0) - (d < 0)


def incircle(P, a, b, c, d) -> int:
    """+1 where d lies strictly inside the circumcircle of the CCW triangle (a, b, c)."""
    rows = []
    for v in (a, b, c):
        x, y = P[v][0] - P[d][0], P[v][1] - P[d][1]
        rows.append((x, y, x * x + y * y))
    (ax, ay, al), (bx, by, bl), (cx, cy, cl) = rows
    det = al * (bx * cy - by * cx) - bl * (ax * cy - ay * cx) + cl * (ax * by - ay * bx)
    return (det > 0) - (det < 0)


def canonical(tris) -> np.ndarray:
    """Each CCW triangle rotated to start at its smallest node, rows sorted: a set in order."""
    out = []
    for t in np.asarray(tris, np.int64).reshape(-1, 3):
        k = int(np.argmin(t))
        out.append(tuple(int(t[(k + i) % 3]) for i in range(3)))
    return np.asarray(sorted(out), np.int64).reshape(-1, 3)


# ------------------------------------------------------------------ a triangulation of the hull

def sweep_triangulation(P):
    """Nodes in (x, y) order; each new node is outside the hull so far and joins every hull edge
    it sees strictly.  The first nodes may be collinear: they wait as a chain for the first node
    off their line."""
    n = len(P)
    order = sorted(range(n), key=lambda i: P[i])
    for i in range(1, n):
        if P[order[i]] == P[order[i - 1]]:
            raise TriangulationError(f"node {order[i]} repeats node {order[i - 1]}")
    k = 2
    while k < n and orient(P, order[0], order[1], order[k]) == 0:
        k += 1
    if k == n:
        raise TriangulationError("all nodes are collinear")
    chain, p = order[:k], order[k]
    tris = []
    s = orient(P, chain[0], chain[1], p)
    for a, b in zip(chain[:-1], chain[1:]):
        tris.append((a, b, p) if s > 0 else (b, a, p))
    # hull as a CCW cycle: the chain in its own order when p lies on its left, else reversed
    hull = [*chain, p] if s > 0 else [*reversed(chain), p]
    if not all(orient(P, hull[i], hull[(i + 1) % len(hull)], hull[(i + 2) % len(hull)]) >= 0
               for i in range(len(hull))):
        raise AssertionError("sweep hull lost its orientation")
    for p in order[k + 1:]:
        m = len(hull)
        vis = [orient(P, hull[i], hull[(i + 1) % m], p) < 0 for i in range(m)]
        if not any(vis):
            raise AssertionError("sweep node inside the hull")
        for i in range(m):
            if vis[i]:
                tris.append((hull[(i + 1) % m], hull[i], p))
        # the visible edges form one run; its inner nodes leave the hull, p enters
        first = next(i for i in range(m) if vis[i] and not vis[i - 1])
        last = first
        while vis[(last + 1) % m]:
            last = (last + 1) % m
        keep = [hull[(last + 1 + j) % m] for j in range((first - last - 1) % m + 1)]
        hull = keep + [p]
    return tris


# ------------------------------------------------------------------ flips

class _Tri:
    """Triangles as CCW triples; each directed edge maps to the triangle that holds it."""

    def __init__(self, P, tris):
        self.P = P
        self.t = [tuple(int(v) for v in r) for r in tris]
        self.alive = [True] * len(self.t)
        self.owner = {}
        for i, r in enumerate(self.t):
            self._own(i, r)

    def _own(self, i, r):
        for q in range(3):
            self.owner[(r[q], r[(q + 1) % 3])] = i

    def _drop(self, i):
        r = self.t[i]
        for q in range(3):
            del self.owner[(r[q], r[(q + 1) % 3])]
        self.alive[i] = False

    def apex(self, a, b):
        """The third node of the triangle holding (a, b), or None."""
        i = self.owner.get((a, b))
        if i is None:
            return None
        r = self.t[i]
        return next(v for v in r if v != a and v != b)

    def flippable(self, a, b) -> bool:
        c, d = self.apex(a, b), self.apex(b, a)
        return (c is not None and d is not None and orient(self.P, c, a, d) > 0
                and orient(self.P, d, b, c) > 0)

    def flip(self, a, b):
        """Triangles (a, b, c) and (b, a, d) become (c, a, d) and (d, b, c)."""
        c, d = self.apex(a, b), self.apex(b, a)
        self._drop(self.owner[(a, b)])
        self._drop(self.owner[(b, a)])
        for r in ((c, a, d), (d, b, c)):
            self.t.append(r)
            self.alive.append(True)
            self._own(len(self.t) - 1, r)
        return c, d

    def edges(self):
        return [(a, b) for (a, b) in self.owner if (b, a) not in self.owner or a < b]

    def triangles(self):
        return [r for r, ok in zip(self.t, self.alive) if ok]


def lawson(T: _Tri, fixed=frozenset()) -> int:
    """Flip interior edges outside `fixed` while one is not locally Delaunay."""
    flips = 0
    todo = [e for e in T.edges() if (e[1], e[0]) in T.owner]
    while todo:
        a, b = todo.pop()
        if (a, b) not in T.owner or (b, a) not in T.owner or frozenset((a, b)) in fixed:
            continue
        c, d = T.apex(a, b), T.apex(b, a)
        if incircle(T.P, a, b, c, d) <= 0:
            continue
        # d inside the circle of (a, b, c) and across ab: the quadrilateral is strictly convex
        assert T.flippable(a, b)
        T.flip(a, b)
        flips += 1
        todo += [(c, a), (a, d), (d, b), (b, c)]
    return flips


def _crosses(P, u, v, a, b) -> bool:
    """The open segments uv and ab cross at one interior point."""
    return (orient(P, u, v, a) * orient(P, u, v, b) < 0
            and orient(P, a, b, u) * orient(P, a, b, v) < 0)


def recover_segment(T: _Tri, u: int, v: int, fixed) -> int:
    """Flip refinement (Fig. 5a) of the segment uv; returns the flips made."""
    P = T.P
    for w in range(len(P)):
        if w != u and w != v and orient(P, u, v, w) == 0:
            lo = [min(P[u][i], P[v][i]) for i in range(2)]
            hi = [max(P[u][i], P[v][i]) for i in range(2)]
            if all(lo[i] <= P[w][i] <= hi[i] for i in range(2)):
                raise TriangulationError(f"node {w} lies on segment ({u}, {v})")
    queue = deque(e for e in T.edges() if len({u, v, *e}) == 4 and _crosses(P, u, v, *e))
    for e in queue:
        if frozenset(e) in fixed:
            raise TriangulationError(f"segments ({u}, {v}) and {e} cross")
    # the queue ends after at most about k^2 flips for k crossing edges; the cap only turns a
    # broken refinement into an error instead of an endless loop
    cap = 4 * (len(queue) + 1) ** 2 + 64
    flips, stall = 0, 0
    while queue:
        if flips > cap:
            raise AssertionError("flip refinement does not converge")
        a, b = queue.popleft()
        if not T.flippable(a, b):
            queue.append((a, b))
            stall += 1
            if stall > len(queue):
                raise AssertionError("flip refinement made no progress")
            continue
        stall = 0
        c, d = T.flip(a, b)
        flips += 1
        if len({u, v, c, d}) == 4 and _crosses(P, u, v, c, d):
            queue.append((c, d))
    assert (u, v) in T.owner or (v, u) in T.owner
    return flips


# ------------------------------------------------------------------ regions

def _locate(T: _Tri, pt):
    P = T.P + [(Fraction(float(pt[0])), Fraction(float(pt[1])))]
    q = len(P) - 1
    for i, r in enumerate(T.t):
        if T.alive[i] and all(orient(P, r[k], r[(k + 1) % 3], q) >= 0 for k in range(3)):
            return i
    raise TriangulationError(f"hole point {tuple(pt)} is outside the triangulation")


def drop_regions(T: _Tri, fixed, holes=(), drop_exterior=False):
    seeds = [_locate(T, h) for h in holes]
    if drop_exterior:
        for (a, b), i in T.owner.items():
            if (b, a) not in T.owner and frozenset((a, b)) not in fixed:
                seeds.append(i)
    gone = set(seeds)
    stack = list(seeds)
    while stack:
        r = T.t[stack.pop()]
        for q in range(3):
            a, b = r[q], r[(q + 1) % 3]
            j = T.owner.get((b, a))
            if j is not None and j not in gone and frozenset((a, b)) not in fixed:
                gone.add(j)
                stack.append(j)
    return [r for i, r in enumerate(T.t) if T.alive[i] and i not in gone]


# ------------------------------------------------------------------ the whole step

def triangulate(xy, segs=(), holes=(), drop_exterior=False):
    """(triangles (k, 3) CCW in canonical order, flips made in flip refinement)."""
    P = _F(xy)
    T = _Tri(P, sweep_triangulation(P))
    lawson(T)
    fixed = set()
    flips = 0
    for u, v in np.asarray(segs, np.int64).reshape(-1, 2):
        u, v = int(u), int(v)
        if u == v or not (0 <= u < len(P) and 0 <= v < len(P)):
            raise TriangulationError(f"bad segment ({u}, {v})")
        flips += recover_segment(T, u, v, fixed)
        fixed.add(frozenset((u, v)))
    lawson(T, fixed)
    return canonical(drop_regions(T, fixed, holes, drop_exterior)), flips


def delaunay_brute(xy):
    """The definition, for nodes in general position: every CCW triple whose circumcircle holds
    no other node, inside or on it.  O(n^4): tiny clouds only."""
    P = _F(xy)
    n = len(P)
    out = []
    for a in range(n):
        for b in range(a + 1, n):
            for c in range(b + 1, n):
                s = orient(P, a, b, c)
                if s == 0:
                    continue
                r = (a, b, c) if s > 0 else (a, c, b)
                if all(incircle(P, *r, d) < 0 for d in range(n) if d not in r):
                    out.append(r)
    return canonical(out)
