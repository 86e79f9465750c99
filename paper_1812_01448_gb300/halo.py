"""One mesh split into parts that step side by side and exchange their shared boundary every
step: the multi-GPU decomposition of the paper's "Divide and conqueror" section.

A part owns a set of triangles (a run of consecutive KD or greedy tiles, so that parts are
compact and their shared boundary l_Sigma small, Fig. 6).  Its local mesh is the owned
triangles plus the ring of triangles that share an edge with them, with nodes and triangles
numbered in the global caller order, so that edge directions, the sign table and the order of
every sum are those of the whole mesh.  One leap-frog step of the local mesh then gives, bit
for bit, the whole mesh's values:
- on every edge with an owned triangle (its two triangles' B are local and current);
- on every owned triangle (its three edges are such edges);
but not on the ring, whose outer edges the local mesh treats as boundary.  So after each step a
part receives B of its ring from the parts that own those triangles, and sends them B of its
own triangles that lie in their rings: one message each way per neighbouring part, of about
l_Sigma values.  E and the plasma current are never exchanged: both sides of a shared edge
compute them from the same inputs.

This module holds the host plan (numpy) and the step/exchange loop; the steps and the packing
of the exchanged values run in libue.so (ue_step_n, ue_exchange_tris).  The transport is
torch.distributed point-to-point (NCCL between GPUs, gloo between host processes), or direct
device copies when several parts share one process.
"""
from __future__ import annotations

import numpy as np


def _edge_keys(tris: np.ndarray, n_nodes: int):
    """Unique undirected edges of a triangle list as sorted keys lo * n + hi, and per
    half-edge (3 per triangle, q order of the listed vertices) the index of its edge."""
    t = np.asarray(tris, np.int64)
    a = t[:, [0, 1, 2]].reshape(-1)
    b = t[:, [1, 2, 0]].reshape(-1)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    keys = lo * n_nodes + hi
    uk, inv = np.unique(keys, return_inverse=True)
    return uk, inv.reshape(-1, 3)


def parts_from_tiles(tile_off: np.ndarray, perm_tri: np.ndarray, n_parts: int) -> np.ndarray:
    """Part of each caller triangle: consecutive tiles (in stored order) grouped into n_parts
    runs of nearly equal triangle counts.  tile_off: tile offsets in stored triangles (from
    Mesh.tiles()); perm_tri: caller id of each stored triangle (Mesh.tables()["perm_tri"])."""
    tile_off = np.asarray(tile_off, np.int64)
    n_t = int(tile_off[-1])
    if n_parts < 1 or n_parts > tile_off.size - 1:
        raise ValueError("n_parts must be between 1 and the number of tiles")
    # part boundaries at the tile offsets closest to multiples of n_t / n_parts
    cuts = [0]
    for p in range(1, n_parts):
        target = p * n_t / n_parts
        i = int(np.argmin(np.abs(tile_off - target)))
        i = max(i, cuts[-1] + 1)
        cuts.append(min(i, tile_off.size - 1 - (n_parts - p)))
    cuts.append(tile_off.size - 1)
    part_stored = np.empty(n_t, np.int32)
    for p in range(n_parts):
        part_stored[tile_off[cuts[p]]:tile_off[cuts[p + 1]]] = p
    part = np.empty(n_t, np.int32)
    part[np.asarray(perm_tri, np.int64)] = part_stored
    return part


class Plan:
    """Local meshes and exchange lists of a partition of one mesh.

    xy, tris: the whole mesh (caller numbering); part_of_tri: part of each caller triangle.
    For part p: ``tris_global[p]`` (owned and ring triangles, ascending caller ids; a triangle's
    local id is its position here), ``owned[p]`` (mask over them), ``nodes[p]`` (ascending
    caller node ids), ``local_xy(p)``, ``local_tris(p)``; ``send[p][q]`` (local ids in p of
    p-owned triangles in q's ring) and ``recv[p][q]`` (local ids in p of q-owned triangles in
    p's ring), in the same global order on both sides, so that p's send list to q and q's
    receive list from p name the same triangles.
    """

    def __init__(self, xy, tris, part_of_tri, n_parts: int | None = None):
        self.xy = np.asarray(xy, np.float64)
        self.tris = np.asarray(tris, np.int64)
        self.part = np.asarray(part_of_tri, np.int32)
        n_t = self.tris.shape[0]
        if self.part.shape != (n_t,):
            raise ValueError("part_of_tri must hold one part per triangle")
        self.n_parts = int(n_parts if n_parts is not None else self.part.max() + 1)
        if self.part.min() < 0 or self.part.max() >= self.n_parts:
            raise ValueError("part ids must lie in [0, n_parts)")
        n_nodes = self.xy.shape[0]
        self.edge_keys, he = _edge_keys(self.tris, n_nodes)
        self.he = he
        self._edge_owner = None
        # the triangles across each edge (-1 on the boundary)
        cnt = np.bincount(he.reshape(-1), minlength=self.edge_keys.size)
        if cnt.max() > 2:
            raise ValueError("non-manifold edge")
        order = np.argsort(he.reshape(-1), kind="stable")
        tri_of_he = np.repeat(np.arange(n_t), 3)[order]
        first = np.concatenate([[0], np.cumsum(cnt)[:-1]])
        t0 = tri_of_he[first]
        t1 = np.where(cnt == 2, tri_of_he[np.minimum(first + 1, tri_of_he.size - 1)], -1)
        other = np.where(t0[he] == np.arange(n_t)[:, None], t1[he], t0[he])     # [n_t, 3]
        self.nbr = other
        self.tris_global, self.owned, self.nodes = [], [], []
        for p in range(self.n_parts):
            own = np.nonzero(self.part == p)[0]
            nb = self.nbr[own].reshape(-1)
            nb = nb[nb >= 0]
            ring = np.unique(nb[self.part[nb] != p])
            tg = np.union1d(own, ring)
            self.tris_global.append(tg)
            self.owned.append(self.part[tg] == p)
            self.nodes.append(np.unique(self.tris[tg].reshape(-1)))
        self.send = [dict() for _ in range(self.n_parts)]
        self.recv = [dict() for _ in range(self.n_parts)]
        for p in range(self.n_parts):
            tg = self.tris_global[p]
            ring = tg[~self.owned[p]]
            for q in np.unique(self.part[ring]):
                g = ring[self.part[ring] == q]                 # ascending caller ids
                self.recv[p][int(q)] = np.searchsorted(tg, g).astype(np.int32)
                self.send[int(q)][p] = np.searchsorted(self.tris_global[q], g).astype(np.int32)

    def local_xy(self, p: int) -> np.ndarray:
        return self.xy[self.nodes[p]]

    def local_tris(self, p: int) -> np.ndarray:
        return np.searchsorted(self.nodes[p], self.tris[self.tris_global[p]]).astype(np.int32)

    def shared_boundary(self) -> int:
        """l_Sigma: interior edges whose two triangles lie in different parts (Fig. 6)."""
        a = np.repeat(np.arange(self.tris.shape[0]), 3)
        b = self.nbr.reshape(-1)
        m = (b > a) & (b >= 0)
        return int(np.count_nonzero(self.part[a[m]] != self.part[b[m]]))

    def exchange_sizes(self, p: int) -> dict:
        return {q: int(v.size) for q, v in self.send[p].items()}

    def local_edges(self, p: int, edge_ids: np.ndarray):
        """Global caller edge ids (edges numbered by sorted (lo, hi) node pairs) -> (positions
        in edge_ids that exist in part p's local mesh, their local edge ids)."""
        e = np.asarray(edge_ids, np.int64)
        n = self.xy.shape[0]
        key = self.edge_keys[e]
        lo, hi = key // n, key % n
        nodes = self.nodes[p]
        li, hi_ = np.searchsorted(nodes, lo), np.searchsorted(nodes, hi)
        ok = (li < nodes.size) & (hi_ < nodes.size)
        ok[ok] &= (nodes[li[ok]] == lo[ok]) & (nodes[hi_[ok]] == hi[ok])
        lk, _ = _edge_keys(self.local_tris(p), nodes.size)
        k = li * nodes.size + hi_
        pos = np.searchsorted(lk, k[ok])
        hit = np.zeros(ok.shape, bool)
        hit[np.nonzero(ok)[0]] = (pos < lk.size) & (lk[np.minimum(pos, lk.size - 1)] == k[ok])
        sel = np.nonzero(hit)[0]
        return sel, np.searchsorted(lk, k[sel]).astype(np.int64)

    def local_sources(self, p: int, edge_ids: np.ndarray, amp: np.ndarray):
        """A whole-mesh source (caller edge ids, amplitudes) restricted to part p: the sources
        on edges that are interior in p's local mesh, as (local edge ids, amplitudes)."""
        sel, lids = self.local_edges(p, edge_ids)
        _, he = _edge_keys(self.local_tris(p), self.nodes[p].size)
        cnt = np.bincount(he.reshape(-1))
        keep = cnt[lids] == 2
        return lids[keep].astype(np.int32), np.asarray(amp, np.float64)[sel][keep]

    def local_field_tris(self, p: int, B: np.ndarray) -> np.ndarray:
        return np.asarray(B)[self.tris_global[p]]

    def local_field_edges(self, p: int, E: np.ndarray) -> np.ndarray:
        """A whole-mesh edge field restricted to part p's local edges (local caller order)."""
        nodes = self.nodes[p]
        lk, _ = _edge_keys(self.local_tris(p), nodes.size)
        lo, hi = nodes[lk // nodes.size], nodes[lk % nodes.size]
        return np.asarray(E)[np.searchsorted(self.edge_keys, lo * self.xy.shape[0] + hi)]

    def global_edges_of(self, p: int) -> np.ndarray:
        """Global caller edge id of each local edge of part p."""
        nodes = self.nodes[p]
        lk, _ = _edge_keys(self.local_tris(p), nodes.size)
        lo, hi = nodes[lk // nodes.size], nodes[lk % nodes.size]
        return np.searchsorted(self.edge_keys, lo * self.xy.shape[0] + hi)

    def owned_edges(self, p: int) -> np.ndarray:
        """Mask over part p's local edges: the edges it owns, each edge of the whole mesh being
        owned by the smallest part among its triangles (both of them are local there)."""
        if self._edge_owner is None:
            g = np.full(self.edge_keys.size, np.iinfo(np.int32).max, np.int64)
            np.minimum.at(g, self.he.reshape(-1), np.repeat(self.part, 3))
            self._edge_owner = g
        return self._edge_owner[self.global_edges_of(p)] == p


def exchange_local(engines, plan: Plan):
    """One halo exchange between parts held by one process (engines[p] for part p): each part
    gathers the values its neighbours need, then each scatters what it receives."""
    out = {}
    for p, e in enumerate(engines):
        for q, ids in plan.send[p].items():
            out[(p, q)] = e.gather(ids)
    for p, e in enumerate(engines):
        for q, ids in plan.recv[p].items():
            e.scatter(ids, out[(q, p)])


def exchange_dist(engine, plan: Plan, rank: int, dist, device=None):
    """One halo exchange of this rank's part with its neighbours through torch.distributed
    point-to-point messages (one send and one receive per neighbouring part)."""
    import torch
    ops, recv = [], []
    for q, ids in sorted(plan.send[rank].items()):
        ops.append(dist.P2POp(dist.isend, engine.gather(ids), q))
    for q, ids in sorted(plan.recv[rank].items()):
        buf = torch.empty(ids.size, dtype=engine.dtype, device=device)
        recv.append((ids, buf))
        ops.append(dist.P2POp(dist.irecv, buf, q))
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()
    for ids, buf in recv:
        engine.scatter(ids, buf)


class GpuPart:
    """One part stepped by libue.so on the current CUDA device (plain variant, RCM order)."""

    def __init__(self, plan: Plan, p: int, dt: float, stream=None, precision=None, **build):
        import torch
        from . import api, _native as N
        self.p = p
        self.stream = stream
        self.m = api.Mesh(plan.local_xy(p), plan.local_tris(p))
        prec = N.UE_PREC_FP32 if precision is None else precision
        self.m.geometry_build(stream=stream, dt_mode=N.UE_DT_GIVEN, dt=dt, precision=prec, **build)
        self.dtype = torch.float64 if prec == N.UE_PREC_FP64 else torch.float32
        self._ids = {}

    def _dev_ids(self, ids):
        import torch
        key = (ids.ctypes.data, ids.size)
        t = self._ids.get(key)
        if t is None:
            t = torch.from_numpy(np.ascontiguousarray(ids, np.int32)).cuda()
            self._ids[key] = t
        return t

    def gather(self, ids):
        import torch
        buf = torch.empty(ids.size, dtype=self.dtype, device="cuda")
        self.m.exchange_tris(self._dev_ids(ids), buf, scatter=False, stream=self.stream)
        return buf

    def scatter(self, ids, buf):
        self.m.exchange_tris(self._dev_ids(ids), buf, scatter=True, stream=self.stream)

    def step(self, n: int = 1):
        self.m.step_n(n, self.stream)

    def close(self):
        self.m.close()


def run(engines, plan: Plan, n_steps: int, exchange=None):
    """n_steps leap-frog steps of every part, each followed by the halo exchange."""
    for _ in range(n_steps):
        for e in engines:
            e.step(1)
        (exchange or exchange_local)(engines, plan)
