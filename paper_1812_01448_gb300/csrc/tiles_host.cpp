// Host construction of the temporal-blocking tiles.
//
// A KD tile (a part of the paper's KD partition, "Divide and conqueror") owns a contiguous
// range of stored triangles and the interior edges whose smaller stored triangle it owns
// (also contiguous, since edges are numbered by (min, max) triangle).  Advancing the owned
// values k steps needs the rings of edge-neighbours H_0 = owned, H_{r+1} = H_r + neighbours(H_r)
// up to r = k: step s (1..k) updates the edges of H_{k-s} and the triangles of H_{k-s}.
// Locals are sorted by ring level (owned triangles first; owned edges first), so that "level
// <= lim" is an index bound.  Header layout (ints):
//   0 first owned triangle, 1 owned triangles, 2 first owned edge, 3 owned edges,
//   4 local triangles, 5 local edges, 6 triangle-record offset, 7 edge-record offset,
//   8 source-record offset, 9 source records, 10 k_max,
//   16 + r: local triangles of level <= r, 32 + r: local edges of level <= r  (r <= 15).
// Edge records of a tile start at a multiple of 4 records (padding records follow its last).
#include <algorithm>
#include <string>
#include <vector>

#include "ue_internal.h"

namespace ue {

int build_tiles(const HostMesh& hm, int k_max, TileSet& ts, std::string& err,
                const std::vector<char>* include) {
    if (hm.tile_tri_off.size() < 2) {
        err = "blocked variant needs a mesh loaded with UE_REORDER_KD";
        return UE_ERR_ARG;
    }
    if (k_max < 1 || k_max > 15) {
        err = "block_depth must be in 1..15";
        return UE_ERR_ARG;
    }
    const int64_t nt = hm.n_tris, nei = hm.n_ei;
    const int64_t ntiles = (int64_t)hm.tile_tri_off.size() - 1;
    ts = TileSet();
    ts.k_max = k_max;
    ts.n_tiles = ntiles;
    ts.hdr.assign(ntiles * TileSet::kHdr, 0);
    // owned edge ranges: edge k belongs to the tile of min(R, L)
    std::vector<int64_t> tile_of(nt);
    for (int64_t t = 0; t < ntiles; ++t)
        for (int64_t j = hm.tile_tri_off[t]; j < hm.tile_tri_off[t + 1]; ++j) tile_of[j] = t;
    std::vector<int64_t> edge_off(ntiles + 1, 0);
    for (int64_t k = 0; k < nei; ++k) {
        const int64_t lo = std::min(hm.edge_tri[2 * k], hm.edge_tri[2 * k + 1]);
        edge_off[tile_of[lo] + 1]++;
    }
    for (int64_t t = 0; t < ntiles; ++t) edge_off[t + 1] += edge_off[t];

    std::vector<int32_t> lvl(nt, -1), loc(nt, -1);
    std::vector<int32_t> elvl(nei, -1), eloc(nei, -1);
    std::vector<int64_t> tris, edges;
    std::vector<std::vector<int64_t>> ring(k_max + 1);
    int64_t out = 0;   // index of the tile in the set (tiles left out by `include` are skipped)
    for (int64_t t = 0; t < ntiles; ++t) {
        if (include && !(*include)[t]) continue;
        const int64_t a = hm.tile_tri_off[t], b = hm.tile_tri_off[t + 1];
        for (auto& r : ring) r.clear();
        for (int64_t j = a; j < b; ++j) {
            lvl[j] = 0;
            ring[0].push_back(j);
        }
        for (int r = 1; r <= k_max; ++r) {
            for (int64_t j : ring[r - 1])
                for (int q = 0; q < 3; ++q) {
                    const int64_t k = hm.tri_code[3 * j + q] >> 1;
                    if (k >= nei) continue;
                    const int64_t o = hm.edge_tri[2 * k] == j ? hm.edge_tri[2 * k + 1] : hm.edge_tri[2 * k];
                    if (lvl[o] < 0) {
                        lvl[o] = r;
                        ring[r].push_back(o);
                    }
                }
            std::sort(ring[r].begin(), ring[r].end());
        }
        tris.clear();
        for (int r = 0; r <= k_max; ++r) tris.insert(tris.end(), ring[r].begin(), ring[r].end());
        for (size_t l = 0; l < tris.size(); ++l) loc[tris[l]] = (int32_t)l;
        // edges of H_{k_max-1}, level = min level of their two triangles
        edges.clear();
        for (int64_t j : tris) {
            if (lvl[j] > k_max - 1) continue;
            for (int q = 0; q < 3; ++q) {
                const int64_t k = hm.tri_code[3 * j + q] >> 1;
                if (k >= nei || elvl[k] >= 0) continue;
                elvl[k] = std::min(lvl[hm.edge_tri[2 * k]], lvl[hm.edge_tri[2 * k + 1]]);
                edges.push_back(k);
            }
        }
        const int64_t ea = edge_off[t], eb = edge_off[t + 1];
        std::sort(edges.begin(), edges.end(), [&](int64_t u, int64_t v) {
            const bool ou = u >= ea && u < eb, ov = v >= ea && v < eb;
            if (elvl[u] != elvl[v]) return elvl[u] < elvl[v];
            if (ou != ov) return ou;
            return u < v;
        });
        for (size_t l = 0; l < edges.size(); ++l) eloc[edges[l]] = (int32_t)l;
        const int64_t ntl = (int64_t)tris.size(), nel = (int64_t)edges.size();
        if (nel >= 32767 || ntl >= 65535) {
            err = "a tile with its halo exceeds 65535 triangles or 32767 edges: lower tile_tris or block_depth";
            for (int64_t j : tris) lvl[j] = loc[j] = -1;
            for (int64_t k : edges) elvl[k] = eloc[k] = -1;
            return UE_ERR_ARG;
        }
        int32_t* h = &ts.hdr[out * TileSet::kHdr];
        h[0] = (int32_t)a;
        h[1] = (int32_t)(b - a);
        h[2] = (int32_t)ea;
        h[3] = (int32_t)(eb - ea);
        h[4] = (int32_t)ntl;
        h[5] = (int32_t)nel;
        h[6] = (int32_t)(ts.trec.size() / 4);
        h[7] = (int32_t)(ts.erec.size() / 4);
        h[10] = k_max;
        for (int r = 0; r < 16; ++r) {
            int32_t ct = 0, ce = 0;
            for (int64_t j : tris) ct += lvl[j] <= r;
            for (int64_t k : edges) ce += elvl[k] <= r;
            h[16 + r] = ct;
            h[32 + r] = ce;
        }
        // the owned edges must be exactly the first h[3] local edges
        for (int64_t l = 0; l < eb - ea; ++l)
            if (edges[l] != ea + l) {
                err = "internal error: owned edges are not contiguous";
                return UE_ERR_ARG;
            }
        for (int64_t j : tris) {
            int32_t c[3] = {0, 0, 0};
            if (lvl[j] <= k_max - 1)
                for (int q = 0; q < 3; ++q) {
                    const int32_t code = hm.tri_code[3 * j + q];
                    const int64_t k = code >> 1;
                    c[q] = k >= nei ? (int32_t)(nel << 1) : (int32_t)((eloc[k] << 1) | (code & 1));
                }
            ts.trec.push_back((int32_t)j);
            ts.trec.push_back((c[0] & 0xFFFF) | (c[1] << 16));
            ts.trec.push_back(c[2]);
            ts.trec.push_back(0);
        }
        for (int64_t k : edges) {
            ts.erec.push_back((int32_t)k);
            ts.erec.push_back(loc[hm.edge_tri[2 * k]] | (loc[hm.edge_tri[2 * k + 1]] << 16));
            ts.erec.push_back(0);
            ts.erec.push_back(0);
            ts.erec_tile.push_back(out);
        }
        // each tile's edge records start at a multiple of 4 (padding records: gid 0, R = L = 0),
        // so that the blocked kernel's bulk copies of 12-byte records stay 16-byte aligned
        while ((ts.erec.size() / 4) % 4 != 0) {
            ts.erec.insert(ts.erec.end(), {0, 0, 0, 0});
            ts.erec_tile.push_back(out);
        }
        ts.max_tri_loc = std::max<int>(ts.max_tri_loc, (int)ntl);
        ts.max_edge_loc = std::max<int>(ts.max_edge_loc, (int)nel);
        for (int64_t j : tris) lvl[j] = loc[j] = -1;
        for (int64_t k : edges) elvl[k] = eloc[k] = -1;
        ++out;
    }
    ts.n_tiles = out;
    ts.hdr.resize(out * TileSet::kHdr);
    return UE_OK;
}

// Fused records: local triangle l of a tile (levels <= k_max - 1; the outermost ring only
// needs its gid) with local edge codes c_q = 2 e_q + (s_q < 0) (e_q = nel: boundary); edge
// records {gid, 0}, then {-1, 0} for the zero slot (and padding):
//   r0 gid;
//   r1 bits 0-15: 4 * local id of the triangle across edge 0 (itself on the boundary),
//      16-31: the same for edge 1;
//   r2 bits 0-13: 4 * the neighbour across edge 2, 14-26: e_0, 27 / 28: s0 s1 < 0, s0 s2 < 0,
//      29: s0 < 0;
//   r3 bits 0-12: e_1, 16-28: e_2, bit 13 / 14 / 29: sign of the signed edge coefficient of
//      edge 0 / 1 / 2 (see below);
//   r4 bits of -s0 dt/S (filled on the device).
// The signed edge coefficient is s0 s_q t_q dt|e|/d, t_q = +1 when the triangle is R of the
// edge, -1 when it is L; with the edge values held as V_q = s0 s_q U_q it advances V_q by
// fma(coefficient, B_own - B_nbr, V_q), which rounds exactly as U += (dt|e|/d)(B_R - B_L).
int build_fused_records(const HostMesh& hm, TileSet& ts, std::string& err) {
    ts.frec.clear();
    ts.fedge.clear();
    (void)hm;
    for (int64_t t = 0; t < ts.n_tiles; ++t) {
        int32_t* h = &ts.hdr[t * TileSet::kHdr];
        const int ntl = h[4], nel = h[5], k = h[10];
        if (ntl > 4096 || nel + 1 > 8191) {
            err = "a tile with its halo is too large for the fused records (4096 triangles, 8190 edges)";
            return UE_ERR_ARG;
        }
        const int32_t* tr = &ts.trec[4 * (size_t)h[6]];
        const int32_t* er = &ts.erec[4 * (size_t)h[7]];
        h[11] = (int32_t)(ts.frec.size() / 5);
        h[12] = (int32_t)(ts.fedge.size() / 2);
        const int nupd = h[16 + k - 1];
        for (int l = 0; l < ntl; ++l) {
            int32_t r[5] = {tr[4 * l], 0, 0, 0, 0};
            if (l < nupd) {
                const uint32_t code[3] = {(uint32_t)tr[4 * l + 1] & 0xFFFFu, (uint32_t)tr[4 * l + 1] >> 16,
                                          (uint32_t)tr[4 * l + 2]};
                uint32_t nb[3], e[3], csign[3];
                const uint32_t s0 = code[0] & 1u;
                for (int q = 0; q < 3; ++q) {
                    e[q] = code[q] >> 1;
                    if ((int)e[q] >= nel) {          // boundary edge: coefficient 0, itself
                        nb[q] = (uint32_t)l;
                        csign[q] = 0;
                        e[q] = (uint32_t)nel;
                        continue;
                    }
                    const uint32_t R = (uint32_t)er[4 * e[q] + 1] & 0xFFFFu, L = (uint32_t)er[4 * e[q] + 1] >> 16;
                    if (R != (uint32_t)l && L != (uint32_t)l) {
                        err = "internal error: a triangle's edge does not name it";
                        return UE_ERR_ARG;
                    }
                    nb[q] = R == (uint32_t)l ? L : R;
                    const uint32_t neg_t = R == (uint32_t)l ? 0u : 1u;
                    csign[q] = (s0 ^ (code[q] & 1u)) ^ neg_t;
                }
                r[1] = (int32_t)((4u * nb[0]) | ((4u * nb[1]) << 16));
                r[2] = (int32_t)((4u * nb[2]) | (e[0] << 14) | (((code[1] ^ code[0]) & 1u) << 27) |
                                 (((code[2] ^ code[0]) & 1u) << 28) | (s0 << 29));
                r[3] = (int32_t)(e[1] | (csign[0] << 13) | (csign[1] << 14) | (e[2] << 16) | (csign[2] << 29));
            }
            ts.frec.insert(ts.frec.end(), r, r + 5);
        }
        while ((ts.frec.size() / 5) % 4 != 0) ts.frec.insert(ts.frec.end(), {0, 0, 0, 0, 0});
        for (int l = 0; l < nel; ++l) ts.fedge.insert(ts.fedge.end(), {er[4 * l], 0});
        ts.fedge.insert(ts.fedge.end(), {-1, 0});          // the zero slot
        if ((ts.fedge.size() / 2) % 2 != 0) ts.fedge.insert(ts.fedge.end(), {-1, 0});
    }
    return UE_OK;
}

int build_region(const HostMesh& hm, const std::vector<char>& owned, int k, const std::vector<int64_t>& islot,
                 const std::vector<int32_t>& ineg, Region& r, std::string& err) {
    const int64_t nt = hm.n_tris, nei = hm.n_ei;
    r = Region();
    std::vector<int32_t> lvl(nt, -1);
    std::vector<std::vector<int64_t>> ring(k + 1);
    for (int64_t j = 0; j < nt; ++j)
        if (owned[j]) {
            lvl[j] = 0;
            ring[0].push_back(j);
        }
    for (int q = 1; q <= k; ++q) {
        for (int64_t j : ring[q - 1])
            for (int c = 0; c < 3; ++c) {
                const int64_t e = hm.tri_code[3 * j + c] >> 1;
                if (e >= nei) continue;
                const int64_t o = hm.edge_tri[2 * e] == j ? hm.edge_tri[2 * e + 1] : hm.edge_tri[2 * e];
                if (lvl[o] < 0) {
                    lvl[o] = q;
                    ring[q].push_back(o);
                }
            }
        std::sort(ring[q].begin(), ring[q].end());
    }
    for (int q = 0; q <= k; ++q) r.tgid.insert(r.tgid.end(), ring[q].begin(), ring[q].end());
    r.n_own_t = (int64_t)ring[0].size();
    std::vector<int32_t> loc(nt, -1);
    for (size_t l = 0; l < r.tgid.size(); ++l) loc[r.tgid[l]] = (int32_t)l;
    // edges with a triangle of level <= k-1, owned ones first (an edge belongs to its smaller
    // stored triangle), then by level and id
    std::vector<int32_t> elvl(nei, -1);
    std::vector<int64_t> edges;
    for (int64_t j : r.tgid) {
        if (lvl[j] > k - 1) continue;
        for (int c = 0; c < 3; ++c) {
            const int64_t e = hm.tri_code[3 * j + c] >> 1;
            if (e >= nei || elvl[e] >= 0) continue;
            elvl[e] = std::min(lvl[hm.edge_tri[2 * e]], lvl[hm.edge_tri[2 * e + 1]]);
            edges.push_back(e);
        }
    }
    auto own_e = [&](int64_t e) { return (bool)owned[std::min(hm.edge_tri[2 * e], hm.edge_tri[2 * e + 1])]; };
    std::sort(edges.begin(), edges.end(), [&](int64_t u, int64_t v) {
        const bool ou = own_e(u), ov = own_e(v);
        if (ou != ov) return ou;
        if (elvl[u] != elvl[v]) return elvl[u] < elvl[v];
        return u < v;
    });
    r.n_own_e = 0;
    for (int64_t e : edges) r.n_own_e += own_e(e);
    const int64_t nel = (int64_t)edges.size();
    std::vector<int32_t> eloc(nei, -1);
    for (size_t l = 0; l < edges.size(); ++l) eloc[edges[l]] = (int32_t)l;
    r.egid.assign(edges.begin(), edges.end());
    r.rl.resize(2 * nel);
    for (int64_t l = 0; l < nel; ++l) {
        r.rl[2 * l] = loc[hm.edge_tri[2 * edges[l]]];
        r.rl[2 * l + 1] = loc[hm.edge_tri[2 * edges[l] + 1]];
        if (r.rl[2 * l] < 0 || r.rl[2 * l + 1] < 0) {
            err = "internal error: a region edge has a triangle outside the region";
            return UE_ERR_ARG;
        }
    }
    // triangle codes: local edges; the mesh's outer edges at the interface slots after the
    // region's zero slot; triangles of level k (read only) on the zero slot
    const int64_t u_off = (nel + 4) / 4 * 4;   // the padded local edge count
    std::vector<int64_t> if_of(3 * nt, -1);
    for (size_t i = 0; i < islot.size(); ++i) if_of[islot[i]] = (int64_t)i;
    r.code.assign(3 * r.tgid.size(), (int32_t)(2 * nel));
    r.upd.assign(r.tgid.size(), 0);
    for (size_t l = 0; l < r.tgid.size(); ++l) {
        const int64_t j = r.tgid[l];
        if (lvl[j] > k - 1) continue;
        r.upd[l] = 1;
        for (int c = 0; c < 3; ++c) {
            const int32_t code = hm.tri_code[3 * j + c];
            const int64_t e = code >> 1;
            if (e < nei) {
                r.code[3 * l + c] = (int32_t)((eloc[e] << 1) | (code & 1));
            } else if (if_of[3 * j + c] >= 0) {
                const int64_t i = if_of[3 * j + c];
                r.code[3 * l + c] = (int32_t)(2 * (u_off + i) + ineg[i]);
            }
        }
    }
    r.tloc.assign(loc.begin(), loc.end());
    return UE_OK;
}

}  // namespace ue
