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
#include <algorithm>
#include <string>
#include <vector>

#include "ue_internal.h"

namespace ue {

int build_tiles(const HostMesh& hm, int k_max, TileSet& ts, std::string& err) {
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
    for (int64_t t = 0; t < ntiles; ++t) {
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
        int32_t* h = &ts.hdr[t * TileSet::kHdr];
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
            ts.erec_tile.push_back(t);
        }
        ts.max_tri_loc = std::max<int>(ts.max_tri_loc, (int)ntl);
        ts.max_edge_loc = std::max<int>(ts.max_edge_loc, (int)nel);
        for (int64_t j : tris) lvl[j] = loc[j] = -1;
        for (int64_t k : edges) elvl[k] = eloc[k] = -1;
    }
    return UE_OK;
}

}  // namespace ue
