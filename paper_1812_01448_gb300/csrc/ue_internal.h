// Internal definitions shared by the library's translation units (not part of the ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ue.h"

namespace ue {

// Host-side connectivity in the stored (reordered) numbering.  Built once by ue_mesh_load.
struct HostMesh {
    int64_t n_nodes = 0, n_tris = 0, n_edges = 0, n_ei = 0;
    std::vector<double> xy;             // 2*n_nodes, caller numbering
    std::vector<int64_t> edges;         // 2*n_edges (low, high) caller node ids, caller edge order
    std::vector<int64_t> perm_tri;      // stored triangle -> caller triangle
    std::vector<int64_t> edge_caller;   // stored interior edge -> caller edge
    std::vector<int64_t> k_of_edge;     // caller edge -> stored interior edge or -1
    std::vector<int32_t> edge_tri;      // 2*n_ei: (R, L) stored triangle ids
    std::vector<int32_t> tri_code;      // 3*n_tris: 2*k + neg (k = n_ei for a boundary edge)
    std::vector<int32_t> tri_nodes;     // 3*n_tris: caller node ids, rotated, CCW
    std::vector<int32_t> edge_nodes;    // 2*n_ei: (low, high) caller node ids
    std::vector<int32_t> edge_opp;      // 2*n_ei: node opposite the edge in R, in L
    std::vector<int64_t> tile_tri_off;  // KD order: n_tiles+1 stored-triangle offsets
};

// Temporal-blocking tiles: for each KD tile, its owned triangles and edges plus the rings of
// edge-neighbours needed to advance them k_max steps without communication.
struct TileSet {
    int k_max = 0;
    int64_t n_tiles = 0;
    int max_tri_loc = 0, max_edge_loc = 0, max_src = 0;
    static constexpr int kHdr = 48;       // ints per tile header
    std::vector<int32_t> hdr;             // n_tiles * kHdr (layout in kernels_tb.cu)
    std::vector<int32_t> trec;            // 4 ints per local triangle: gid, codes01, code2, 0
    std::vector<int32_t> erec;            // 4 ints per local edge: gid, R|L<<16, 0, 0; each
                                          // tile's records start at a multiple of 4 records
    std::vector<int64_t> erec_tile;       // per local edge record: its tile (for sources)
    // records of the fused kernel (build_fused_records; header 11 and 12 hold each tile's
    // offsets, in records): per local triangle 5 ints, each tile's block a multiple of 4
    // records; per local edge and the tile's zero slot 2 ints {gid, 0}, a multiple of 2
    std::vector<int32_t> frec, fedge;
};

// Records of the fused triangle-centric kernel from a built tile set (layout in kernels_tbf.cu).
// Fails (UE_ERR_ARG) when a tile is too large for them (4096 local triangles, 8191 edges).
int build_fused_records(const HostMesh& hm, TileSet& ts, std::string& err);

// include (may be NULL): build only the tiles t with (*include)[t] != 0, in order.
int build_tiles(const HostMesh& hm, int k_max, TileSet& ts, std::string& err,
                const std::vector<char>* include = nullptr);

// A region advanced k steps at once by the plain kernels on local copies: its owned triangles
// and the rings of edge-neighbours H_1..H_k around them, laid out like a tile (owned first,
// then by level; owned edges first).  Codes of triangles of level <= k-1 point at local edges,
// or, for the mesh's outer edges listed in islot (3 * stored triangle + q), at slot
// u_off + i with sign bit ineg[i], u_off = (nel + 4) / 4 * 4 the padded local edge count;
// level-k triangles (read only) and other boundary edges point at the zero slot nel.
struct Region {
    std::vector<int64_t> tgid, egid;   // stored ids of the local triangles / edges
    int64_t n_own_t = 0, n_own_e = 0;
    std::vector<int32_t> rl;           // 2 per local edge: local (R, L)
    std::vector<int32_t> code;         // 3 per local triangle
    std::vector<char> upd;             // local triangle updated (level <= k-1)
    std::vector<int32_t> tloc;         // stored triangle -> local index, or -1
};
int build_region(const HostMesh& hm, const std::vector<char>& owned, int k, const std::vector<int64_t>& islot,
                 const std::vector<int32_t>& ineg, Region& r, std::string& err);

// Returns UE_OK or an error code with a message in err.
int build_host_mesh(const double* xy, int64_t n_nodes, const int32_t* tris, int64_t n_tris,
                    int reorder, int tile_tris, HostMesh& hm, std::string& err);

// Constrained Delaunay triangulation of a node cloud (ue_triangulate); out: 3 ids per triangle.
int triangulate(const double* xy, int64_t nn, const int32_t* segs, int64_t n_segs, const double* holes,
                int64_t n_holes, int flags, std::vector<int32_t>& out, int64_t* n_flips, std::string& err);

}  // namespace ue
