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
    std::vector<int32_t> erec;            // 4 ints per local edge: gid, R|L<<16, 0, 0
    std::vector<int64_t> erec_tile;       // per local edge record: its tile (for sources)
};

int build_tiles(const HostMesh& hm, int k_max, TileSet& ts, std::string& err);

// Returns UE_OK or an error code with a message in err.
int build_host_mesh(const double* xy, int64_t n_nodes, const int32_t* tris, int64_t n_tris,
                    int reorder, int tile_tris, HostMesh& hm, std::string& err);

}  // namespace ue
