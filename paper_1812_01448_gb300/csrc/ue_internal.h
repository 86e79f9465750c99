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
};

// Returns UE_OK or an error code with a message in err.
int build_host_mesh(const double* xy, int64_t n_nodes, const int32_t* tris, int64_t n_tris,
                    int reorder, HostMesh& hm, std::string& err);

}  // namespace ue
