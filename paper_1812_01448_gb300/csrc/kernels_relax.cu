// Mesh optimisation by the jello model with flip refinement (Section 3, "Mesh generation").
//
// Nodes joined by springs along the triangle edges and along the heights relax, strongly
// damped (first order, Euler), towards near-equilateral triangles of a given size; the nodes of
// the input geometry (the boundary) stay.  Every few steps the triangulation is refreshed by
// Lawson flips, because deformed triangles stop the relaxation around them.
// Model: unit springs, so the force is -grad E with
//   E = sum_edges (|ab| - L0)^2 / 2 + sum_heights (|v - m| - H0)^2 / 2,
// a height spring joining vertex v to the midpoint m of its opposite edge; L0 = (h_a + h_b)/2,
// H0 = sqrt(3)/2 times the mean L0 of the triangle's edges.  One step: x += tau F, the
// displacement clamped to 0.1 of the node's shortest rest edge and to 0.15 of the smallest
// height h of its triangles: moves of at most d per vertex change twice a triangle's area by at
// most 3 d L + 4 d^2 <= 0.54 h L (L its longest edge), less than the h L it has, so no triangle
// turns over.
// GPU, FP64, positions double-buffered: per step one thread per triangle evaluates its three
// height springs and its cap once, then one thread per node gathers its edge springs and its
// triangles' shares (node -> edge and node -> triangle lists).
// Host: the lists, and the flips (a flip changes the lists).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <unordered_set>
#include <utility>
#include <vector>

#include "device.cuh"

namespace ue {

namespace {

constexpr int kRxThreads = 256;

// adjacency of one triangulation, as uploaded
struct RxLists {
    std::vector<int32_t> e_off, e_nb;     // node -> (neighbour node) of each incident edge
    std::vector<double> e_L0;             // rest length of that edge
    std::vector<int32_t> t_off, t_tri;    // node -> incident triangle
    std::vector<int32_t> t_loc;           // local index of the node in it (0..2)
    std::vector<double> H0;               // rest height per triangle
    std::vector<double> cap;              // displacement cap per node
    std::vector<uint8_t> fixed;           // boundary node
};

// Per triangle, once per step: the three height springs' pulls on its vertices and the cap
// 0.15 * (2 area / longest edge).  Spring q (apex q over the edge (q+1, q+2)) with
// g_q = ((|w| - H0) / |w|) w, w = x_q - (x_{q+1} + x_{q+2}) / 2, pulls the apex by -g_q and each
// end of its edge by g_q / 2, so vertex j takes -g_j + (g_{j+1} + g_{j+2}) / 2.
// out: 8 doubles per triangle {F_0, F_1, F_2 (x, y each), cap, 0}.
__global__ void k_rx_tri(const double* __restrict__ x, const int32_t* __restrict__ tris,
                         const double* __restrict__ H0, double* __restrict__ out, int64_t n_tris) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tris) return;
    double px[3], py[3];
    for (int q = 0; q < 3; ++q) {
        const int32_t n = tris[3 * t + q];
        px[q] = x[2 * n];
        py[q] = x[2 * n + 1];
    }
    const double a2 = fabs((px[1] - px[0]) * (py[2] - py[0]) - (py[1] - py[0]) * (px[2] - px[0]));
    double lm = 0.0;
    for (int q = 0; q < 3; ++q) {
        const int p = q == 2 ? 0 : q + 1;
        const double ex = px[p] - px[q], ey = py[p] - py[q];
        lm = fmax(lm, sqrt(ex * ex + ey * ey));
    }
    const double h0 = H0[t];
    double gx[3], gy[3];
    for (int q = 0; q < 3; ++q) {
        const int p = q == 2 ? 0 : q + 1, r = q == 0 ? 2 : q - 1;
        const double wx = px[q] - 0.5 * (px[p] + px[r]), wy = py[q] - 0.5 * (py[p] + py[r]);
        const double hm = sqrt(wx * wx + wy * wy);
        const double sc = (hm - h0) / hm;
        gx[q] = sc * wx;
        gy[q] = sc * wy;
    }
    double* o = out + 8 * t;
    for (int j = 0; j < 3; ++j) {
        const int p = j == 2 ? 0 : j + 1, r = j == 0 ? 2 : j - 1;
        o[2 * j] = 0.5 * (gx[p] + gx[r]) - gx[j];
        o[2 * j + 1] = 0.5 * (gy[p] + gy[r]) - gy[j];
    }
    o[6] = 0.15 * (a2 / lm);
    o[7] = 0.0;
}

// Per node: its edge springs, its shares of its triangles' height springs, the smallest cap;
// then the capped Euler step (fixed nodes copy through).
__global__ void k_rx_node(const double* __restrict__ x, double* __restrict__ xn,
                          const int32_t* __restrict__ e_off, const int32_t* __restrict__ e_nb,
                          const double* __restrict__ e_L0, const int32_t* __restrict__ t_off,
                          const int32_t* __restrict__ t_tri, const int32_t* __restrict__ t_loc,
                          const double* __restrict__ tri_out, const double* __restrict__ cap,
                          const uint8_t* __restrict__ fixed, double tau, int64_t n_nodes) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_nodes) return;
    const double vx = x[2 * v], vy = x[2 * v + 1];
    if (fixed[v]) {
        xn[2 * v] = vx;
        xn[2 * v + 1] = vy;
        return;
    }
    double fx = 0.0, fy = 0.0;
    for (int32_t i = e_off[v]; i < e_off[v + 1]; ++i) {   // edge springs
        const int32_t b = e_nb[i];
        const double dx = x[2 * b] - vx, dy = x[2 * b + 1] - vy;
        const double L = sqrt(dx * dx + dy * dy);
        const double s = (L - e_L0[i]) / L;
        fx += s * dx;
        fy += s * dy;
    }
    double c = cap[v];
    for (int32_t i = t_off[v]; i < t_off[v + 1]; ++i) {   // its triangles' height springs
        const double* o = tri_out + 8 * (int64_t)t_tri[i];
        const int l = t_loc[i];
        fx += o[2 * l];
        fy += o[2 * l + 1];
        c = fmin(c, o[6]);
    }
    double dx = tau * fx, dy = tau * fy;
    const double n = sqrt(dx * dx + dy * dy);
    if (n > c) {
        const double k = c / n;
        dx *= k;
        dy *= k;
    }
    xn[2 * v] = vx + dx;
    xn[2 * v + 1] = vy + dy;
}

double orient2d(const std::vector<double>& x, int a, int b, int c) {
    return (x[2 * b] - x[2 * a]) * (x[2 * c + 1] - x[2 * a + 1]) -
           (x[2 * b + 1] - x[2 * a + 1]) * (x[2 * c] - x[2 * a]);
}

// d strictly inside the circumcircle of the CCW triangle abc, beyond a relative 1e-10 margin
bool in_circle(const std::vector<double>& x, int a, int b, int c, int d) {
    const double ax = x[2 * a] - x[2 * d], ay = x[2 * a + 1] - x[2 * d + 1];
    const double bx = x[2 * b] - x[2 * d], by = x[2 * b + 1] - x[2 * d + 1];
    const double cx = x[2 * c] - x[2 * d], cy = x[2 * c + 1] - x[2 * d + 1];
    const double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
    const double det = a2 * (bx * cy - by * cx) - b2 * (ax * cy - ay * cx) + c2 * (ax * by - ay * bx);
    const double s = std::max(a2, std::max(b2, c2));
    return det > 1e-10 * s * s;
}

// Lawson flips until every interior edge is locally Delaunay; returns the number of flips.
// nb[3 i + q] is the triangle across edge q = (t[q], t[q+1]) of triangle i (-1 on the boundary).
// The stack holds (triangle, a, b) for a directed CCW edge a->b; an entry whose triangle no longer
// holds that edge is stale and skipped: every flip pushes its four outer edges with their current
// triangles, so no live edge is lost.
// node -> incident triangles (CSR by counting), in triangle order
void node_tris(int64_t nn, const std::vector<int32_t>& t, std::vector<int32_t>& off,
               std::vector<int32_t>& tri, std::vector<int32_t>* loc) {
    const int64_t nt = (int64_t)t.size() / 3;
    off.assign(nn + 1, 0);
    for (int32_t n : t) ++off[n + 1];
    for (int64_t v = 0; v < nn; ++v) off[v + 1] += off[v];
    tri.assign(off[nn], 0);
    if (loc) loc->assign(off[nn], 0);
    std::vector<int32_t> p(off.begin(), off.end() - 1);
    for (int64_t i = 0; i < nt; ++i)
        for (int q = 0; q < 3; ++q) {
            const int32_t n = t[3 * i + q];
            if (loc) (*loc)[p[n]] = q;
            tri[p[n]++] = (int32_t)i;
        }
}

uint64_t edge_key(int32_t a, int32_t b) {
    return ((uint64_t)(uint32_t)std::min(a, b) << 32) | (uint32_t)std::max(a, b);
}

// keep: edges (edge_key) that are never flipped (the input geometry's).
int64_t lawson(const std::vector<double>& x, std::vector<int32_t>& t, const std::unordered_set<uint64_t>& keep) {
    const int64_t nt = (int64_t)t.size() / 3;
    const int64_t nn = (int64_t)x.size() / 2;
    std::vector<int64_t> nb(3 * nt, -1);
    {   // the twin of a -> b in triangle i is b -> a in one of b's other triangles
        std::vector<int32_t> off, tri;
        node_tris(nn, t, off, tri, nullptr);
        for (int64_t i = 0; i < nt; ++i)
            for (int q = 0; q < 3; ++q) {
                if (nb[3 * i + q] >= 0) continue;   // found from the other side
                const int32_t a = t[3 * i + q], b = t[3 * i + (q + 1) % 3];
                for (int32_t k = off[b]; k < off[b + 1] && nb[3 * i + q] < 0; ++k) {
                    const int32_t j = tri[k];
                    if (j == i) continue;
                    for (int r = 0; r < 3; ++r)
                        if (t[3 * j + r] == b && t[3 * j + (r + 1) % 3] == a) {
                            nb[3 * i + q] = j;
                            nb[3 * j + r] = i;
                            break;
                        }
                }
            }
    }
    struct Item { int64_t tri; int32_t a, b; };
    std::vector<Item> stack;
    stack.reserve(3 * nt);
    for (int64_t s = 3 * nt - 1; s >= 0; --s)
        if (nb[s] > s / 3) stack.push_back({s / 3, t[s], t[3 * (s / 3) + (s % 3 + 1) % 3]});
    auto slot_of = [&](int64_t i, int32_t a, int32_t b) -> int {
        for (int q = 0; q < 3; ++q)
            if (t[3 * i + q] == a && t[3 * i + (q + 1) % 3] == b) return q;
        return -1;
    };
    int64_t flips = 0;
    while (!stack.empty()) {
        const Item it = stack.back();
        stack.pop_back();
        const int64_t i = it.tri;
        const int qi = slot_of(i, it.a, it.b);
        if (qi < 0) continue;                       // stale: the edge left this triangle
        const int64_t j = nb[3 * i + qi];
        if (j < 0) continue;
        const int32_t a = it.a, b = it.b, c = t[3 * i + (qi + 2) % 3];
        if (!keep.empty() && keep.count(edge_key(a, b))) continue;
        const int qj = slot_of(j, b, a);
        const int32_t d = t[3 * j + (qj + 2) % 3];
        if (!in_circle(x, a, b, c, d)) continue;
        if (orient2d(x, a, d, c) <= 0 || orient2d(x, d, b, c) <= 0) continue;   // not convex
        const int64_t X_bc = nb[3 * i + (qi + 1) % 3], X_ca = nb[3 * i + (qi + 2) % 3];
        const int64_t X_ad = nb[3 * j + (qj + 1) % 3], X_db = nb[3 * j + (qj + 2) % 3];
        // new i = (a, d, c), new j = (d, b, c)
        t[3 * i] = a; t[3 * i + 1] = d; t[3 * i + 2] = c;
        t[3 * j] = d; t[3 * j + 1] = b; t[3 * j + 2] = c;
        nb[3 * i] = X_ad; nb[3 * i + 1] = j; nb[3 * i + 2] = X_ca;
        nb[3 * j] = X_db; nb[3 * j + 1] = X_bc; nb[3 * j + 2] = i;
        auto repoint = [&](int64_t X, int64_t from, int64_t to) {
            if (X < 0) return;
            for (int q = 0; q < 3; ++q)
                if (nb[3 * X + q] == from) { nb[3 * X + q] = to; return; }
        };
        repoint(X_ad, j, i);
        repoint(X_bc, i, j);
        ++flips;
        stack.push_back({i, a, d});
        stack.push_back({j, d, b});
        stack.push_back({j, b, c});
        stack.push_back({i, c, a});
    }
    return flips;
}

void build_lists(int64_t nn, const std::vector<int32_t>& t, const std::vector<double>& h, RxLists& L) {
    const int64_t nt = (int64_t)t.size() / 3;
    // node -> triangles (with the node's local index), in triangle order
    node_tris(nn, t, L.t_off, L.t_tri, &L.t_loc);
    L.H0.assign(nt, 0.0);
    for (int64_t i = 0; i < nt; ++i) {
        double s = 0.0;
        for (int q = 0; q < 3; ++q) s += 0.5 * (h[t[3 * i + q]] + h[t[3 * i + (q + 1) % 3]]);
        L.H0[i] = std::sqrt(3.0) / 2.0 * s / 3.0;
    }
    // node -> edges in increasing neighbour order (each triangle names each of its vertices'
    // two neighbours; an edge named once is on the boundary, its ends fixed)
    L.fixed.assign(nn, 0);
    L.e_off.assign(nn + 1, 0);
    L.e_nb.clear();
    L.e_L0.clear();
    L.cap.assign(nn, INFINITY);
    std::vector<int32_t> nbr;
    for (int64_t v = 0; v < nn; ++v) {
        nbr.clear();
        for (int32_t k = L.t_off[v]; k < L.t_off[v + 1]; ++k) {
            const int32_t i = L.t_tri[k], q = L.t_loc[k];
            nbr.push_back(t[3 * i + (q + 1) % 3]);
            nbr.push_back(t[3 * i + (q + 2) % 3]);
        }
        std::sort(nbr.begin(), nbr.end());
        for (size_t k = 0; k < nbr.size();) {
            size_t r = k + 1;
            while (r < nbr.size() && nbr[r] == nbr[k]) ++r;
            const int32_t b = nbr[k];
            if (r - k == 1) L.fixed[v] = L.fixed[b] = 1;
            const double l0 = 0.5 * (h[v] + h[b]);
            L.e_nb.push_back(b);
            L.e_L0.push_back(l0);
            L.cap[v] = std::min(L.cap[v], 0.1 * l0);
            k = r;
        }
        L.e_off[v + 1] = (int32_t)L.e_nb.size();
    }
}

}  // namespace

// See include/ue.h (ue_mesh_relax).  Device buffers are owned here (cudaMalloc/cudaFree):
// the call is a one-off preprocessing step outside any mesh.
namespace {

// Orients the triangles CCW in t (a copy of tris); accumulates the area.
int orient_input(const std::vector<double>& x, int64_t nn, std::vector<int32_t>& t, double* area,
                 std::string& err) {
    const int64_t nt = (int64_t)t.size() / 3;
    for (int64_t i = 0; i < nt; ++i) {
        int32_t* r = &t[3 * i];
        for (int q = 0; q < 3; ++q)
            if (r[q] < 0 || r[q] >= nn) {
                err = "triangle node index out of range";
                return UE_ERR_ARG;
            }
        double o = orient2d(x, r[0], r[1], r[2]);
        if (o < 0) {
            std::swap(r[1], r[2]);
            o = -o;
        }
        if (!(o > 0)) {
            err = "degenerate triangle " + std::to_string(i);
            return UE_ERR_DEGENERATE;
        }
        *area += 0.5 * o;
    }
    return UE_OK;
}

int keep_set(const int32_t* segs, int64_t n_segs, int64_t nn, std::unordered_set<uint64_t>& keep,
             std::string& err) {
    for (int64_t k = 0; k < n_segs; ++k) {
        const int32_t a = segs[2 * k], b = segs[2 * k + 1];
        if (a < 0 || b < 0 || a >= nn || b >= nn || a == b) {
            err = "kept edge " + std::to_string(k) + " has a bad node id";
            return UE_ERR_ARG;
        }
        keep.insert(edge_key(a, b));
    }
    return UE_OK;
}

}  // namespace

// See include/ue.h (ue_mesh_flip): the remesh step alone, on the host.
int mesh_flip(const double* xy, int64_t nn, const int32_t* tris, int64_t nt, const int32_t* segs,
              int64_t n_segs, int32_t* tris_out, int64_t* n_flips, std::string& err) {
    std::vector<double> x(xy, xy + 2 * nn);
    std::vector<int32_t> t(tris, tris + 3 * nt);
    double area = 0.0;
    std::unordered_set<uint64_t> keep;
    int rc = orient_input(x, nn, t, &area, err);
    if (rc == UE_OK) rc = keep_set(segs, n_segs, nn, keep, err);
    if (rc != UE_OK) return rc;
    const int64_t k = lawson(x, t, keep);
    std::copy(t.begin(), t.end(), tris_out);
    if (n_flips) *n_flips = k;
    return UE_OK;
}

int mesh_relax(const double* xy, int64_t nn, const int32_t* tris, int64_t nt, const double* h_nodes,
               int32_t iters, int32_t flip_every, double tau, const int32_t* anchors, int64_t n_anchors,
               const int32_t* segs, int64_t n_segs, double* xy_out, int32_t* tris_out, int64_t* n_flips,
               cudaStream_t s, std::string& err) {
    std::vector<double> x(xy, xy + 2 * nn);
    std::vector<int32_t> t(tris, tris + 3 * nt);
    double area = 0.0;
    std::unordered_set<uint64_t> keep;
    {
        int rc = orient_input(x, nn, t, &area, err);
        if (rc == UE_OK) rc = keep_set(segs, n_segs, nn, keep, err);
        if (rc != UE_OK) return rc;
        for (int64_t k = 0; k < n_anchors; ++k)
            if (anchors[k] < 0 || anchors[k] >= nn) {
                err = "anchor " + std::to_string(k) + " is not a node id";
                return UE_ERR_ARG;
            }
    }
    std::vector<double> h(nn);
    if (h_nodes) {
        for (int64_t v = 0; v < nn; ++v) {
            if (!(h_nodes[v] > 0)) {
                err = "sizes must be positive";
                return UE_ERR_ARG;
            }
            h[v] = h_nodes[v];
        }
    } else {
        std::fill(h.begin(), h.end(), std::sqrt(4.0 * area / (std::sqrt(3.0) * (double)nt)));
    }
    RxLists L;
    // the boundary nodes are fixed by build_lists; the caller's anchors join them
    auto lists = [&]() {
        build_lists(nn, t, h, L);
        for (int64_t k = 0; k < n_anchors; ++k) L.fixed[anchors[k]] = 1;
    };
    lists();
    // device buffers, sized for the lists (their sizes do not change under flips)
    double *dx0 = nullptr, *dx1 = nullptr, *dL0 = nullptr, *dH0 = nullptr, *dcap = nullptr,
           *dtri = nullptr;
    int32_t *dt = nullptr, *deo = nullptr, *den = nullptr, *dto = nullptr, *dtt = nullptr, *dtl = nullptr;
    uint8_t* dfix = nullptr;
    const size_t ne2 = L.e_nb.size(), nt3 = L.t_tri.size();
    cudaError_t e = cudaSuccess;
    auto ck = [&](cudaError_t r) {
        if (e == cudaSuccess && r != cudaSuccess) e = r;
    };
    ck(cudaMalloc(&dx0, 16 * nn));
    ck(cudaMalloc(&dx1, 16 * nn));
    ck(cudaMalloc(&dt, 12 * nt));
    ck(cudaMalloc(&deo, 4 * (nn + 1)));
    ck(cudaMalloc(&den, 4 * ne2));
    ck(cudaMalloc(&dL0, 8 * ne2));
    ck(cudaMalloc(&dto, 4 * (nn + 1)));
    ck(cudaMalloc(&dtt, 4 * nt3));
    ck(cudaMalloc(&dtl, 4 * nt3));
    ck(cudaMalloc(&dH0, 8 * nt));
    ck(cudaMalloc(&dcap, 8 * nn));
    ck(cudaMalloc(&dfix, nn));
    ck(cudaMalloc(&dtri, 64 * nt));
    auto upload_lists = [&]() {
        ck(cudaMemcpyAsync(dt, t.data(), 12 * nt, cudaMemcpyHostToDevice, s));
        ck(cudaMemcpyAsync(deo, L.e_off.data(), 4 * (nn + 1), cudaMemcpyHostToDevice, s));
        ck(cudaMemcpyAsync(den, L.e_nb.data(), 4 * ne2, cudaMemcpyHostToDevice, s));
        ck(cudaMemcpyAsync(dL0, L.e_L0.data(), 8 * ne2, cudaMemcpyHostToDevice, s));
        ck(cudaMemcpyAsync(dto, L.t_off.data(), 4 * (nn + 1), cudaMemcpyHostToDevice, s));
        ck(cudaMemcpyAsync(dtt, L.t_tri.data(), 4 * nt3, cudaMemcpyHostToDevice, s));
        ck(cudaMemcpyAsync(dtl, L.t_loc.data(), 4 * nt3, cudaMemcpyHostToDevice, s));
        ck(cudaMemcpyAsync(dH0, L.H0.data(), 8 * nt, cudaMemcpyHostToDevice, s));
        ck(cudaMemcpyAsync(dcap, L.cap.data(), 8 * nn, cudaMemcpyHostToDevice, s));
        ck(cudaMemcpyAsync(dfix, L.fixed.data(), nn, cudaMemcpyHostToDevice, s));
        ck(cudaStreamSynchronize(s));   // the host lists may change after this
    };
    if (e == cudaSuccess) {
        ck(cudaMemcpyAsync(dx0, x.data(), 16 * nn, cudaMemcpyHostToDevice, s));
        upload_lists();
    }
    int64_t flips = 0;
    const unsigned grid = (unsigned)((nn + kRxThreads - 1) / kRxThreads);
    const unsigned grid_t = (unsigned)((nt + kRxThreads - 1) / kRxThreads);
    for (int32_t it = 0; it < iters && e == cudaSuccess; ++it) {
        k_rx_tri<<<grid_t, kRxThreads, 0, s>>>(dx0, dt, dH0, dtri, nt);
        k_rx_node<<<grid, kRxThreads, 0, s>>>(dx0, dx1, deo, den, dL0, dto, dtt, dtl, dtri, dcap, dfix,
                                               tau, nn);
        ck(cudaGetLastError());
        std::swap(dx0, dx1);
        if (flip_every > 0 && (it + 1) % flip_every == 0 && e == cudaSuccess) {
            ck(cudaMemcpyAsync(x.data(), dx0, 16 * nn, cudaMemcpyDeviceToHost, s));
            ck(cudaStreamSynchronize(s));
            if (e != cudaSuccess) break;
            const int64_t k = lawson(x, t, keep);
            flips += k;
            if (k > 0) {
                lists();
                upload_lists();
            }
        }
    }
    if (e == cudaSuccess) {
        ck(cudaMemcpyAsync(x.data(), dx0, 16 * nn, cudaMemcpyDeviceToHost, s));
        ck(cudaStreamSynchronize(s));
    }
    for (void* p : {(void*)dx0, (void*)dx1, (void*)dt, (void*)deo, (void*)den, (void*)dL0, (void*)dto,
                    (void*)dtt, (void*)dtl, (void*)dH0, (void*)dcap, (void*)dfix, (void*)dtri})
        if (p) cudaFree(p);
    if (e != cudaSuccess) {
        err = std::string("mesh relaxation: ") + cudaGetErrorString(e);
        return UE_ERR_CUDA;
    }
    for (int64_t i = 0; i < nt; ++i)
        if (!(orient2d(x, t[3 * i], t[3 * i + 1], t[3 * i + 2]) > 0)) {
            err = "relaxation inverted triangle " + std::to_string(i) + ": lower tau";
            return UE_ERR_DEGENERATE;
        }
    std::copy(x.begin(), x.end(), xy_out);
    std::copy(t.begin(), t.end(), tris_out);
    if (n_flips) *n_flips = flips;
    return UE_OK;
}

}  // namespace ue
