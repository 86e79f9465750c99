// Host mesh ingest: the Fig. 2 symbols (edges e_i, R(i), L(i), A(j,q) and the sign factor of
// eq. 4), PEC boundary edges removed from the unknowns (eq. 10), and the locality reordering
// of the triangles (reverse Cuthill-McKee on the dual graph; the "Divide and conqueror"
// section motivates keeping neighbours together).  Compiled with -ffp-contract=off so that
// the FP64 orientation determinant rounds the same way on every host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <utility>

#include "ue_internal.h"

namespace ue {

namespace {

// (p1 - p0) x (p2 - p0), twice the signed area.
inline double orient2d(const double* a, const double* b, const double* c) {
    const double bx = b[0] - a[0], by = b[1] - a[1];
    const double cx = c[0] - a[0], cy = c[1] - a[1];
    return bx * cy - by * cx;
}

struct Canon {
    std::vector<int64_t> tri;       // 3*n_t CCW caller node ids
    std::vector<int64_t> tri_edge;  // 3*n_t caller edge ids, A(j,q) = (v_q, v_{q+1})
    std::vector<int8_t> tri_neg;    // 3*n_t: 1 where s(j,q) = -1
    std::vector<int64_t> edges;     // 2*n_e
    std::vector<int64_t> R, L;      // n_e
};

int canonicalize(const double* xy, int64_t nn, const int32_t* tris, int64_t nt, Canon& c,
                 std::string& err) {
    c.tri.resize(3 * nt);
    for (int64_t j = 0; j < nt; ++j) {
        int64_t v0 = tris[3 * j], v1 = tris[3 * j + 1], v2 = tris[3 * j + 2];
        if (v0 < 0 || v1 < 0 || v2 < 0 || v0 >= nn || v1 >= nn || v2 >= nn) {
            err = "triangle " + std::to_string(j) + " has a vertex index out of range";
            return UE_ERR_ARG;
        }
        if (v0 == v1 || v1 == v2 || v0 == v2) {
            err = "triangle " + std::to_string(j) + " repeats a vertex";
            return UE_ERR_DEGENERATE;
        }
        const double det = orient2d(xy + 2 * v0, xy + 2 * v1, xy + 2 * v2);
        if (det == 0.0 || !std::isfinite(det)) {
            err = "triangle " + std::to_string(j) + " is degenerate (zero orientation determinant)";
            return UE_ERR_DEGENERATE;
        }
        if (det < 0) std::swap(v1, v2);
        c.tri[3 * j] = v0;
        c.tri[3 * j + 1] = v1;
        c.tri[3 * j + 2] = v2;
    }
    // half-edges in (low, high) order: counted by low node, then each node's few sorted by
    // (high, half-edge), the same order as one sort by (low * nn + high, half-edge)
    const int64_t nh = 3 * nt;
    std::vector<std::pair<int64_t, int64_t>> he(nh);
    {
        std::vector<int64_t> start(nn + 1, 0);
        for (int64_t h = 0; h < nh; ++h) {
            const int64_t j = h / 3, q = h % 3;
            ++start[std::min(c.tri[3 * j + q], c.tri[3 * j + (q + 1) % 3]) + 1];
        }
        for (int64_t v = 0; v < nn; ++v) start[v + 1] += start[v];
        std::vector<int64_t> at(start.begin(), start.end() - 1);
        for (int64_t h = 0; h < nh; ++h) {
            const int64_t j = h / 3, q = h % 3;
            const int64_t a = c.tri[3 * j + q], b = c.tri[3 * j + (q + 1) % 3];
            const int64_t lo = std::min(a, b);
            he[at[lo]++] = {lo * nn + std::max(a, b), h};
        }
        for (int64_t v = 0; v < nn; ++v) std::sort(he.begin() + start[v], he.begin() + start[v + 1]);
    }
    c.tri_edge.assign(nh, -1);
    c.tri_neg.assign(nh, 0);
    c.edges.clear();
    c.edges.reserve(nh);
    int64_t ne = 0;
    for (int64_t s = 0; s < nh;) {
        int64_t e = s;
        while (e < nh && he[e].first == he[s].first) ++e;
        if (e - s > 2) {
            err = "edge shared by more than two triangles";
            return UE_ERR_NONMANIFOLD;
        }
        const int64_t key = he[s].first;
        c.edges.push_back(key / nn);
        c.edges.push_back(key % nn);
        for (int64_t t = s; t < e; ++t) c.tri_edge[he[t].second] = ne;
        ++ne;
        s = e;
    }
    c.R.assign(ne, -1);
    c.L.assign(ne, -1);
    for (int64_t h = 0; h < nh; ++h) {
        const int64_t j = h / 3, q = h % 3;
        const int64_t a = c.tri[3 * j + q], b = c.tri[3 * j + (q + 1) % 3];
        const int64_t e = c.tri_edge[h];
        if (a < b) {
            if (c.R[e] >= 0) {
                err = "edge walked twice in the same direction (folded or overlapping triangles)";
                return UE_ERR_NONMANIFOLD;
            }
            c.R[e] = j;
        } else {
            c.tri_neg[h] = 1;
            if (c.L[e] >= 0) {
                err = "edge walked twice in the same direction (folded or overlapping triangles)";
                return UE_ERR_NONMANIFOLD;
            }
            c.L[e] = j;
        }
    }
    return UE_OK;
}

// Reverse Cuthill-McKee on the dual graph with the tie-breaks: components by smallest caller
// id, start = min (degree, id), neighbours appended in (degree, id) order, reversed at the end.
std::vector<int64_t> rcm(const Canon& c, int64_t nt) {
    std::vector<int64_t> ptr(nt + 1, 0);
    const int64_t ne = (int64_t)c.R.size();
    for (int64_t e = 0; e < ne; ++e)
        if (c.R[e] >= 0 && c.L[e] >= 0) {
            ++ptr[c.R[e] + 1];
            ++ptr[c.L[e] + 1];
        }
    for (int64_t j = 0; j < nt; ++j) ptr[j + 1] += ptr[j];
    std::vector<int64_t> adj(ptr[nt]);
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t e = 0; e < ne; ++e)
        if (c.R[e] >= 0 && c.L[e] >= 0) {
            adj[fill[c.R[e]]++] = c.L[e];
            adj[fill[c.L[e]]++] = c.R[e];
        }
    auto deg = [&](int64_t v) { return ptr[v + 1] - ptr[v]; };
    auto less = [&](int64_t a, int64_t b) {
        const int64_t da = deg(a), db = deg(b);
        return da != db ? da < db : a < b;
    };
    std::vector<char> seen(nt, 0);
    std::vector<int64_t> order;
    order.reserve(nt);
    std::vector<int64_t> comp;
    std::vector<int64_t> nb;
    for (int64_t root = 0; root < nt; ++root) {
        if (seen[root]) continue;
        comp.clear();
        comp.push_back(root);
        seen[root] = 1;
        for (size_t k = 0; k < comp.size(); ++k)
            for (int64_t p = ptr[comp[k]]; p < ptr[comp[k] + 1]; ++p)
                if (!seen[adj[p]]) {
                    seen[adj[p]] = 1;
                    comp.push_back(adj[p]);
                }
        int64_t start = comp[0];
        for (int64_t v : comp) {
            seen[v] = 0;
            if (less(v, start)) start = v;
        }
        size_t head = order.size();
        order.push_back(start);
        seen[start] = 1;
        while (head < order.size()) {
            const int64_t v = order[head++];
            nb.clear();
            for (int64_t p = ptr[v]; p < ptr[v + 1]; ++p)
                if (!seen[adj[p]]) nb.push_back(adj[p]);
            std::sort(nb.begin(), nb.end(), less);
            for (int64_t w : nb) {
                seen[w] = 1;
                order.push_back(w);
            }
        }
    }
    std::reverse(order.begin(), order.end());
    return order;
}

// KD partition (the paper's "KD tree idea": recursive bisection into parts of equal size
// along x or y): split at the median of the triangle centroids along the longer extent of
// their bounding box, ties by RCM position, until a part has at most tile_tris triangles.
// Parts are emitted depth-first (left before right); inside a part the RCM order is kept.
void kd_order(const Canon& c, const double* xy, const std::vector<int64_t>& rcm_order,
              int64_t tile_tris, std::vector<int64_t>& order, std::vector<int64_t>& tile_off) {
    const int64_t nt = (int64_t)rcm_order.size();
    std::vector<int64_t> pos(nt);
    for (int64_t i = 0; i < nt; ++i) pos[rcm_order[i]] = i;
    std::vector<double> cx(nt), cy(nt);
    for (int64_t j = 0; j < nt; ++j) {
        const int64_t a = c.tri[3 * j], b = c.tri[3 * j + 1], d = c.tri[3 * j + 2];
        cx[j] = (xy[2 * a] + xy[2 * b] + xy[2 * d]) / 3.0;
        cy[j] = (xy[2 * a + 1] + xy[2 * b + 1] + xy[2 * d + 1]) / 3.0;
    }
    std::vector<int64_t> ids(rcm_order);
    order.clear();
    tile_off.assign(1, 0);
    struct Part { int64_t lo, hi; };
    std::vector<Part> stack{{0, nt}};
    while (!stack.empty()) {
        Part p = stack.back();
        stack.pop_back();
        const int64_t n = p.hi - p.lo;
        if (n <= tile_tris) {
            std::sort(ids.begin() + p.lo, ids.begin() + p.hi,
                      [&](int64_t u, int64_t v) { return pos[u] < pos[v]; });
            order.insert(order.end(), ids.begin() + p.lo, ids.begin() + p.hi);
            tile_off.push_back((int64_t)order.size());
            continue;
        }
        double x0 = cx[ids[p.lo]], x1 = x0, y0 = cy[ids[p.lo]], y1 = y0;
        for (int64_t i = p.lo; i < p.hi; ++i) {
            const int64_t j = ids[i];
            x0 = std::min(x0, cx[j]);
            x1 = std::max(x1, cx[j]);
            y0 = std::min(y0, cy[j]);
            y1 = std::max(y1, cy[j]);
        }
        const std::vector<double>& key = (x1 - x0 >= y1 - y0) ? cx : cy;
        // only the set below the median matters (both halves are split again or sorted by RCM
        // position), and (key, RCM position) is a strict total order: a selection gives the
        // same sets as a full sort
        const int64_t mid = p.lo + n / 2;
        std::nth_element(ids.begin() + p.lo, ids.begin() + mid, ids.begin() + p.hi, [&](int64_t u, int64_t v) {
            return key[u] != key[v] ? key[u] < key[v] : pos[u] < pos[v];
        });
        stack.push_back({mid, p.hi});   // right part, processed after the left one
        stack.push_back({p.lo, mid});
    }
}

// Greedy partition (the paper's "greedy" method of the "Divide and conqueror" section) with its
// two refinements.  No part ever holds more than tile_tris triangles.
// * Growth: a part grows breadth first from its root, each dequeued triangle adding its
//   unassigned neighbours in RCM-position order, until it has target = tile_tris - tile_tris/8
//   triangles or its front is used up.  The next root is the "sharpest" unassigned triangle of
//   the current boundary: among the unassigned triangles with fewer than 3 unassigned neighbours,
//   one with the fewest, ties by RCM position.
// * Small parts: in creation order, a part of fewer than theta = tile_tris/8 triangles joins the
//   smallest neighbouring part of at least theta triangles (ties by part index) that can take it.
// * Hanging triangles: a triangle with one edge on its own part and its two other edges on one
//   other part Q moves to Q if Q has room.  Sweeps in RCM order, moving as found, until a sweep
//   moves none; each move adds a same-part adjacency, so the sweeps end.
// Parts are emitted in index order, RCM order inside each.
// A set of positions 0..n-1 with a smallest-member query: a 64-ary tree of bit words, a bit of
// one level set where the word below it is not empty.
struct PosSet {
    std::vector<std::vector<uint64_t>> lv;   // lv[0]: one bit per position; the last: one word
    explicit PosSet(int64_t n) {
        int64_t m = n;
        do {
            m = (m + 63) / 64;
            lv.emplace_back(m, 0);
        } while (m > 1);
    }
    void insert(int64_t p) {
        for (auto& w : lv) {
            const bool had = w[p >> 6] != 0;
            w[p >> 6] |= 1ull << (p & 63);
            if (had) return;
            p >>= 6;
        }
    }
    void erase(int64_t p) {
        for (auto& w : lv) {
            w[p >> 6] &= ~(1ull << (p & 63));
            if (w[p >> 6] != 0) return;
            p >>= 6;
        }
    }
    int64_t first() const {   // -1 when empty
        if (lv.back()[0] == 0) return -1;
        int64_t i = 0;
        for (size_t l = lv.size(); l-- > 0;) i = i * 64 + __builtin_ctzll(lv[l][i]);
        return i;
    }
};

// Inside each tile, the triangles within kRingCap rings of the tile's boundary (the triangles
// with an edge-neighbour in another tile are ring 0) come first, ring by ring, each ring in
// order of the angle of its centroids around the tile's centroid; deeper triangles keep their
// order.  A neighbouring tile's halo holds the rings next to their shared boundary: an arc of
// each ring, which this order stores as one run, so the blocked kernel gathers it from few
// 32-byte sectors instead of one per value.  The tiles themselves (their sets and offsets) do
// not change.
constexpr int kRingCap = 15;

void ring_order_in_tiles(const Canon& c, const double* xy, int64_t nt, std::vector<int64_t>& order,
                         const std::vector<int64_t>& tile_off) {
    std::vector<int64_t> ptr(nt + 1, 0);
    const int64_t ne = (int64_t)c.R.size();
    for (int64_t e = 0; e < ne; ++e)
        if (c.R[e] >= 0 && c.L[e] >= 0) {
            ++ptr[c.R[e] + 1];
            ++ptr[c.L[e] + 1];
        }
    for (int64_t j = 0; j < nt; ++j) ptr[j + 1] += ptr[j];
    std::vector<int64_t> adj(ptr[nt]);
    {
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t e = 0; e < ne; ++e)
            if (c.R[e] >= 0 && c.L[e] >= 0) {
                adj[fill[c.R[e]]++] = c.L[e];
                adj[fill[c.L[e]]++] = c.R[e];
            }
    }
    const int64_t ntiles = (int64_t)tile_off.size() - 1;
    std::vector<int64_t> tile_of(nt);
    for (int64_t t = 0; t < ntiles; ++t)
        for (int64_t i = tile_off[t]; i < tile_off[t + 1]; ++i) tile_of[order[i]] = t;
    std::vector<int32_t> ring(nt, kRingCap);
    std::vector<double> cx(nt), cy(nt), ang(nt);
    for (int64_t j = 0; j < nt; ++j) {
        double x = 0.0, y = 0.0;
        for (int q = 0; q < 3; ++q) {
            x += xy[2 * c.tri[3 * j + q]];
            y += xy[2 * c.tri[3 * j + q] + 1];
        }
        cx[j] = x / 3.0;
        cy[j] = y / 3.0;
    }
    std::vector<int64_t> queue, pos_in_tile(nt);
    for (int64_t t = 0; t < ntiles; ++t) {
        const int64_t a = tile_off[t], b = tile_off[t + 1];
        double mx = 0.0, my = 0.0;
        queue.clear();
        for (int64_t i = a; i < b; ++i) {
            const int64_t j = order[i];
            pos_in_tile[j] = i;
            mx += cx[j];
            my += cy[j];
            for (int64_t p = ptr[j]; p < ptr[j + 1]; ++p)
                if (tile_of[adj[p]] != t) {
                    ring[j] = 0;
                    queue.push_back(j);
                    break;
                }
        }
        mx /= (double)(b - a);
        my /= (double)(b - a);
        for (size_t h = 0; h < queue.size(); ++h) {   // breadth first inside the tile
            const int64_t j = queue[h];
            if (ring[j] + 1 >= kRingCap) continue;
            for (int64_t p = ptr[j]; p < ptr[j + 1]; ++p) {
                const int64_t o = adj[p];
                if (tile_of[o] == t && ring[o] > ring[j] + 1) {
                    ring[o] = ring[j] + 1;
                    queue.push_back(o);
                }
            }
        }
        for (int64_t i = a; i < b; ++i) {
            const int64_t j = order[i];
            ang[j] = std::atan2(cy[j] - my, cx[j] - mx);
        }
        std::stable_sort(order.begin() + a, order.begin() + b, [&](int64_t u, int64_t v) {
            if (ring[u] != ring[v]) return ring[u] < ring[v];
            if (ring[u] == kRingCap) return pos_in_tile[u] < pos_in_tile[v];
            if (ang[u] != ang[v]) return ang[u] < ang[v];
            return pos_in_tile[u] < pos_in_tile[v];
        });
    }
}

void greedy_order(const Canon& c, int64_t nt, const std::vector<int64_t>& rcm_order, int64_t tile_tris,
                  std::vector<int64_t>& order, std::vector<int64_t>& tile_off) {
    const int64_t theta = tile_tris / 8, target = tile_tris - theta;
    std::vector<int64_t> pos(nt);
    for (int64_t i = 0; i < nt; ++i) pos[rcm_order[i]] = i;
    std::vector<int64_t> ptr(nt + 1, 0);
    const int64_t ne = (int64_t)c.R.size();
    for (int64_t e = 0; e < ne; ++e)
        if (c.R[e] >= 0 && c.L[e] >= 0) {
            ++ptr[c.R[e] + 1];
            ++ptr[c.L[e] + 1];
        }
    for (int64_t j = 0; j < nt; ++j) ptr[j + 1] += ptr[j];
    std::vector<int64_t> adj(ptr[nt]);
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t e = 0; e < ne; ++e)
        if (c.R[e] >= 0 && c.L[e] >= 0) {
            adj[fill[c.R[e]]++] = c.L[e];
            adj[fill[c.L[e]]++] = c.R[e];
        }
    for (int64_t j = 0; j < nt; ++j)   // neighbours in RCM-position order
        std::sort(adj.begin() + ptr[j], adj.begin() + ptr[j + 1],
                  [&](int64_t a, int64_t b) { return pos[a] < pos[b]; });

    // growth
    std::vector<int> free_cnt(nt);
    std::vector<int64_t> part_of(nt, -1);
    PosSet bucket[3] = {PosSet(nt), PosSet(nt), PosSet(nt)};   // RCM positions by free count
    for (int64_t j = 0; j < nt; ++j) {
        free_cnt[j] = (int)(ptr[j + 1] - ptr[j]);
        if (free_cnt[j] < 3) bucket[free_cnt[j]].insert(pos[j]);
    }
    std::vector<int64_t> psize;
    std::vector<std::vector<int64_t>> members;
    auto take = [&](int64_t u, int64_t p) {
        part_of[u] = p;
        if (free_cnt[u] < 3) bucket[free_cnt[u]].erase(pos[u]);
        for (int64_t k = ptr[u]; k < ptr[u + 1]; ++k) {
            const int64_t w = adj[k];
            if (part_of[w] >= 0) continue;
            if (free_cnt[w] < 3) bucket[free_cnt[w]].erase(pos[w]);
            --free_cnt[w];
            bucket[free_cnt[w]].insert(pos[w]);
        }
    };
    int64_t left = nt, next_free = 0;   // next_free: fallback scan in RCM order
    while (left > 0) {
        int64_t root = -1;
        for (int k = 0; k < 3 && root < 0; ++k) {
            const int64_t f = bucket[k].first();
            if (f >= 0) root = rcm_order[f];
        }
        if (root < 0) {
            while (part_of[rcm_order[next_free]] >= 0) ++next_free;
            root = rcm_order[next_free];
        }
        const int64_t p = (int64_t)psize.size();
        members.emplace_back();
        std::vector<int64_t>& q = members.back();   // the part, in BFS order, is its own queue
        take(root, p);
        q.push_back(root);
        for (size_t qh = 0; qh < q.size() && (int64_t)q.size() < target; ++qh) {
            const int64_t u = q[qh];
            for (int64_t k = ptr[u]; k < ptr[u + 1] && (int64_t)q.size() < target; ++k) {
                const int64_t w = adj[k];
                if (part_of[w] >= 0) continue;
                take(w, p);
                q.push_back(w);
            }
        }
        psize.push_back((int64_t)q.size());
        left -= (int64_t)q.size();
    }
    const int64_t np = (int64_t)psize.size();

    // small parts (a receiver has >= theta triangles, so it is never small itself)
    for (int64_t p = 0; p < np; ++p) {
        if (psize[p] == 0 || psize[p] >= theta) continue;
        int64_t best = -1;
        for (int64_t u : members[p])
            for (int64_t k = ptr[u]; k < ptr[u + 1]; ++k) {
                const int64_t o = part_of[adj[k]];
                if (o == p || psize[o] < theta || psize[o] + psize[p] > tile_tris) continue;
                if (best < 0 || psize[o] < psize[best] || (psize[o] == psize[best] && o < best)) best = o;
            }
        if (best < 0) continue;
        for (int64_t u : members[p]) part_of[u] = best;
        psize[best] += psize[p];
        psize[p] = 0;
    }

    // hanging triangles
    for (bool moved = true; moved;) {
        moved = false;
        for (int64_t i = 0; i < nt; ++i) {
            const int64_t u = rcm_order[i];
            if (ptr[u + 1] - ptr[u] != 3) continue;
            const int64_t p = part_of[u];
            int own = 0;
            int64_t q = -1;
            bool one_other = true;
            for (int64_t k = ptr[u]; k < ptr[u + 1]; ++k) {
                const int64_t o = part_of[adj[k]];
                if (o == p) ++own;
                else if (q < 0) q = o;
                else if (o != q) one_other = false;
            }
            if (own != 1 || !one_other || psize[q] >= tile_tris) continue;
            part_of[u] = q;
            --psize[p];
            ++psize[q];
            moved = true;
        }
    }

    // emit: parts in index order, RCM order inside
    std::vector<int64_t> start(np + 1, 0);
    for (int64_t j = 0; j < nt; ++j) ++start[part_of[j] + 1];
    for (int64_t p = 0; p < np; ++p) start[p + 1] += start[p];
    order.assign(nt, -1);
    std::vector<int64_t> at(start.begin(), start.end() - 1);
    for (int64_t i = 0; i < nt; ++i) {
        const int64_t u = rcm_order[i];
        order[at[part_of[u]]++] = u;
    }
    tile_off.assign(1, 0);
    for (int64_t p = 0; p < np; ++p)
        if (start[p + 1] > start[p]) tile_off.push_back(start[p + 1]);
}

}  // namespace

int build_host_mesh(const double* xy, int64_t n_nodes, const int32_t* tris, int64_t n_tris,
                    int reorder, int tile_tris, HostMesh& hm, std::string& err) {
    if (!xy || !tris || n_nodes < 3 || n_tris < 1 || n_nodes > INT32_MAX || n_tris > (INT32_MAX / 4)) {
        err = "bad mesh arguments (null pointer or size out of range)";
        return UE_ERR_ARG;
    }
    for (int64_t i = 0; i < 2 * n_nodes; ++i)
        if (!std::isfinite(xy[i])) {
            err = "non-finite node coordinate";
            return UE_ERR_ARG;
        }
    Canon c;
    int rc = canonicalize(xy, n_nodes, tris, n_tris, c, err);
    if (rc != UE_OK) return rc;
    const int64_t ne = (int64_t)c.R.size();
    hm.n_nodes = n_nodes;
    hm.n_tris = n_tris;
    hm.n_edges = ne;
    hm.xy.assign(xy, xy + 2 * n_nodes);
    hm.edges = c.edges;
    // triangle order
    hm.tile_tri_off.clear();
    if (reorder == UE_REORDER_RCM) {
        hm.perm_tri = rcm(c, n_tris);
    } else if (reorder == UE_REORDER_KD || reorder == UE_REORDER_GREEDY || reorder == UE_REORDER_GREEDY_RINGS) {
        if (tile_tris < 16) {
            err = "tile_tris must be >= 16";
            return UE_ERR_ARG;
        }
        std::vector<int64_t> r = rcm(c, n_tris);
        if (reorder == UE_REORDER_KD) kd_order(c, xy, r, tile_tris, hm.perm_tri, hm.tile_tri_off);
        else greedy_order(c, n_tris, r, tile_tris, hm.perm_tri, hm.tile_tri_off);
        if (reorder == UE_REORDER_GREEDY_RINGS) ring_order_in_tiles(c, xy, n_tris, hm.perm_tri, hm.tile_tri_off);
    } else {
        hm.perm_tri.resize(n_tris);
        std::iota(hm.perm_tri.begin(), hm.perm_tri.end(), 0);
    }
    std::vector<int64_t> new_of(n_tris);
    for (int64_t j = 0; j < n_tris; ++j) new_of[hm.perm_tri[j]] = j;
    // interior edges numbered by (min, max) stored triangle id: counted by the smaller
    // triangle (at most 3 edges each), then each bucket sorted by the larger one
    std::vector<std::pair<std::pair<int64_t, int64_t>, int64_t>> ie;
    {
        std::vector<int64_t> start(n_tris + 1, 0);
        int64_t n_int = 0;
        for (int64_t e = 0; e < ne; ++e)
            if (c.R[e] >= 0 && c.L[e] >= 0) {
                ++start[std::min(new_of[c.R[e]], new_of[c.L[e]]) + 1];
                ++n_int;
            }
        for (int64_t j = 0; j < n_tris; ++j) start[j + 1] += start[j];
        std::vector<int64_t> at(start.begin(), start.end() - 1);
        ie.resize(n_int);
        for (int64_t e = 0; e < ne; ++e)
            if (c.R[e] >= 0 && c.L[e] >= 0) {
                const int64_t r = new_of[c.R[e]], l = new_of[c.L[e]];
                const int64_t lo = std::min(r, l);
                ie[at[lo]++] = {{lo, std::max(r, l)}, e};
            }
        for (int64_t j = 0; j < n_tris; ++j) std::sort(ie.begin() + start[j], ie.begin() + start[j + 1]);
    }
    const int64_t n_ei = (int64_t)ie.size();
    hm.n_ei = n_ei;
    hm.edge_caller.resize(n_ei);
    hm.k_of_edge.assign(ne, -1);
    hm.edge_tri.resize(2 * n_ei);
    hm.edge_nodes.resize(2 * n_ei);
    for (int64_t k = 0; k < n_ei; ++k) {
        const int64_t e = ie[k].second;
        hm.edge_caller[k] = e;
        hm.k_of_edge[e] = k;
        hm.edge_tri[2 * k] = (int32_t)new_of[c.R[e]];
        hm.edge_tri[2 * k + 1] = (int32_t)new_of[c.L[e]];
        hm.edge_nodes[2 * k] = (int32_t)c.edges[2 * e];
        hm.edge_nodes[2 * k + 1] = (int32_t)c.edges[2 * e + 1];
    }
    // per stored triangle: vertices rotated to start at the smallest caller node id
    hm.tri_nodes.resize(3 * n_tris);
    hm.tri_code.resize(3 * n_tris);
    hm.edge_opp.assign(2 * n_ei, -1);
    for (int64_t j = 0; j < n_tris; ++j) {
        const int64_t cj = hm.perm_tri[j];
        const int64_t* v = &c.tri[3 * cj];
        int rot = 0;
        if (v[1] < v[rot]) rot = 1;
        if (v[2] < v[rot]) rot = 2;
        for (int q = 0; q < 3; ++q) {
            const int src = (rot + q) % 3;
            hm.tri_nodes[3 * j + q] = (int32_t)v[src];
            const int64_t e = c.tri_edge[3 * cj + src];
            const int64_t k = hm.k_of_edge[e];
            if (k < 0) {
                hm.tri_code[3 * j + q] = (int32_t)(2 * n_ei);
            } else {
                const int neg = c.tri_neg[3 * cj + src];
                hm.tri_code[3 * j + q] = (int32_t)(2 * k + neg);
                hm.edge_opp[2 * k + neg] = (int32_t)v[(src + 2) % 3];
            }
        }
    }
    return UE_OK;
}

}  // namespace ue
