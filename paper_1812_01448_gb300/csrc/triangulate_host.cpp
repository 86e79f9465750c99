// Mesh generation on the host (Section 3, "Mesh generation"): the Delaunay triangulation of a
// seeded node cloud over its convex hull, then the flip refinement of Fig. 5a that restores
// geometry segments crossed by triangle edges, a Lawson pass that makes every other edge locally
// Delaunay again (so the result is the constrained Delaunay triangulation), and the removal of
// holes and of the part outside the outer contour.
//
// Construction: Bowyer-Watson insertion in Hilbert-curve order.  The hull carries "ghost"
// triangles (a, b, G) with G a vertex at infinity beyond the hull edge a->b; a node lies in a
// ghost's circle when it is strictly beyond that edge, or on the open edge itself.  With exact
// predicates every cavity is star-shaped around the new node, nodes outside the hull need no
// enclosing triangle, and no triangle is ever flat.
//
// Predicates: orientation and in-circle signs are exact.  A double-precision evaluation is
// accepted when it exceeds a bound on its rounding error far above the true one; otherwise the
// determinant is recomputed as a floating-point expansion (a sum of non-overlapping doubles)
// built from error-free transformations: Knuth's two-sum, and the exact product error given by
// a fused multiply-add (the method of Priest and of Shewchuk's adaptive-precision predicates).
// The expansion's sign is the sign of its largest component.  Compiled with -ffp-contract=off,
// so every other operation rounds on its own and the result is the same on every host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <unordered_set>
#include <utility>

#include "ue_internal.h"

namespace ue {

namespace {

// ------------------------------------------------------------------ exact arithmetic

inline void two_sum(double a, double b, double& x, double& y) {
    x = a + b;
    const double bv = x - a, av = x - bv;
    y = (a - av) + (b - bv);
}

inline void two_prod(double a, double b, double& x, double& y) {
    x = a * b;
    y = std::fma(a, b, -x);
}

// Expansions: components of increasing magnitude, non-overlapping, zeros removed; at most N
// components, held on the stack (each operation's worst-case length is known statically).
template <int N>
struct Exp {
    double v[N];
    int n = 0;
};

template <int N, int M>
void copy(const Exp<M>& e, Exp<N>& h) {
    static_assert(N >= M, "expansion capacity");
    h.n = e.n;
    std::memcpy(h.v, e.v, sizeof(double) * e.n);
}

// h = e + b (growing the expansion by one double; h has room for e.n + 1 components)
template <int N, int M>
void grow(const Exp<M>& e, double b, Exp<N>& h) {
    h.n = 0;
    double q = b;
    for (int i = 0; i < e.n; ++i) {
        double s, t;
        two_sum(q, e.v[i], s, t);
        if (t != 0.0) h.v[h.n++] = t;
        q = s;
    }
    if (q != 0.0 || h.n == 0) h.v[h.n++] = q;
}

// out = e + f, by growing e with each component of f (two buffers used in turn)
template <int N, int M, int K>
void sum(const Exp<M>& e, const Exp<K>& f, Exp<N>& out) {
    static_assert(N >= M + K, "expansion capacity");
    if (f.n == 0) {
        copy(e, out);
        return;
    }
    Exp<N> tmp;
    Exp<N>* dst = (f.n - 1) % 2 == 0 ? &out : &tmp;   // so that the last grow lands in out
    Exp<N>* src = dst == &out ? &tmp : &out;
    grow(e, f.v[0], *dst);
    for (int j = 1; j < f.n; ++j) {
        std::swap(dst, src);
        grow(*src, f.v[j], *dst);
    }
}

// out = e * b
template <int M>
void scale(const Exp<M>& e, double b, Exp<2 * M>& out) {
    Exp<2 * M> tmp;
    out.n = 0;
    for (int i = 0; i < e.n; ++i) {
        double p, q;
        two_prod(e.v[i], b, p, q);
        grow(out, q, tmp);
        grow(tmp, p, out);
    }
}

// out = e * f
template <int M, int K>
void mul(const Exp<M>& e, const Exp<K>& f, Exp<2 * M * K>& out) {
    Exp<2 * M * K> tmp;
    Exp<2 * M> s;
    Exp<2 * M * K>* acc = &out;
    Exp<2 * M * K>* nxt = &tmp;
    out.n = 0;
    for (int j = 0; j < f.n; ++j) {
        scale(e, f.v[j], s);
        for (int i = 0; i < s.n; ++i) {
            grow(*acc, s.v[i], *nxt);
            std::swap(acc, nxt);
        }
    }
    if (acc != &out) copy(*acc, out);
}

Exp<2> diff(double a, double b) {
    double x, y;
    two_sum(a, -b, x, y);
    Exp<2> e;
    if (y != 0.0) e.v[e.n++] = y;
    e.v[e.n++] = x;
    return e;
}

template <int N>
void negate(Exp<N>& e) {
    for (int i = 0; i < e.n; ++i) e.v[i] = -e.v[i];
}

template <int N>
int sign_of(const Exp<N>& e) {
    for (int i = e.n; i-- > 0;)
        if (e.v[i] != 0.0) return e.v[i] > 0 ? 1 : -1;
    return 0;
}

// Sign of (b - a) x (c - a): +1 counter-clockwise.
int orient(const double* a, const double* b, const double* c) {
    const double acx = a[0] - c[0], bcx = b[0] - c[0], acy = a[1] - c[1], bcy = b[1] - c[1];
    const double l = acx * bcy, r = acy * bcx, det = l - r;
    // relative rounding error of this form is below 4e-16; accept far above it
    if (std::fabs(det) > 1e-14 * (std::fabs(l) + std::fabs(r))) return det > 0 ? 1 : -1;
    Exp<8> p, q;
    mul(diff(a[0], c[0]), diff(b[1], c[1]), p);
    mul(diff(a[1], c[1]), diff(b[0], c[0]), q);
    negate(q);
    Exp<16> d;
    sum(p, q, d);
    return sign_of(d);
}

// x1 y2 - y1 x2
void cross(const Exp<2>& x1, const Exp<2>& y1, const Exp<2>& x2, const Exp<2>& y2, Exp<16>& out) {
    Exp<8> p, q;
    mul(x1, y2, p);
    mul(y1, x2, q);
    negate(q);
    sum(p, q, out);
}

// x^2 + y^2
void lift(const Exp<2>& x, const Exp<2>& y, Exp<16>& out) {
    Exp<8> p, q;
    mul(x, x, p);
    mul(y, y, q);
    sum(p, q, out);
}

// +1 where d lies strictly inside the circle through the CCW triangle (a, b, c).
int incircle(const double* a, const double* b, const double* c, const double* d) {
    const double adx = a[0] - d[0], ady = a[1] - d[1], bdx = b[0] - d[0], bdy = b[1] - d[1];
    const double cdx = c[0] - d[0], cdy = c[1] - d[1];
    const double al = adx * adx + ady * ady, bl = bdx * bdx + bdy * bdy, cl = cdx * cdx + cdy * cdy;
    const double bc = bdx * cdy - bdy * cdx, ca = cdx * ady - cdy * adx, ab = adx * bdy - ady * bdx;
    const double det = al * bc + bl * ca + cl * ab;
    const double perm = al * (std::fabs(bdx * cdy) + std::fabs(bdy * cdx)) +
                        bl * (std::fabs(cdx * ady) + std::fabs(cdy * adx)) +
                        cl * (std::fabs(adx * bdy) + std::fabs(ady * bdx));
    // relative rounding error of this form is below 1.2e-15; accept far above it
    if (std::fabs(det) > 1e-13 * perm) return det > 0 ? 1 : -1;
    const Exp<2> ax = diff(a[0], d[0]), ay = diff(a[1], d[1]), bx = diff(b[0], d[0]);
    const Exp<2> by = diff(b[1], d[1]), cx = diff(c[0], d[0]), cy = diff(c[1], d[1]);
    Exp<16> l, x;
    Exp<512> s0, s1, s2;
    lift(ax, ay, l);
    cross(bx, by, cx, cy, x);
    mul(l, x, s0);
    lift(bx, by, l);
    cross(cx, cy, ax, ay, x);
    mul(l, x, s1);
    lift(cx, cy, l);
    cross(ax, ay, bx, by, x);
    mul(l, x, s2);
    Exp<1024> s01;
    Exp<1536> s;
    sum(s0, s1, s01);
    sum(s01, s2, s);
    return sign_of(s);
}

// ------------------------------------------------------------------ the triangulation

constexpr int32_t G = -1;        // the vertex at infinity
constexpr int32_t DEAD = -2;     // v[0] of a recycled slot

struct Tri {
    int32_t v[3];   // counter-clockwise; a ghost keeps G in v[2]
    int32_t n[3];   // n[q]: the triangle across edge (v[q], v[q+1])
};

struct Delaunay {
    const double* xy;
    int64_t nn;
    std::vector<Tri> T;
    std::vector<int32_t> free_slots;
    std::vector<int32_t> vt;          // a live triangle at each inserted node
    std::vector<uint32_t> mark;       // per triangle: stamp of the last cavity search
    uint32_t stamp = 0;
    int32_t last = 0;                 // where the next walk starts
    std::vector<int32_t> cav, stack;
    struct BEdge { int32_t a, b, out, t; };
    std::vector<BEdge> bnd;

    const double* P(int32_t v) const { return xy + 2 * (int64_t)v; }
    bool ghost(int32_t t) const { return T[t].v[2] == G; }

    int32_t new_tri(int32_t a, int32_t b, int32_t c) {
        // rotate a ghost so that G comes last
        if (a == G) { a = b; b = c; c = G; }
        else if (b == G) { const int32_t t = a; a = c; b = t; c = G; }
        int32_t id;
        if (!free_slots.empty()) {
            id = free_slots.back();
            free_slots.pop_back();
        } else {
            id = (int32_t)T.size();
            T.push_back({});
            mark.push_back(0);
        }
        T[id] = Tri{{a, b, c}, {-1, -1, -1}};
        return id;
    }

    int edge_at(int32_t t, int32_t a, int32_t b) const {
        for (int q = 0; q < 3; ++q)
            if (T[t].v[q] == a && T[t].v[(q + 1) % 3] == b) return q;
        return -1;
    }

    bool between(int32_t a, int32_t b, const double* p) const {
        const double *A = P(a), *B = P(b);
        const int k = A[0] != B[0] ? 0 : 1;
        return std::min(A[k], B[k]) < p[k] && p[k] < std::max(A[k], B[k]);
    }

    bool in_circle(int32_t t, const double* p) const {
        const Tri& r = T[t];
        if (r.v[2] == G) {
            const int o = orient(P(r.v[0]), P(r.v[1]), p);
            return o > 0 || (o == 0 && between(r.v[0], r.v[1], p));
        }
        return incircle(P(r.v[0]), P(r.v[1]), P(r.v[2]), p) > 0;
    }

    // A triangle whose circle holds p: a real one containing p, or a ghost beyond whose edge
    // p lies.  -1: p repeats a node.
    int32_t locate(const double* p, bool& dup) {
        dup = false;
        int32_t t = last;
        if (T[t].v[0] == DEAD || ghost(t)) {
            t = -1;
            for (int32_t i = 0; i < (int32_t)T.size() && t < 0; ++i)
                if (T[i].v[0] != DEAD && !ghost(i)) t = i;
        }
        const int64_t cap = 64 + 4 * (int64_t)T.size();
        uint32_t rot = 0;
        for (int64_t step = 0; step < cap; ++step) {
            if (ghost(t)) return t;
            const Tri& r = T[t];
            int moved = -1;
            ++rot;
            for (int k = 0; k < 3 && moved < 0; ++k) {
                const int q = (int)((k + rot) % 3);
                if (orient(P(r.v[q]), P(r.v[(q + 1) % 3]), p) < 0) moved = q;
            }
            if (moved < 0) {
                for (int q = 0; q < 3; ++q)
                    if (P(r.v[q])[0] == p[0] && P(r.v[q])[1] == p[1]) dup = true;
                return dup ? -1 : t;
            }
            t = r.n[moved];
        }
        // the walk did not settle (it always does with exact predicates): scan
        for (int32_t i = 0; i < (int32_t)T.size(); ++i) {
            if (T[i].v[0] == DEAD) continue;
            if (!ghost(i)) {
                const Tri& r = T[i];
                bool inside = true;
                for (int q = 0; q < 3 && inside; ++q)
                    inside = orient(P(r.v[q]), P(r.v[(q + 1) % 3]), p) >= 0;
                if (inside) {
                    for (int q = 0; q < 3; ++q)
                        if (P(r.v[q])[0] == p[0] && P(r.v[q])[1] == p[1]) dup = true;
                    return dup ? -1 : i;
                }
            } else if (in_circle(i, p)) {
                return i;
            }
        }
        dup = true;
        return -1;
    }

    void link(int32_t t, int32_t a, int32_t b, int32_t s) {
        const int q = edge_at(t, a, b);
        T[t].n[q] = s;
    }

    // Bowyer-Watson: remove every triangle whose circle holds node p, join p to the cavity's
    // boundary.  Returns false if p repeats a node.
    bool insert(int32_t pv) {
        const double* p = P(pv);
        bool dup;
        const int32_t seed = locate(p, dup);
        if (seed < 0) return false;
        ++stamp;
        cav.clear();
        stack.clear();
        bnd.clear();
        mark[seed] = stamp;
        stack.push_back(seed);
        while (!stack.empty()) {
            const int32_t t = stack.back();
            stack.pop_back();
            cav.push_back(t);
            for (int q = 0; q < 3; ++q) {
                const int32_t s = T[t].n[q];
                if (mark[s] == stamp) continue;
                if (in_circle(s, p)) {
                    mark[s] = stamp;
                    stack.push_back(s);
                }
            }
        }
        for (int32_t t : cav)
            for (int q = 0; q < 3; ++q) {
                const int32_t s = T[t].n[q];
                if (mark[s] != stamp) bnd.push_back({T[t].v[q], T[t].v[(q + 1) % 3], s, -1});
            }
        for (int32_t t : cav) {
            T[t].v[0] = DEAD;
            free_slots.push_back(t);
        }
        for (BEdge& e : bnd) {
            e.t = new_tri(e.a, e.b, pv);
            link(e.t, e.a, e.b, e.out);
            link(e.out, e.b, e.a, e.t);
        }
        // the boundary is one cycle around p: edge (b, p) of the triangle on (a, b) meets edge
        // (p, b) of the triangle on (b, c)
        for (const BEdge& e : bnd)
            for (const BEdge& f : bnd)
                if (f.a == e.b) {
                    link(e.t, e.b, pv, f.t);
                    link(f.t, pv, f.a, e.t);
                    break;
                }
        for (const BEdge& e : bnd) {
            if (e.a != G) vt[e.a] = e.t;
            if (e.b != G) vt[e.b] = e.t;
            if (!ghost(e.t)) last = e.t;
        }
        vt[pv] = bnd.front().t;
        return true;
    }

    // The triangle holding directed edge (a, b), found around node a; -1 if none.
    int32_t find_edge(int32_t a, int32_t b, int* qout) const {
        int32_t t = vt[a];
        for (int guard = 0; guard < (1 << 20); ++guard) {
            int qa = -1;
            for (int q = 0; q < 3; ++q)
                if (T[t].v[q] == a) qa = q;
            if (T[t].v[(qa + 1) % 3] == b) {
                *qout = qa;
                return t;
            }
            t = T[t].n[(qa + 2) % 3];   // next triangle counter-clockwise around a
            if (t == vt[a]) return -1;
        }
        return -1;
    }

    // Triangles (a, b, c) and (b, a, d) become (c, a, d) and (d, b, c).
    void flip(int32_t t1, int q1, int32_t* c_out, int32_t* d_out) {
        const int32_t a = T[t1].v[q1], b = T[t1].v[(q1 + 1) % 3], c = T[t1].v[(q1 + 2) % 3];
        const int32_t t2 = T[t1].n[q1];
        const int q2 = edge_at(t2, b, a);
        const int32_t d = T[t2].v[(q2 + 2) % 3];
        const int32_t n_bc = T[t1].n[(q1 + 1) % 3], n_ca = T[t1].n[(q1 + 2) % 3];
        const int32_t n_ad = T[t2].n[(q2 + 1) % 3], n_db = T[t2].n[(q2 + 2) % 3];
        T[t1] = Tri{{c, a, d}, {n_ca, n_ad, t2}};
        T[t2] = Tri{{d, b, c}, {n_db, n_bc, t1}};
        link(n_ad, d, a, t1);
        link(n_bc, c, b, t2);
        vt[a] = t1;
        vt[b] = t2;
        vt[c] = t1;
        vt[d] = t1;
        *c_out = c;
        *d_out = d;
    }

    bool convex(int32_t a, int32_t b, int32_t c, int32_t d) const {
        return orient(P(c), P(a), P(d)) > 0 && orient(P(d), P(b), P(c)) > 0;
    }
};

// Hilbert index of (x, y) in [0, 2^16)^2, by the curve's recursive quadrant rule: at each
// level the quadrant adds (3 qx) ^ qy times the level's area, and the lower quadrants are
// reflected or transposed so that the curve enters and leaves them at the right corners.
uint64_t hilbert(uint32_t x, uint32_t y) {
    uint64_t d = 0;
    for (uint32_t s = 1u << 15; s > 0; s >>= 1) {
        const uint32_t rx = (x & s) ? 1 : 0, ry = (y & s) ? 1 : 0;
        d += (uint64_t)s * s * ((3 * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = s - 1 - (x & (s - 1)) + (x & ~(s - 1));
                y = s - 1 - (y & (s - 1)) + (y & ~(s - 1));
            }
            std::swap(x, y);
        }
    }
    return d;
}

uint64_t ekey(int32_t a, int32_t b) {
    return ((uint64_t)(uint32_t)std::min(a, b) << 32) | (uint32_t)std::max(a, b);
}

}  // namespace

int triangulate(const double* xy, int64_t nn, const int32_t* segs, int64_t n_segs, const double* holes,
                int64_t n_holes, int flags, std::vector<int32_t>& out, int64_t* n_flips, std::string& err) {
    if (!xy || nn < 3 || nn >= ((int64_t)1 << 29) || n_segs < 0 || n_holes < 0 || (n_segs > 0 && !segs) ||
        (n_holes > 0 && !holes)) {
        err = "ue_triangulate: bad arguments";
        return UE_ERR_ARG;
    }
    for (int64_t i = 0; i < 2 * nn; ++i)
        if (!std::isfinite(xy[i])) {
            err = "ue_triangulate: non-finite node coordinate";
            return UE_ERR_ARG;
        }
    for (int64_t s = 0; s < n_segs; ++s) {
        const int64_t u = segs[2 * s], v = segs[2 * s + 1];
        if (u < 0 || v < 0 || u >= nn || v >= nn || u == v) {
            err = "ue_triangulate: segment " + std::to_string(s) + " has a bad node id";
            return UE_ERR_ARG;
        }
    }
    // insertion order: along a Hilbert curve over the bounding box
    double lo[2] = {xy[0], xy[1]}, hi[2] = {xy[0], xy[1]};
    for (int64_t i = 0; i < nn; ++i)
        for (int k = 0; k < 2; ++k) {
            lo[k] = std::min(lo[k], xy[2 * i + k]);
            hi[k] = std::max(hi[k], xy[2 * i + k]);
        }
    std::vector<std::pair<uint64_t, int32_t>> key(nn);
    for (int64_t i = 0; i < nn; ++i) {
        uint32_t c[2];
        for (int k = 0; k < 2; ++k) {
            const double w = hi[k] > lo[k] ? (xy[2 * i + k] - lo[k]) / (hi[k] - lo[k]) : 0.0;
            c[k] = (uint32_t)std::min(65535.0, std::floor(w * 65536.0));
        }
        key[i] = {hilbert(c[0], c[1]), (int32_t)i};
    }
    std::sort(key.begin(), key.end());
    Delaunay D;
    D.xy = xy;
    D.nn = nn;
    D.vt.assign(nn, -1);
    D.T.reserve(2 * nn + 8);
    D.mark.reserve(2 * nn + 8);
    // the first triangle: the first two nodes and the first node off their line
    const int32_t a0 = key[0].second;
    int64_t i1 = 1;
    while (i1 < nn && xy[2 * key[i1].second] == xy[2 * a0] && xy[2 * key[i1].second + 1] == xy[2 * a0 + 1]) ++i1;
    if (i1 == nn) {
        err = "ue_triangulate: node " + std::to_string(key[1].second) + " repeats another node";
        return UE_ERR_DEGENERATE;
    }
    const int32_t b0 = key[i1].second;
    int64_t i2 = i1 + 1;
    while (i2 < nn && orient(D.P(a0), D.P(b0), D.P(key[i2].second)) == 0) ++i2;
    if (i2 == nn) {
        err = "ue_triangulate: all nodes are collinear (or repeated)";
        return UE_ERR_DEGENERATE;
    }
    int32_t c0 = key[i2].second, b1 = b0;
    if (orient(D.P(a0), D.P(b0), D.P(c0)) < 0) std::swap(b1, c0);
    {
        const int32_t t = D.new_tri(a0, b1, c0);
        const int32_t g0 = D.new_tri(b1, a0, G), g1 = D.new_tri(c0, b1, G), g2 = D.new_tri(a0, c0, G);
        D.T[t].n[0] = g0;
        D.T[t].n[1] = g1;
        D.T[t].n[2] = g2;
        // ghost (x, y, G): n[0] the real triangle, n[1] across (y, G), n[2] across (G, x)
        D.T[g0].n[0] = t;  D.T[g0].n[1] = g2;  D.T[g0].n[2] = g1;
        D.T[g1].n[0] = t;  D.T[g1].n[1] = g0;  D.T[g1].n[2] = g2;
        D.T[g2].n[0] = t;  D.T[g2].n[1] = g1;  D.T[g2].n[2] = g0;
        D.vt[a0] = D.vt[b1] = D.vt[c0] = t;
        D.last = t;
    }
    for (int64_t i = 1; i < nn; ++i) {
        if (i == i1 || i == i2) continue;
        const int32_t p = key[i].second;
        if (!D.insert(p)) {
            err = "ue_triangulate: node " + std::to_string(p) + " repeats another node";
            return UE_ERR_DEGENERATE;
        }
    }
    for (int64_t i = 0; i < nn; ++i)
        if (D.vt[i] < 0) {
            err = "ue_triangulate: node " + std::to_string(i) + " repeats another node";
            return UE_ERR_DEGENERATE;
        }

    // flip refinement of each segment (Fig. 5a), by a queue of crossing edges
    std::unordered_set<uint64_t> fixed;
    std::vector<std::pair<int32_t, int32_t>> touched;
    int64_t flips = 0;
    auto crosses = [&](int32_t u, int32_t v, int32_t a, int32_t b) {
        return orient(D.P(u), D.P(v), D.P(a)) * orient(D.P(u), D.P(v), D.P(b)) < 0 &&
               orient(D.P(a), D.P(b), D.P(u)) * orient(D.P(a), D.P(b), D.P(v)) < 0;
    };
    for (int64_t s = 0; s < n_segs; ++s) {
        const int32_t u = segs[2 * s], v = segs[2 * s + 1];
        int q = 0;
        if (D.find_edge(u, v, &q) >= 0 || D.find_edge(v, u, &q) >= 0) {
            fixed.insert(ekey(u, v));
            continue;
        }
        // walk from u towards v, collecting the crossed edges
        const double *pu = D.P(u), *pv = D.P(v);
        std::deque<std::pair<int32_t, int32_t>> queue;
        int32_t t = D.vt[u], x = -1, y = -1;
        for (int guard = 0; guard < (1 << 20); ++guard) {
            int qa = 0;
            while (D.T[t].v[qa] != u) ++qa;
            const int32_t b = D.T[t].v[(qa + 1) % 3], c = D.T[t].v[(qa + 2) % 3];
            if (b != G && c != G) {
                const int ob = orient(pu, D.P(b), pv), oc = orient(pu, D.P(c), pv);
                if ((ob == 0 && orient(pu, pv, D.P(b)) == 0 && D.between(u, v, D.P(b))) ||
                    (oc == 0 && orient(pu, pv, D.P(c)) == 0 && D.between(u, v, D.P(c)))) {
                    err = "ue_triangulate: a node lies on segment " + std::to_string(s);
                    return UE_ERR_ARG;
                }
                if (ob > 0 && oc < 0) {
                    x = b;
                    y = c;
                    break;
                }
            }
            t = D.T[t].n[(qa + 2) % 3];
            if (t == D.vt[u]) break;
        }
        if (x < 0) {
            err = "ue_triangulate: segment " + std::to_string(s) + " leaves the triangulation";
            return UE_ERR_ARG;
        }
        for (int guard = 0;; ++guard) {
            if (fixed.count(ekey(x, y))) {
                err = "ue_triangulate: segment " + std::to_string(s) + " crosses another segment";
                return UE_ERR_ARG;
            }
            queue.push_back({x, y});
            int qe = 0;
            const int32_t ta = D.find_edge(y, x, &qe);   // the triangle beyond (x, y), seen from u
            if (ta < 0 || D.ghost(ta)) {
                err = "ue_triangulate: segment " + std::to_string(s) + " walk lost its triangle";
                return UE_ERR_ARG;
            }
            const int32_t w = D.T[ta].v[(qe + 2) % 3];
            if (w == v) break;
            const int ow = orient(pu, pv, D.P(w));
            if (ow == 0) {
                err = "ue_triangulate: a node lies on segment " + std::to_string(s);
                return UE_ERR_ARG;
            }
            // x stays right of u->v and y left of it
            if (ow > 0) y = w; else x = w;
            if (guard > (1 << 24)) {
                err = "ue_triangulate: segment walk did not end";
                return UE_ERR_ARG;
            }
        }
        // the queue ends after at most about k^2 flips for k crossing edges; the cap turns a
        // broken refinement into an error instead of an endless loop
        const int64_t cap = 4 * ((int64_t)queue.size() + 1) * ((int64_t)queue.size() + 1) + 64;
        int64_t seg_flips = 0;
        size_t stall = 0;
        while (!queue.empty()) {
            if (seg_flips > cap) {
                err = "ue_triangulate: flip refinement of segment " + std::to_string(s) + " does not converge";
                return UE_ERR_ARG;
            }
            const auto e = queue.front();
            queue.pop_front();
            int q1 = 0;
            const int32_t t1 = D.find_edge(e.first, e.second, &q1);
            if (t1 < 0 || D.ghost(t1) || D.ghost(D.T[t1].n[q1])) {
                err = "ue_triangulate: flip refinement lost a crossing edge";
                return UE_ERR_ARG;
            }
            const int32_t t2 = D.T[t1].n[q1];
            const int q2 = D.edge_at(t2, e.second, e.first);
            const int32_t c = D.T[t1].v[(q1 + 2) % 3], d = D.T[t2].v[(q2 + 2) % 3];
            if (!D.convex(e.first, e.second, c, d)) {
                queue.push_back(e);
                if (++stall > queue.size()) {
                    err = "ue_triangulate: flip refinement made no progress";
                    return UE_ERR_ARG;
                }
                continue;
            }
            stall = 0;
            int32_t cc, dd;
            D.flip(t1, q1, &cc, &dd);
            ++flips;
            ++seg_flips;
            touched.push_back({cc, e.first});
            touched.push_back({e.first, dd});
            touched.push_back({dd, e.second});
            touched.push_back({e.second, cc});
            touched.push_back({cc, dd});
            if (cc != u && cc != v && dd != u && dd != v && crosses(u, v, cc, dd)) queue.push_back({cc, dd});
        }
        fixed.insert(ekey(u, v));
    }
    // Lawson: the edges next to the refinement's flips may have lost the Delaunay property
    while (!touched.empty()) {
        const auto e = touched.back();
        touched.pop_back();
        if (e.first == G || e.second == G || fixed.count(ekey(e.first, e.second))) continue;
        int q1 = 0;
        const int32_t t1 = D.find_edge(e.first, e.second, &q1);
        if (t1 < 0 || D.ghost(t1)) continue;
        const int32_t t2 = D.T[t1].n[q1];
        if (D.ghost(t2)) continue;
        const int q2 = D.edge_at(t2, e.second, e.first);
        const Tri& r = D.T[t1];
        const int32_t d = D.T[t2].v[(q2 + 2) % 3];
        if (incircle(D.P(r.v[q1]), D.P(r.v[(q1 + 1) % 3]), D.P(r.v[(q1 + 2) % 3]), D.P(d)) <= 0) continue;
        int32_t cc, dd;
        D.flip(t1, q1, &cc, &dd);
        touched.push_back({cc, e.first});
        touched.push_back({e.first, dd});
        touched.push_back({dd, e.second});
        touched.push_back({e.second, cc});
    }

    // regions: flood from the hole points, and from the hull edges that are not segments
    const int32_t nt_all = (int32_t)D.T.size();
    std::vector<char> gone(nt_all, 0);
    std::vector<int32_t> st;
    for (int64_t h = 0; h < n_holes; ++h) {
        if (!std::isfinite(holes[2 * h]) || !std::isfinite(holes[2 * h + 1])) {
            err = "ue_triangulate: non-finite hole point";
            return UE_ERR_ARG;
        }
        bool dup;
        D.last = D.vt[0];
        if (D.ghost(D.last)) D.last = D.T[D.last].n[0];
        const int32_t t = D.locate(holes + 2 * h, dup);
        if (t < 0 || D.ghost(t)) {
            err = "ue_triangulate: hole point " + std::to_string(h) + " is not inside the triangulation";
            return UE_ERR_ARG;
        }
        if (!gone[t]) {
            gone[t] = 1;
            st.push_back(t);
        }
    }
    if (flags & UE_TRI_DROP_EXTERIOR)
        for (int32_t t = 0; t < nt_all; ++t) {
            if (D.T[t].v[0] == DEAD || !D.ghost(t)) continue;
            const int32_t r = D.T[t].n[0];
            if (!gone[r] && !fixed.count(ekey(D.T[t].v[0], D.T[t].v[1]))) {
                gone[r] = 1;
                st.push_back(r);
            }
        }
    while (!st.empty()) {
        const int32_t t = st.back();
        st.pop_back();
        for (int q = 0; q < 3; ++q) {
            const int32_t s = D.T[t].n[q];
            if (D.ghost(s) || gone[s] || fixed.count(ekey(D.T[t].v[q], D.T[t].v[(q + 1) % 3]))) continue;
            gone[s] = 1;
            st.push_back(s);
        }
    }
    out.clear();
    for (int32_t t = 0; t < nt_all; ++t) {
        if (D.T[t].v[0] == DEAD || D.ghost(t) || gone[t]) continue;
        out.insert(out.end(), D.T[t].v, D.T[t].v + 3);
    }
    if (n_flips) *n_flips = flips;
    return UE_OK;
}

}  // namespace ue
