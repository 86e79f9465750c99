// FP64 setup kernels: geometry of eqs. 3-4 and 7, update coefficients, the power iteration of
// Section 2 ("complex time" method) for rho(M), and field transfer between the caller's
// numbering and the stored one.  One thread per triangle or edge; these run once per mesh.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "device.cuh"

namespace ue {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// Circumcentre O_j (where B_j lives, Fig. 2) and area S_j of each stored triangle.
__global__ void k_geom_tri(const double* __restrict__ xy, const int32_t* __restrict__ tn,
                           double* __restrict__ O, double* __restrict__ S, int64_t n_t) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_t) return;
    const int a = tn[3 * j], b = tn[3 * j + 1], c = tn[3 * j + 2];
    const double ax = xy[2 * a], ay = xy[2 * a + 1];
    const double bx = xy[2 * b] - ax, by = xy[2 * b + 1] - ay;
    const double cx = xy[2 * c] - ax, cy = xy[2 * c + 1] - ay;
    const double det = bx * cy - by * cx;
    const double b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
    O[2 * j] = ax + (cy * b2 - by * c2) / (2.0 * det);
    O[2 * j + 1] = ay + (bx * c2 - cx * b2) / (2.0 * det);
    S[j] = 0.5 * det;
}

// cot of the angle at o in triangle (a, b, o).
__device__ __forceinline__ double cot_at(double ax, double ay, double bx, double by, double ox,
                                         double oy) {
    const double ux = ax - ox, uy = ay - oy, vx = bx - ox, vy = by - oy;
    return (ux * vx + uy * vy) / fabs(ux * vy - uy * vx);
}

// |e_i| and the dual length |O_R O_L| of eq. 3 in the cotangent form
// d_i = |e_i|/2 (cot alpha_R + cot alpha_L), alpha = angle opposite e_i (stable for
// near-degenerate triangles, where subtracting two circumcentres would cancel).
__global__ void k_geom_edge(const double* __restrict__ xy, const int32_t* __restrict__ en,
                            const int32_t* __restrict__ eo, double* __restrict__ elen,
                            double* __restrict__ d, int64_t n_ei) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_ei) return;
    const int a = en[2 * k], b = en[2 * k + 1], r = eo[2 * k], l = eo[2 * k + 1];
    const double ax = xy[2 * a], ay = xy[2 * a + 1], bx = xy[2 * b], by = xy[2 * b + 1];
    const double len = hypot(bx - ax, by - ay);
    const double cr = cot_at(ax, ay, bx, by, xy[2 * r], xy[2 * r + 1]);
    const double cl = cot_at(ax, ay, bx, by, xy[2 * l], xy[2 * l + 1]);
    elen[k] = len;
    d[k] = 0.5 * len * (cr + cl);
}

template <typename T>
__global__ void k_coeff_edge(const double* __restrict__ elen, const double* __restrict__ d,
                             T* __restrict__ cU, double dt, int64_t n_ei) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_ei) return;
    cU[k] = (T)(dt * elen[k] / d[k]);
}

// Triangle record {code0, code1, code2, bits of (float)(dt/S)}; FP64 build: separate dt/S.
// Padding records [n_t, n_t_pad) point all three codes at the zero slot with coefficient 0.
__global__ void k_coeff_tri(const int32_t* __restrict__ code, const double* __restrict__ S,
                            int4* __restrict__ tri, double* __restrict__ cB64, double dt,
                            int64_t n_t, int64_t n_t_pad, int zero_code) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_t_pad) return;
    int4 r;
    double c = 0.0;
    if (j < n_t) {
        c = dt / S[j];
        r.x = code[3 * j];
        r.y = code[3 * j + 1];
        r.z = code[3 * j + 2];
    } else {
        r.x = r.y = r.z = zero_code;
    }
    r.w = cB64 ? 0 : __float_as_int((float)c);
    tri[j] = r;
    if (cB64) cB64[j] = c;
}

template <typename T>
__global__ void k_source_flags(T* __restrict__ cU, const int32_t* __restrict__ k, int64_t n, bool on) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T v = fabs(cU[k[i]]);
    cU[k[i]] = on ? -v : v;
}

// ---------------------------------------------------------------------------------------
// power iteration, FP64.  (K v)_j = (1/S_j) sum_q s(j,q) |e_q| (v_R - v_L)/d_q.
// ---------------------------------------------------------------------------------------

// SplitMix64 (Steele, Lea, Flood 2014), published constants.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Per edge c_k = |e_k| / d_k and per triangle 1/S_j, once: the iterations then only multiply
// and add (FP64 division and square root are slow on GB300's few FP64 pipes).
__global__ void k_pi_prep(const double* __restrict__ elen, const double* __restrict__ d,
                          const double* __restrict__ S, double* __restrict__ c,
                          double* __restrict__ invS, int64_t n_ei, int64_t n_t) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_ei) c[i] = elen[i] / d[i];
    if (i < n_t) invS[i] = 1.0 / S[i];
}

// Fixed-order sum of the block partials (x_b, y_b) by the last block of a grid (deterministic
// whichever block finishes last); sc = {sum x, sum y, 1/sqrt(sum y)}.  The sum covers this
// grid's partials and `extra` more after them, written by an earlier launch (a frame's cells).
// counter: zero before, zero after.
__device__ void pi_last_block(const double* __restrict__ part, double* __restrict__ sc,
                              unsigned int* __restrict__ counter, double* s_a, double* s_b,
                              int64_t extra) {
    __shared__ int last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double x = 0.0, y = 0.0;
    for (int64_t i = threadIdx.x; i < (int64_t)gridDim.x + extra; i += kThreads) {
        x += __ldcg(part + 2 * i);
        y += __ldcg(part + 2 * i + 1);
    }
    s_a[threadIdx.x] = x;
    s_b[threadIdx.x] = y;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s_a[threadIdx.x] += s_a[threadIdx.x + o];
            s_b[threadIdx.x] += s_b[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sc[0] = s_a[0];
        sc[1] = s_b[0];
        sc[2] = s_b[0] > 0.0 ? 1.0 / sqrt(s_b[0]) : 0.0;
        *counter = 0u;
    }
}

// Block tree of (x, y) into part[2 * block]; then, unless sc is NULL, the last block's
// fixed-order total.
__device__ void pi_block_sums(double x, double y, double* __restrict__ part, double* __restrict__ sc,
                              unsigned int* __restrict__ counter, int64_t extra = 0) {
    __shared__ double s_a[kThreads], s_b[kThreads];
    s_a[threadIdx.x] = x;
    s_b[threadIdx.x] = y;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s_a[threadIdx.x] += s_a[threadIdx.x + o];
            s_b[threadIdx.x] += s_b[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s_a[0];
        part[2 * blockIdx.x + 1] = s_b[0];
    }
    if (!sc) return;
    __syncthreads();
    pi_last_block(part, sc, counter, s_a, s_b, extra);
}

// Start: w = SplitMix64 vector, sc = {0, S-norm^2 of w, 1/S-norm of w}.
__global__ void k_pi_start(double* __restrict__ w, const int64_t* __restrict__ perm,
                           const double* __restrict__ S, uint32_t seed, int64_t n_t,
                           double* __restrict__ part, double* __restrict__ sc,
                           unsigned int* __restrict__ counter, int64_t extra) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double ww = 0.0;
    if (j < n_t) {
        const uint64_t z = splitmix64(((uint64_t)seed << 32) + (uint64_t)perm[j]);
        const double x = (double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0;
        w[j] = x;
        ww = S[j] * x * x;
    }
    pi_block_sums(0.0, ww, part, sc, counter, extra);
}

// g_k = c_k (v_R - v_L) with v = w * sc[2], the S-normalised iterate.
__global__ void k_pi_edge(const int2* __restrict__ rl, const double* __restrict__ c,
                          const double* __restrict__ w, const double* __restrict__ sc,
                          double* __restrict__ g, int64_t n_ei) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_ei) return;
    const double inv = sc[2];
    const int2 e = rl[k];
    g[k] = c[k] * (w[e.x] * inv - w[e.y] * inv);
}

// wn = K v: t_j = signed sum of the three g, wn_j = t_j / S_j.  Sums S v wn = v t (the
// Rayleigh quotient, v S-normalised) and S wn^2 = wn t go to sc_next with 1/sqrt of the latter.
__global__ void k_pi_tri(const int4* __restrict__ tri, const double* __restrict__ invS,
                         const double* __restrict__ g, const double* __restrict__ w,
                         const double* __restrict__ sc, double* __restrict__ wn,
                         double* __restrict__ part, double* __restrict__ sc_next,
                         unsigned int* __restrict__ counter, int64_t n_t, int64_t extra) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double vw = 0.0, ww = 0.0;
    if (j < n_t) {
        const int4 q = tri[j];
        double a = g[q.x >> 1], b = g[q.y >> 1], c = g[q.z >> 1];
        if (q.x & 1) a = -a;
        if (q.y & 1) b = -b;
        if (q.z & 1) c = -c;
        const double t = a + b + c;
        const double x = t * invS[j];
        wn[j] = x;
        vw = (w[j] * sc[2]) * t;
        ww = x * t;
    }
    pi_block_sums(vw, ww, part, sc_next, counter, extra);
}

// Frame cells of the coupled system (see kernels_frame.cu for the layout): the iterate's
// entries n_t + c, S = h^2, start vector keyed by n_t + c; partials go after the triangles'.
__global__ void k_fpi_start(FrameDev f, double* __restrict__ w, uint32_t seed, int64_t n_t,
                            double* __restrict__ part) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double ww = 0.0;
    if (c < f.n_fc) {
        const uint64_t z = splitmix64(((uint64_t)seed << 32) + (uint64_t)(n_t + c));
        const double x = (double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0;
        w[n_t + c] = x;
        ww = f.h * f.h * x * x;
    }
    pi_block_sums(0.0, ww, part, nullptr, nullptr);
}

// g on frame sides (|e| / d = 1: g = v_R - v_L) and on interface edges (ic (v_R - v_L)).
__global__ void k_fpi_edge(FrameDev f, const double* __restrict__ w, const double* __restrict__ sc,
                           int64_t n_t, double* __restrict__ g, double* __restrict__ gH,
                           double* __restrict__ gV) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double inv = sc[2];
    if (t < f.n_fc) {
        int I, J;
        frame_ij(f, t, I, J);
        const double vc = w[n_t + t] * inv;
        if (frame_is_cell(f, I, J - 1))
            gH[(int64_t)J * f.NX + I] = vc - w[n_t + frame_cell(f, I, J - 1)] * inv;
        if (frame_is_cell(f, I - 1, J))
            gV[(int64_t)J * (f.NX + 1) + I] = w[n_t + frame_cell(f, I - 1, J)] * inv - vc;
    } else if (t < f.n_fc + f.n_if) {
        const int64_t k = t - f.n_fc;
        const int32_t code = f.itri[k];
        const double vt = w[code >= 0 ? code : ~code] * inv, vc = w[n_t + f.icell[k]] * inv;
        g[f.u_off + k] = f.ic[k] * (code >= 0 ? vt - vc : vc - vt);
    }
}

// t_c = counter-clockwise signed sum of g over the cell's sides, wn = t_c / h^2; block
// partials of v t_c and wn t_c after the triangles' (no total here).
__global__ void k_fpi_cell(FrameDev f, const double* __restrict__ g, const double* __restrict__ gH,
                           const double* __restrict__ gV, const double* __restrict__ w,
                           const double* __restrict__ sc, double* __restrict__ wn, int64_t n_t,
                           double* __restrict__ part) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double vw = 0.0, ww = 0.0;
    if (c < f.n_fc) {
        int I, J;
        frame_ij(f, c, I, J);
        const bool in_x = I >= f.W && I < f.W + f.nx, in_y = J >= f.W && J < f.W + f.ny;
        auto iface = [&](int64_t k) { return f.itri[k] >= 0 ? -g[f.u_off + k] : g[f.u_off + k]; };
        double t = 0.0;
        if (frame_is_cell(f, I, J - 1)) t += gH[(int64_t)J * f.NX + I];
        else if (in_x && J == f.W + f.ny) t += iface(f.nx + (I - f.W));
        if (frame_is_cell(f, I, J + 1)) t -= gH[(int64_t)(J + 1) * f.NX + I];
        else if (in_x && J == f.W - 1) t += iface(I - f.W);
        if (frame_is_cell(f, I - 1, J)) t -= gV[(int64_t)J * (f.NX + 1) + I];
        else if (in_y && I == f.W + f.nx) t += iface(2 * (int64_t)f.nx + f.ny + (J - f.W));
        if (frame_is_cell(f, I + 1, J)) t += gV[(int64_t)J * (f.NX + 1) + I + 1];
        else if (in_y && I == f.W - 1) t += iface(2 * (int64_t)f.nx + (J - f.W));
        const double x = t / (f.h * f.h);
        wn[n_t + c] = x;
        vw = (w[n_t + c] * sc[2]) * t;
        ww = x * t;
    }
    pi_block_sums(vw, ww, part, nullptr, nullptr);
}

// ---------------------------------------------------------------------------------------
// fields: caller numbering (E per edge, B per triangle, FP64) <-> stored circulation form
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void k_fields_in_edges(const double* __restrict__ Ec, const int64_t* __restrict__ ec,
                                  const double* __restrict__ elen, T* __restrict__ U, int64_t n_ei) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n_ei) return;
    U[k] = (k == n_ei) ? (T)0 : (T)(elen[k] * Ec[ec[k]]);
}

template <typename T>
__global__ void k_fields_in_tris(const double* __restrict__ Bc, const int64_t* __restrict__ perm,
                                 T* __restrict__ B, int64_t n_t) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_t) return;
    B[j] = (T)Bc[perm[j]];
}

template <typename T>
__global__ void k_fields_out_edges(const T* __restrict__ U, const int64_t* __restrict__ ec,
                                   const double* __restrict__ relen, double* __restrict__ Ec,
                                   int64_t n_ei) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_ei) return;
    Ec[ec[k]] = (double)U[k] * relen[k];
}

template <typename T>
__global__ void k_fields_out_tris(const T* __restrict__ B, const int64_t* __restrict__ perm,
                                  double* __restrict__ Bc, int64_t n_t) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_t) return;
    Bc[perm[j]] = (double)B[j];
}

// Field transfer in caller order: from or to the caller's arrays in pinned host memory through
// their mapped device addresses, or a device copy of them.  Each thread takes V = 16 /
// sizeof(H) consecutive caller elements, so that the caller's side moves in 16-byte accesses
// (when the array is 16-byte aligned; element by element otherwise) and in order.  H is the
// caller's element type (double, or float for the FP32 calls); the arithmetic is that of the
// staged kernels above, in FP64, rounded once to H or T.  k_of[c] = stored interior edge of
// caller edge c or -1; inv[c] = stored triangle of caller triangle c.
template <typename H> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

template <typename H>
__device__ __forceinline__ void load_caller(const H* __restrict__ p, int64_t c0, int64_t n, bool vec,
                                            H (&x)[16 / sizeof(H)]) {
    constexpr int V = 16 / sizeof(H);
    if (vec && c0 + V <= n) {
        const typename Vec16<H>::type v = *reinterpret_cast<const typename Vec16<H>::type*>(p + c0);
        memcpy(x, &v, 16);
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i) x[i] = c0 + i < n ? p[c0 + i] : H(0);
    }
}

template <typename H>
__device__ __forceinline__ void store_caller(H* __restrict__ p, int64_t c0, int64_t n, bool vec,
                                             const H (&x)[16 / sizeof(H)]) {
    constexpr int V = 16 / sizeof(H);
    if (vec && c0 + V <= n) {
        typename Vec16<H>::type v;
        memcpy(&v, x, 16);
        *reinterpret_cast<typename Vec16<H>::type*>(p + c0) = v;
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i)
            if (c0 + i < n) p[c0 + i] = x[i];
    }
}

template <int V>
__device__ __forceinline__ void load_ids(const int32_t* __restrict__ a, int64_t c0, int64_t n, int32_t (&k)[V]) {
    if constexpr (V == 4) {
        if (c0 + 4 <= n) {
            const int4 v = __ldg(reinterpret_cast<const int4*>(a + c0));
            k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
            return;
        }
    } else {
        if (c0 + 2 <= n) {
            const int2 v = __ldg(reinterpret_cast<const int2*>(a + c0));
            k[0] = v.x; k[1] = v.y;
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < V; ++i) k[i] = c0 + i < n ? __ldg(a + c0 + i) : -1;
}

template <typename T, typename H>
__global__ void k_fields_in_edges_c(const H* __restrict__ Ec, const int32_t* __restrict__ k_of,
                                    const double* __restrict__ elen, T* __restrict__ U, int64_t n_e,
                                    int64_t n_ei, bool vec) {
    constexpr int V = 16 / sizeof(H);
    const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (c0 == 0) U[n_ei] = (T)0;
    if (c0 >= n_e) return;
    H e[V];
    int32_t k[V];
    load_caller(Ec, c0, n_e, vec, e);
    load_ids<V>(k_of, c0, n_e, k);
#pragma unroll
    for (int i = 0; i < V; ++i)
        if (k[i] >= 0) U[k[i]] = (T)(elen[k[i]] * (double)e[i]);
}

template <typename T, typename H>
__global__ void k_fields_in_tris_c(const H* __restrict__ Bc, const int32_t* __restrict__ inv,
                                   T* __restrict__ B, int64_t n_t, bool vec) {
    constexpr int V = 16 / sizeof(H);
    const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (c0 >= n_t) return;
    H b[V];
    int32_t j[V];
    load_caller(Bc, c0, n_t, vec, b);
    load_ids<V>(inv, c0, n_t, j);
#pragma unroll
    for (int i = 0; i < V; ++i)
        if (j[i] >= 0) B[j[i]] = (T)b[i];
}

template <typename T, typename H>
__global__ void k_fields_out_edges_c(const T* __restrict__ U, const int32_t* __restrict__ k_of,
                                     const double* __restrict__ relen, H* __restrict__ Ec, int64_t n_e, bool vec) {
    constexpr int V = 16 / sizeof(H);
    const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (c0 >= n_e) return;
    int32_t k[V];
    load_ids<V>(k_of, c0, n_e, k);
    H e[V];
#pragma unroll
    for (int i = 0; i < V; ++i) e[i] = k[i] >= 0 ? (H)((double)U[k[i]] * relen[k[i]]) : (H)0;
    store_caller(Ec, c0, n_e, vec, e);
}

template <typename T, typename H>
__global__ void k_fields_out_tris_c(const T* __restrict__ B, const int32_t* __restrict__ inv,
                                    H* __restrict__ Bc, int64_t n_t, bool vec) {
    constexpr int V = 16 / sizeof(H);
    const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (c0 >= n_t) return;
    int32_t j[V];
    load_ids<V>(inv, c0, n_t, j);
    H b[V];
#pragma unroll
    for (int i = 0; i < V; ++i) b[i] = j[i] >= 0 ? (H)B[j[i]] : (H)0;
    store_caller(Bc, c0, n_t, vec, b);
}

// B of the triangles with the given caller ids to / from a packed buffer (the halo exchange
// of a partitioned mesh): out[i] = B[inv[ids[i]]], B[inv[ids[i]]] = in[i].  Ids outside
// [0, n_t) are skipped and counted in *bad.
template <typename T>
__global__ void k_gather_tris(const T* __restrict__ B, const int32_t* __restrict__ inv,
                              const int32_t* __restrict__ ids, T* __restrict__ out, int64_t n,
                              int64_t n_t, unsigned* __restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t c = ids[i];
    if (c < 0 || c >= n_t) {
        atomicAdd(bad, 1u);
        return;
    }
    out[i] = B[inv[c]];
}

template <typename T>
__global__ void k_scatter_tris(T* __restrict__ B, const int32_t* __restrict__ inv,
                               const int32_t* __restrict__ ids, const T* __restrict__ in, int64_t n,
                               int64_t n_t, unsigned* __restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t c = ids[i];
    if (c < 0 || c >= n_t) {
        atomicAdd(bad, 1u);
        return;
    }
    B[inv[c]] = in[i];
}

template <typename T>
__global__ void k_plasma_coeff(const double* __restrict__ nn, const int32_t* __restrict__ en,
                               T* __restrict__ pb, double c, int64_t n_ei) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_ei) return;
    pb[k] = (T)(c * 0.5 * (nn[en[2 * k]] + nn[en[2 * k + 1]]));
}

template <typename T>
__global__ void k_source_coeff(const int32_t* __restrict__ sk, const int32_t* __restrict__ grp,
                               const double* __restrict__ par, const double* __restrict__ amp,
                               const double* __restrict__ elen, T* __restrict__ sc, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dt = par[4 * grp[i]];
    sc[i] = (T)(dt * elen[sk[i]] * amp[i]);
}

__global__ void k_scatter_geom_tri(const double* __restrict__ O, const double* __restrict__ S,
                                   const int64_t* __restrict__ perm, double* __restrict__ Oc,
                                   double* __restrict__ Sc, int64_t n_t) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_t) return;
    const int64_t c = perm[j];
    if (Oc) {
        Oc[2 * c] = O[2 * j];
        Oc[2 * c + 1] = O[2 * j + 1];
    }
    if (Sc) Sc[c] = S[j];
}

__global__ void k_fill_nan(double* __restrict__ a, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = __longlong_as_double(0x7ff8000000000000ll);
}

__global__ void k_scatter_geom_edge(const double* __restrict__ elen, const double* __restrict__ d,
                                    const int64_t* __restrict__ ec, double* __restrict__ lc,
                                    double* __restrict__ dc, int64_t n_ei) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_ei) return;
    if (lc) lc[ec[k]] = elen[k];
    if (dc) dc[ec[k]] = d[k];
}

}  // namespace

cudaError_t launch_geom_tri(const double* xy, const int32_t* tri_nodes, double* O, double* S,
                            int64_t n_t, cudaStream_t s) {
    k_geom_tri<<<blocks_for(n_t), kThreads, 0, s>>>(xy, tri_nodes, O, S, n_t);
    return cudaGetLastError();
}

// 1/|e| of every interior edge (the zero slot n_ei gets 0): the readout multiplies by it, since
// an FP64 division per element costs more than the transfer on GB300's FP64 pipes.
__global__ void k_recip(const double* __restrict__ elen, double* __restrict__ relen, int64_t n_ei) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n_ei) relen[k] = 1.0 / elen[k];
    else if (k == n_ei) relen[k] = 0.0;
}

cudaError_t launch_recip(const double* elen, double* relen, int64_t n_ei, cudaStream_t s) {
    k_recip<<<blocks_for(n_ei + 1), kThreads, 0, s>>>(elen, relen, n_ei);
    return cudaGetLastError();
}

cudaError_t launch_geom_edge(const double* xy, const int32_t* edge_nodes, const int32_t* edge_opp,
                             double* elen, double* d, int64_t n_ei, cudaStream_t s) {
    if (n_ei == 0) return cudaSuccess;
    k_geom_edge<<<blocks_for(n_ei), kThreads, 0, s>>>(xy, edge_nodes, edge_opp, elen, d, n_ei);
    return cudaGetLastError();
}

cudaError_t launch_coeff(const DevMesh& m, const double* elen, const double* d, const double* S,
                         const int32_t* tri_code, double dt, cudaStream_t s) {
    if (m.n_ei > 0) {
        if (m.precision == UE_PREC_FP64)
            k_coeff_edge<double><<<blocks_for(m.n_ei), kThreads, 0, s>>>(elen, d, (double*)m.cU, dt, m.n_ei);
        else
            k_coeff_edge<float><<<blocks_for(m.n_ei), kThreads, 0, s>>>(elen, d, (float*)m.cU, dt, m.n_ei);
    }
    k_coeff_tri<<<blocks_for(m.n_t_pad), kThreads, 0, s>>>(
        tri_code, S, m.tri, m.precision == UE_PREC_FP64 ? (double*)m.cB : nullptr, dt, m.n_t,
        m.n_t_pad, (int)(2 * m.n_ei));
    return cudaGetLastError();
}

namespace {

template <typename T>
__global__ void k_copy_abs(T* __restrict__ dst, const T* __restrict__ src, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = fabs(src[i]);
}

// Triangle records of one mesh placed in a batch: edge codes shifted by the mesh's first
// stored edge; the mesh's zero slot (code 2*nei_m) becomes the batch's zero slot.
__global__ void k_tri_offset(int4* __restrict__ dst, const int4* __restrict__ src, int64_t n,
                             int ei_off, int nei_m, int nei_all) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int4 r = src[j];
    r.x = (r.x >> 1) == nei_m ? 2 * nei_all : r.x + 2 * ei_off;
    r.y = (r.y >> 1) == nei_m ? 2 * nei_all : r.y + 2 * ei_off;
    r.z = (r.z >> 1) == nei_m ? 2 * nei_all : r.z + 2 * ei_off;
    dst[j] = r;
}

}  // namespace

namespace {

// Energy of eq. 8 with the eq. 7 weights, in circulation variables:
//   W = sum_i (d_i / |e_i|) U_i^2 + sum_j S_j B_j^2   (U = |e| E).
// Blocks [0, nbe) cover edges, [nbe, nbe + nbt) triangles; fixed-order partial sums.
template <typename T>
__global__ void k_energy_parts(const T* __restrict__ U, const T* __restrict__ B,
                               const double* __restrict__ elen, const double* __restrict__ d,
                               const double* __restrict__ S, int64_t n_ei, int64_t n_t, int nbe,
                               double* __restrict__ part) {
    __shared__ double a[kThreads];
    double x = 0.0;
    if ((int)blockIdx.x < nbe) {
        const int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x;
        if (k < n_ei) {
            const double u = (double)U[k];
            x = d[k] / elen[k] * u * u;
        }
    } else {
        const int64_t j = (int64_t)(blockIdx.x - nbe) * kThreads + threadIdx.x;
        if (j < n_t) {
            const double b = (double)B[j];
            x = S[j] * b * b;
        }
    }
    a[threadIdx.x] = x;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) a[threadIdx.x] += a[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = a[0];
}

// wd = {W at the previous check, W now, growth factor, flag}: flag 1 = non-finite energy,
// 2 = energy grew by more than the factor since the previous check.  A set flag stays set.
__global__ void k_energy_check(const double* __restrict__ part, int nb, double* __restrict__ wd) {
    __shared__ double a[kThreads];
    double x = 0.0;
    for (int i = threadIdx.x; i < nb; i += kThreads) x += part[i];
    a[threadIdx.x] = x;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) a[threadIdx.x] += a[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double W = a[0];
        wd[1] = W;
        if (wd[3] == 0.0) {
            if (!isfinite(W)) wd[3] = 1.0;
            else if (wd[2] > 0.0 && wd[0] > 0.0 && W > wd[2] * wd[0]) wd[3] = 2.0;
        }
        wd[0] = W;
    }
}

}  // namespace

size_t energy_parts(int64_t n_ei, int64_t n_t) {
    return (size_t)((n_ei + kThreads - 1) / kThreads + (n_t + kThreads - 1) / kThreads);
}

cudaError_t launch_energy(const DevMesh& m, const double* elen, const double* d, const double* S,
                          double* part, double* wd, cudaStream_t s) {
    const int nbe = (int)((m.n_ei + kThreads - 1) / kThreads);
    const int nbt = (int)((m.n_t + kThreads - 1) / kThreads);
    if (m.precision == UE_PREC_FP64)
        k_energy_parts<double><<<nbe + nbt, kThreads, 0, s>>>((const double*)m.U, (const double*)m.B,
                                                              elen, d, S, m.n_ei, m.n_t, nbe, part);
    else
        k_energy_parts<float><<<nbe + nbt, kThreads, 0, s>>>((const float*)m.U, (const float*)m.B,
                                                             elen, d, S, m.n_ei, m.n_t, nbe, part);
    k_energy_check<<<1, kThreads, 0, s>>>(part, nbe + nbt, wd);
    return cudaGetLastError();
}

cudaError_t launch_copy_abs(void* dst, const void* src, int64_t n, bool f64, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (f64) k_copy_abs<double><<<blocks_for(n), kThreads, 0, s>>>((double*)dst, (const double*)src, n);
    else k_copy_abs<float><<<blocks_for(n), kThreads, 0, s>>>((float*)dst, (const float*)src, n);
    return cudaGetLastError();
}

cudaError_t launch_tri_offset(int4* dst, const int4* src, int64_t n, int64_t ei_off, int64_t nei_m,
                              int64_t nei_all, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_tri_offset<<<blocks_for(n), kThreads, 0, s>>>(dst, src, n, (int)ei_off, (int)nei_m, (int)nei_all);
    return cudaGetLastError();
}

cudaError_t launch_source_flags(const DevMesh& m, const int32_t* k, int64_t n, bool on,
                                cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (m.precision == UE_PREC_FP64)
        k_source_flags<double><<<blocks_for(n), kThreads, 0, s>>>((double*)m.cU, k, n, on);
    else
        k_source_flags<float><<<blocks_for(n), kThreads, 0, s>>>((float*)m.cU, k, n, on);
    return cudaGetLastError();
}

size_t power_iteration_work_doubles(int64_t n_t, int64_t n_ei, const FrameDev* f) {
    const int64_t nb = (n_t + kThreads - 1) / kThreads;
    if (!f) return (size_t)(3 * n_t + 2 * n_ei + 1 + 2 * nb + 8 + 2);
    const int64_t nc = n_t + f->n_fc, nbf = (f->n_fc + kThreads - 1) / kThreads;
    const int64_t ng = f->u_off + f->n_if;
    const int64_t nh = (int64_t)f->NX * (f->NY + 1), nv = (int64_t)(f->NX + 1) * f->NY;
    return (size_t)(2 * nc + n_t + ng + n_ei + nh + nv + 2 * (nb + nbf) + 8 + 2);
}

// Two launches per iteration (edge, triangle with the reductions in its last block); the
// iterate is normalised on the fly by the scale its previous reduction left.  A frame adds
// its side and cell launches before them, its cells' partials summed by the triangles' last
// block after their own.
cudaError_t power_iteration(const int2* rl, const int4* tri, const double* elen, const double* d,
                            const double* S, const int64_t* perm_tri, int64_t n_t, int64_t n_ei,
                            int iters, uint32_t seed, double* work, double* rho, cudaStream_t s,
                            const FrameDev* f) {
    const int64_t nb = (n_t + kThreads - 1) / kThreads;
    const int64_t nbf = f ? (f->n_fc + kThreads - 1) / kThreads : 0;
    const int64_t nc = n_t + (f ? f->n_fc : 0);
    const int64_t ng = f ? f->u_off + f->n_if : n_ei + 1;
    const int64_t nh = f ? (int64_t)f->NX * (f->NY + 1) : 0, nv = f ? (int64_t)(f->NX + 1) * f->NY : 0;
    double* w[2] = {work, work + nc};
    double* invS = work + 2 * nc;
    double* g = invS + n_t;
    double* c = g + ng;
    double* gH = c + n_ei;
    double* gV = gH + nh;
    double* part = gV + nv;
    double* sc[2] = {part + 2 * (nb + nbf), part + 2 * (nb + nbf) + 4};
    unsigned int* counter = reinterpret_cast<unsigned int*>(part + 2 * (nb + nbf) + 8);
    cudaError_t e;
    if ((e = cudaMemsetAsync(g, 0, sizeof(double) * ng, s)) != cudaSuccess) return e;
    if (f && (e = cudaMemsetAsync(gH, 0, sizeof(double) * (nh + nv), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(counter, 0, sizeof(double), s)) != cudaSuccess) return e;
    k_pi_prep<<<blocks_for(n_ei > n_t ? n_ei : n_t), kThreads, 0, s>>>(elen, d, S, c, invS, n_ei, n_t);
    if (f) k_fpi_start<<<(unsigned)nbf, kThreads, 0, s>>>(*f, w[0], seed, n_t, part + 2 * nb);
    k_pi_start<<<(unsigned)nb, kThreads, 0, s>>>(w[0], perm_tri, S, seed, n_t, part, sc[0], counter, nbf);
    for (int it = 0; it < iters; ++it) {
        const int cur = it & 1;
        if (n_ei > 0) k_pi_edge<<<blocks_for(n_ei), kThreads, 0, s>>>(rl, c, w[cur], sc[cur], g, n_ei);
        if (f) {
            k_fpi_edge<<<blocks_for(f->n_fc + f->n_if), kThreads, 0, s>>>(*f, w[cur], sc[cur], n_t, g, gH, gV);
            k_fpi_cell<<<(unsigned)nbf, kThreads, 0, s>>>(*f, g, gH, gV, w[cur], sc[cur], w[cur ^ 1], n_t,
                                                         part + 2 * nb);
        }
        k_pi_tri<<<(unsigned)nb, kThreads, 0, s>>>(tri, invS, g, w[cur], sc[cur], w[cur ^ 1], part,
                                                  sc[cur ^ 1], counter, n_t, nbf);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    double h[2];
    if ((e = cudaMemcpyAsync(h, sc[iters & 1], sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    *rho = sqrt(h[0] > 0 ? h[0] : 0.0);
    return cudaSuccess;
}

cudaError_t launch_fields_in(const DevMesh& m, const double* Ec, const double* Bc, const double* Jc,
                             const int64_t* edge_caller, const int64_t* perm_tri,
                             const double* elen, cudaStream_t s) {
    const bool f64 = m.precision == UE_PREC_FP64;
    if (Ec) {
        if (f64) k_fields_in_edges<double><<<blocks_for(m.n_ei + 1), kThreads, 0, s>>>(Ec, edge_caller, elen, (double*)m.U, m.n_ei);
        else k_fields_in_edges<float><<<blocks_for(m.n_ei + 1), kThreads, 0, s>>>(Ec, edge_caller, elen, (float*)m.U, m.n_ei);
    }
    if (Jc && m.J) {
        if (f64) k_fields_in_edges<double><<<blocks_for(m.n_ei + 1), kThreads, 0, s>>>(Jc, edge_caller, elen, (double*)m.J, m.n_ei);
        else k_fields_in_edges<float><<<blocks_for(m.n_ei + 1), kThreads, 0, s>>>(Jc, edge_caller, elen, (float*)m.J, m.n_ei);
    }
    if (Bc) {
        if (f64) k_fields_in_tris<double><<<blocks_for(m.n_t), kThreads, 0, s>>>(Bc, perm_tri, (double*)m.B, m.n_t);
        else k_fields_in_tris<float><<<blocks_for(m.n_t), kThreads, 0, s>>>(Bc, perm_tri, (float*)m.B, m.n_t);
    }
    return cudaGetLastError();
}

cudaError_t launch_fields_out(const DevMesh& m, double* Ec, double* Bc, double* Jc,
                              const int64_t* edge_caller, const int64_t* perm_tri,
                              const double* relen, cudaStream_t s) {
    const bool f64 = m.precision == UE_PREC_FP64;
    if (Ec && m.n_ei > 0) {
        if (f64) k_fields_out_edges<double><<<blocks_for(m.n_ei), kThreads, 0, s>>>((const double*)m.U, edge_caller, relen, Ec, m.n_ei);
        else k_fields_out_edges<float><<<blocks_for(m.n_ei), kThreads, 0, s>>>((const float*)m.U, edge_caller, relen, Ec, m.n_ei);
    }
    if (Jc && m.J && m.n_ei > 0) {
        if (f64) k_fields_out_edges<double><<<blocks_for(m.n_ei), kThreads, 0, s>>>((const double*)m.J, edge_caller, relen, Jc, m.n_ei);
        else k_fields_out_edges<float><<<blocks_for(m.n_ei), kThreads, 0, s>>>((const float*)m.J, edge_caller, relen, Jc, m.n_ei);
    }
    if (Bc) {
        if (f64) k_fields_out_tris<double><<<blocks_for(m.n_t), kThreads, 0, s>>>((const double*)m.B, perm_tri, Bc, m.n_t);
        else k_fields_out_tris<float><<<blocks_for(m.n_t), kThreads, 0, s>>>((const float*)m.B, perm_tri, Bc, m.n_t);
    }
    return cudaGetLastError();
}

namespace {
inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
// threads for n caller elements of type H, V = 16 / sizeof(H) each
template <typename H>
inline unsigned blocks_for_vec(int64_t n) { return blocks_for((n + (16 / sizeof(H)) - 1) / (16 / sizeof(H))); }

template <typename T, typename H>
void fields_in_c(const DevMesh& m, const H* Ec, const H* Bc, const H* Jc, const int32_t* k_of, const int32_t* inv,
                 const double* elen, int64_t n_e, cudaStream_t s) {
    const int64_t ne = n_e > 0 ? n_e : 1;
    if (Ec) k_fields_in_edges_c<T, H><<<blocks_for_vec<H>(ne), kThreads, 0, s>>>(Ec, k_of, elen, (T*)m.U, n_e, m.n_ei, aligned16(Ec));
    if (Jc && m.J) k_fields_in_edges_c<T, H><<<blocks_for_vec<H>(ne), kThreads, 0, s>>>(Jc, k_of, elen, (T*)m.J, n_e, m.n_ei, aligned16(Jc));
    if (Bc) k_fields_in_tris_c<T, H><<<blocks_for_vec<H>(m.n_t), kThreads, 0, s>>>(Bc, inv, (T*)m.B, m.n_t, aligned16(Bc));
}

template <typename T, typename H>
void fields_out_c(const DevMesh& m, H* Ec, H* Bc, H* Jc, const int32_t* k_of, const int32_t* inv,
                  const double* relen, int64_t n_e, cudaStream_t s) {
    if (Ec && n_e > 0) k_fields_out_edges_c<T, H><<<blocks_for_vec<H>(n_e), kThreads, 0, s>>>((const T*)m.U, k_of, relen, Ec, n_e, aligned16(Ec));
    if (Jc && m.J && n_e > 0) k_fields_out_edges_c<T, H><<<blocks_for_vec<H>(n_e), kThreads, 0, s>>>((const T*)m.J, k_of, relen, Jc, n_e, aligned16(Jc));
    if (Bc) k_fields_out_tris_c<T, H><<<blocks_for_vec<H>(m.n_t), kThreads, 0, s>>>((const T*)m.B, inv, Bc, m.n_t, aligned16(Bc));
}
}  // namespace

cudaError_t launch_fields_in_caller(const DevMesh& m, const void* Ec, const void* Bc, const void* Jc, bool f32,
                                    const int32_t* k_of, const int32_t* inv, const double* elen, int64_t n_e,
                                    cudaStream_t s) {
    const bool f64 = m.precision == UE_PREC_FP64;
    if (f32) {
        auto E = (const float*)Ec, B = (const float*)Bc, J = (const float*)Jc;
        f64 ? fields_in_c<double, float>(m, E, B, J, k_of, inv, elen, n_e, s)
            : fields_in_c<float, float>(m, E, B, J, k_of, inv, elen, n_e, s);
    } else {
        auto E = (const double*)Ec, B = (const double*)Bc, J = (const double*)Jc;
        f64 ? fields_in_c<double, double>(m, E, B, J, k_of, inv, elen, n_e, s)
            : fields_in_c<float, double>(m, E, B, J, k_of, inv, elen, n_e, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_fields_out_caller(const DevMesh& m, void* Ec, void* Bc, void* Jc, bool f32, const int32_t* k_of,
                                     const int32_t* inv, const double* relen, int64_t n_e, cudaStream_t s) {
    const bool f64 = m.precision == UE_PREC_FP64;
    if (f32) {
        auto E = (float*)Ec, B = (float*)Bc, J = (float*)Jc;
        f64 ? fields_out_c<double, float>(m, E, B, J, k_of, inv, relen, n_e, s)
            : fields_out_c<float, float>(m, E, B, J, k_of, inv, relen, n_e, s);
    } else {
        auto E = (double*)Ec, B = (double*)Bc, J = (double*)Jc;
        f64 ? fields_out_c<double, double>(m, E, B, J, k_of, inv, relen, n_e, s)
            : fields_out_c<float, double>(m, E, B, J, k_of, inv, relen, n_e, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_tri_exchange(const DevMesh& m, const int32_t* inv, const int32_t* ids, int64_t n, void* buf,
                                int scatter, unsigned* bad, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (m.precision == UE_PREC_FP64) {
        if (scatter) k_scatter_tris<double><<<blocks_for(n), kThreads, 0, s>>>((double*)m.B, inv, ids, (const double*)buf, n, m.n_t, bad);
        else k_gather_tris<double><<<blocks_for(n), kThreads, 0, s>>>((const double*)m.B, inv, ids, (double*)buf, n, m.n_t, bad);
    } else {
        if (scatter) k_scatter_tris<float><<<blocks_for(n), kThreads, 0, s>>>((float*)m.B, inv, ids, (const float*)buf, n, m.n_t, bad);
        else k_gather_tris<float><<<blocks_for(n), kThreads, 0, s>>>((const float*)m.B, inv, ids, (float*)buf, n, m.n_t, bad);
    }
    return cudaGetLastError();
}

cudaError_t launch_plasma_coeff(const DevMesh& m, const double* n_nodes, const int32_t* edge_nodes,
                                double nu, double dt, cudaStream_t s) {
    if (m.n_ei == 0) return cudaSuccess;
    const double c = dt / (1.0 + 0.5 * nu * dt);
    if (m.precision == UE_PREC_FP64)
        k_plasma_coeff<double><<<blocks_for(m.n_ei), kThreads, 0, s>>>(n_nodes, edge_nodes, (double*)m.pb, c, m.n_ei);
    else
        k_plasma_coeff<float><<<blocks_for(m.n_ei), kThreads, 0, s>>>(n_nodes, edge_nodes, (float*)m.pb, c, m.n_ei);
    return cudaGetLastError();
}

cudaError_t launch_source_coeff(const DevMesh& m, const double* amp, const double* elen,
                                cudaStream_t s) {
    if (m.n_src == 0) return cudaSuccess;
    if (m.precision == UE_PREC_FP64)
        k_source_coeff<double><<<blocks_for(m.n_src), kThreads, 0, s>>>(m.src_k, m.src_grp, m.grp_par, amp, elen, (double*)m.src_c, m.n_src);
    else
        k_source_coeff<float><<<blocks_for(m.n_src), kThreads, 0, s>>>(m.src_k, m.src_grp, m.grp_par, amp, elen, (float*)m.src_c, m.n_src);
    return cudaGetLastError();
}

cudaError_t launch_scatter_geometry(const double* O, const double* S, const double* elen,
                                    const double* d, const int64_t* perm_tri,
                                    const int64_t* edge_caller, int64_t n_t, int64_t n_ei,
                                    int64_t n_e, double* O_c, double* S_c, double* elen_c,
                                    double* d_c, cudaStream_t s) {
    if (O_c || S_c) k_scatter_geom_tri<<<blocks_for(n_t), kThreads, 0, s>>>(O, S, perm_tri, O_c, S_c, n_t);
    if (elen_c) k_fill_nan<<<blocks_for(n_e), kThreads, 0, s>>>(elen_c, n_e);
    if (d_c) k_fill_nan<<<blocks_for(n_e), kThreads, 0, s>>>(d_c, n_e);
    if ((elen_c || d_c) && n_ei > 0)
        k_scatter_geom_edge<<<blocks_for(n_ei), kThreads, 0, s>>>(elen, d, edge_caller, elen_c, d_c, n_ei);
    return cudaGetLastError();
}

}  // namespace ue
