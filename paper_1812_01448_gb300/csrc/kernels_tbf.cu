// Fused, triangle-centric temporally blocked leap-frog (vacuum media): the same tiles, rings and
// pipeline as k_tbp (kernels_tb.cu), but one thread per local triangle carries the step of
// eqs. 3-4 (14-15) for its triangle and its three edges.
//
// Each edge is held, in registers, by both of its triangles, as V_q = s0 s_q U_q (s_q the
// orientation sign of edge q in the triangle, eq. 4).  One step of a triangle with own field b
// and neighbours n_q across its edges is
//   V_q = fma(c_q, rn(b - n_q), V_q)              c_q = s0 s_q t_q dt|e_q|/d_q   (eq. 3)
//   V_q = fma(s0 s_q a_q, g(t), V_q)              on a source edge
//   b   = fma(-s0 dt/S, rn(rn(V_0 + V_1) + V_2), b)                              (eq. 4)
// with t_q = +1 when the triangle is R of edge q and -1 when it is L.  Round-to-nearest is odd
// (rn(-y) = -rn(y)) and the sign factors are exact, so every value equals, bit for bit, the
// plain kernels' U_q += (dt|e|/d) rn(B_R - B_L), then the source, and B -= (dt/S) rn(rn(s0 U0 +
// s1 U1) + s2 U2): both triangles of an edge compute its value from the same inputs.  A step
// reads the neighbours' B from one buffer and writes the own B to the other, so it needs one
// barrier and three shared-memory gathers per triangle (the split kernel needs two barriers
// and, per triangle, the two gathers of 1.5 edges and three more).
//
// Per launch of kk steps a tile's triangles of level <= kk - 1 are advanced (level l at steps
// 1 .. kk - l); the level-kk ring is read only.  Owned triangles and edges are written back:
// B from registers, U through shared memory (each owned edge from an owned triangle).
// Pipeline: headers in a ring of three (TMA bulk copies), the next tile's records (TMA) as soon
// as this tile has read its own, and its fields (4-byte cp.async gathers) after step min(3, kk).
// Record layout: tiles_host.cpp build_fused_records.
#include <cuda_runtime.h>

#include "device.cuh"

namespace ue {

namespace {

struct TBFArgs {
    const int* hdr;
    const int* frec;      // 5 ints per local triangle
    const int* fedge;     // 2 ints per local edge {gid, bits of dt|e|/d, sign: source edge}
    const int2* tsrc;     // per tile {local edge, source index}, sorted by local edge
    const float* Bin;
    const float* Uin;
    float* Bout;
    float* Uout;
    const float* src_c;
    const int32_t* src_grp;
    const double* gtab;
    int gstride;
    int gbase;
    long long* step;
    unsigned* done;
    unsigned* err;
    int ksteps;
    int test_cta;         // tests only (-1 otherwise): as in kernels_tb.cu
};

template <int NT, int TS>
struct TbfLayout {
    static constexpr int TLC = TS * NT;                      // local triangle capacity
    static constexpr int ELC = 3 * TLC / 2 + 4;              // local edges + zero slot capacity
    // shared memory (bytes): two B buffers (the write-back area of U at the end of a tile),
    // the next tile's B and U, its triangle and edge records, the source positions
    static constexpr size_t BBUF = 0;
    static constexpr size_t BST = BBUF + 2 * 4 * (size_t)TLC;
    static constexpr size_t UST = BST + 4 * (size_t)TLC;
    static constexpr size_t TRST = UST + 4 * (size_t)ELC;
    static constexpr size_t EST = TRST + 20 * (size_t)TLC;
    static constexpr size_t SPOS = EST + 8 * (size_t)ELC;
    static constexpr size_t SMEM = SPOS + 4 * (size_t)TLC;
    static_assert(4 * TLC <= 16384, "14-bit neighbour offsets");
    static_assert(ELC <= 8192 && ELC <= 2 * TLC, "13-bit edge ids; U write-back fits the B buffers");
    static_assert(UST % 16 == 0 && TRST % 16 == 0 && EST % 16 == 0 && SPOS % 16 == 0, "alignment");
};

__device__ __forceinline__ float lds32(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}

__device__ __forceinline__ float flip(float x, uint32_t neg) {
    return __uint_as_float(__float_as_uint(x) ^ (neg << 31));
}

template <int NT, int TS>
__global__ void __launch_bounds__(NT, 1) k_tbf(TBFArgs a, int n_tiles) {
    using Lay = TbfLayout<NT, TS>;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ __align__(16) int hs[3][48];
    __shared__ __align__(8) uint64_t bar_h, bar_r;
    const int tid = threadIdx.x;
    const int stride = gridDim.x;
    const int kk = a.ksteps;
    float* Bb = reinterpret_cast<float*>(smraw + Lay::BBUF);
    float* Bst = reinterpret_cast<float*>(smraw + Lay::BST);
    float* Ust = reinterpret_cast<float*>(smraw + Lay::UST);
    int* trst = reinterpret_cast<int*>(smraw + Lay::TRST);
    int* est = reinterpret_cast<int*>(smraw + Lay::EST);
    int* spos = reinterpret_cast<int*>(smraw + Lay::SPOS);
    const uint32_t bb0 = smem_addr(Bb), bb1 = bb0 + 4u * Lay::TLC;
    if (tid == 0) {
        mbar_init(&bar_h, 1);
        mbar_init(&bar_r, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const long long n0 = *a.step;
    uint32_t ph_h = 0, ph_r = 0;
    int pend_h = 0, pend_r = 0;   // bulk copies issued and not yet waited for (uniform)
    bool ok = true;
    // a wait that runs out ends this CTA's work, agreed by every thread before any staged
    // value is used; the copies in flight are waited for (bounded) before the CTA exits
    auto wait_bar = [&](uint64_t* bar, uint32_t& ph) {
        if (!mbar_wait(bar, ph)) ok = false;
        ph ^= 1u;
        if (bar == &bar_h) --pend_h;
        else --pend_r;
        ok = __syncthreads_and(ok ? 1 : 0) != 0;
        return ok;
    };
    auto n_tri = [&](const int* h) { return h[16 + kk]; };
    auto n_edge = [&](const int* h) { return h[32 + kk - 1]; };
    auto issue_header = [&](int t, int slot) {
        ++pend_h;
        if (tid == 0) {
            fence_proxy_async();
            bulk_g2s(hs[slot], a.hdr + (size_t)t * 48, 48 * sizeof(int), &bar_h);
        }
    };
    bool first_records = true;
    auto issue_records = [&](int slot) {
        ++pend_r;
        const bool extra = first_records && (int)blockIdx.x == a.test_cta;
        first_records = false;
        if (tid == 0) {
            const int* h = hs[slot];
            const uint32_t tb = 20u * ((uint32_t)(n_tri(h) + 3) & ~3u);
            const uint32_t eb = 8u * ((uint32_t)(h[5] + 2) & ~1u);     // all edges and the zero slot
            fence_proxy_async();
            mbar_expect_tx(&bar_r, tb + eb + (extra ? 16u : 0u));
            bulk_copy_g2s(trst, a.frec + 5 * (size_t)h[11], tb, &bar_r);
            bulk_copy_g2s(est, a.fedge + 2 * (size_t)h[12], eb, &bar_r);
        }
    };
    auto issue_fields = [&](int slot) {
        const int* h = hs[slot];
        const int nt = n_tri(h), ne = n_edge(h);
#pragma unroll
        for (int i = 0; i < TS; ++i) {
            const int l = tid + i * NT;
            if (l < nt) cp_async4(Bst + l, a.Bin + trst[5 * l]);
        }
#pragma unroll
        for (int i = 0; i < (Lay::ELC + NT - 1) / NT; ++i) {
            const int l = tid + i * NT;
            if (l < ne) cp_async4(Ust + l, a.Uin + est[2 * l]);
        }
        if (tid == 0) Ust[h[5]] = 0.f;   // the zero slot of boundary edges
        cp_async_commit();
    };
    int tile = blockIdx.x, it = 0;
    if (tile < n_tiles) {
        issue_header(tile, 0);
        if (wait_bar(&bar_h, ph_h)) {
            issue_records(0);
            if (tile + stride < n_tiles) issue_header(tile + stride, 1);
            if (wait_bar(&bar_r, ph_r)) {
                issue_fields(0);
                cp_async_wait_all();
                if (tile + stride < n_tiles) wait_bar(&bar_h, ph_h);
            }
        }
    }
    if (!ok) tile = n_tiles;
    __syncthreads();
    // per slot: neighbour offsets and coefficient signs (r1), neighbour 2, edge 0 and the
    // orientation bits (r2), edges 1 and 2 (r3); the edge values V_q, the signed edge
    // coefficients, -s0 dt/S and B
    uint32_t r1[TS], r2[TS], r3[TS];
    float v0[TS], v1[TS], v2[TS], c0[TS], c1[TS], c2[TS], cb[TS], bv[TS];
    uint32_t srcm = 0;   // 3 bits per slot: edges with a source
    for (; tile < n_tiles; tile += stride, ++it) {
        const bool has_next = tile + stride < n_tiles, has_next2 = tile + 2 * stride < n_tiles;
        const int slot = it % 3, slot1 = (it + 1) % 3, slot2 = (it + 2) % 3;
        const int* h = hs[slot];
        const int nt_upd = h[16 + kk - 1], nt = n_tri(h);
        const bool has_src = h[9] > 0;
        srcm = 0;
#pragma unroll
        for (int i = 0; i < TS; ++i) {
            const int l = tid + i * NT;
            if (l < nt) Bb[l] = Bst[l];           // buffer 0 holds the B of step 0
            if (l < nt_upd) {
                const int* r = trst + 5 * l;
                r1[i] = (uint32_t)r[1];
                r2[i] = (uint32_t)r[2];
                r3[i] = (uint32_t)r[3];
                cb[i] = __int_as_float(r[4]);
                bv[i] = Bst[l];
                const uint32_t e0 = (r2[i] >> 14) & 0x1FFFu, e1 = r3[i] & 0x1FFFu, e2 = (r3[i] >> 16) & 0x1FFFu;
                const int k0 = est[2 * e0 + 1], k1 = est[2 * e1 + 1], k2 = est[2 * e2 + 1];
                c0[i] = flip(fabsf(__int_as_float(k0)), (r3[i] >> 13) & 1u);
                c1[i] = flip(fabsf(__int_as_float(k1)), (r3[i] >> 14) & 1u);
                c2[i] = flip(fabsf(__int_as_float(k2)), (r3[i] >> 29) & 1u);
                v0[i] = Ust[e0];
                v1[i] = flip(Ust[e1], (r2[i] >> 27) & 1u);
                v2[i] = flip(Ust[e2], (r2[i] >> 28) & 1u);
                if (has_src) {
                    const uint32_t f = (k0 < 0 ? 1u : 0u) | (k1 < 0 ? 2u : 0u) | (k2 < 0 ? 4u : 0u);
                    if (f) {
                        // positions of this triangle's source edges in the tile's list (sorted
                        // by local edge), 10 bits each
                        const uint32_t e[3] = {e0, e1, e2};
                        uint32_t pk = 0;
                        for (int q = 0; q < 3; ++q) {
                            if (!((f >> q) & 1u)) continue;
                            int lo = 0, hi = h[9];
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if ((uint32_t)__ldg(&a.tsrc[h[8] + mid].x) < e[q]) lo = mid + 1;
                                else hi = mid;
                            }
                            pk |= (uint32_t)lo << (10 * q);
                        }
                        spos[l] = (int)pk;
                        srcm |= f << (3 * i);
                    }
                }
            }
        }
        __syncthreads();   // staging read, buffer 0 written
        if (has_next) issue_records(slot1);
        if (has_next2) issue_header(tile + 2 * stride, slot2);
        const int s_fields = kk < 3 ? kk : 3;
#pragma unroll 1
        for (int s = 1; s <= kk; ++s) {
            const int tend = h[16 + kk - s];
            const uint32_t bo = (s & 1) ? bb0 : bb1;
            float* Bn = Bb + ((s & 1) ? Lay::TLC : 0);
            
#pragma unroll
            for (int i = 0; i < TS; ++i) {
                if (tid + i * NT < tend) {
                    const float b = bv[i];
                    v0[i] = rn_fma(c0[i], rn_sub(b, lds32(bo + (r1[i] & 0xFFFFu))), v0[i]);
                    v1[i] = rn_fma(c1[i], rn_sub(b, lds32(bo + (r1[i] >> 16))), v1[i]);
                    v2[i] = rn_fma(c2[i], rn_sub(b, lds32(bo + (r2[i] & 0x3FFFu))), v2[i]);
                }
            }
            if (srcm) {
#pragma unroll
                for (int i = 0; i < TS; ++i) {
                    const uint32_t f = (srcm >> (3 * i)) & 7u;
                    if (f && tid + i * NT < tend) {
                        const uint32_t pk = (uint32_t)spos[tid + i * NT];
                        for (int q = 0; q < 3; ++q) {
                            if (!((f >> q) & 1u)) continue;
                            const int2 e = __ldg(a.tsrc + h[8] + ((pk >> (10 * q)) & 0x3FFu));
                            const float g = (float)__ldg(a.gtab + (size_t)__ldg(a.src_grp + e.y) * a.gstride +
                                                         a.gbase + s - 1);
                            const float sc = __ldg(a.src_c + e.y);
                            if (q == 0) v0[i] = rn_fma(sc, g, v0[i]);
                            if (q == 1) v1[i] = rn_fma(flip(sc, (r2[i] >> 27) & 1u), g, v1[i]);
                            if (q == 2) v2[i] = rn_fma(flip(sc, (r2[i] >> 28) & 1u), g, v2[i]);
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < TS; ++i) {
                if (tid + i * NT < tend) {
                    bv[i] = rn_fma(cb[i], rn_add(rn_add(v0[i], v1[i]), v2[i]), bv[i]);
                    Bn[tid + i * NT] = bv[i];
                }
            }

            __syncthreads();
            if (has_next && s == s_fields) {
                if (!wait_bar(&bar_r, ph_r)) break;
                issue_fields(slot1);
            }
        }
        if (!ok) break;
        // write-back: B of the owned triangles from registers; U of the owned edges through
        // the B buffers (free now), each written by its owned triangles
        const int nto = h[1], neo = h[3];
        float* Uw = Bb;
#pragma unroll
        for (int i = 0; i < TS; ++i) {
            const int l = tid + i * NT;
            if (l < nto) {
                a.Bout[h[0] + l] = bv[i];
                Uw[(r2[i] >> 14) & 0x1FFFu] = v0[i];
                Uw[r3[i] & 0x1FFFu] = flip(v1[i], (r2[i] >> 27) & 1u);
                Uw[(r3[i] >> 16) & 0x1FFFu] = flip(v2[i], (r2[i] >> 28) & 1u);
            }
        }
        __syncthreads();
        for (int l = tid; l < neo; l += NT) a.Uout[h[2] + l] = Uw[l];
        if (has_next) cp_async_wait_all();
        if (has_next2 && !wait_bar(&bar_h, ph_h)) break;
        __syncthreads();
    }
    if (!ok) {
        atomicOr(a.err, 1u);
        cp_async_wait_all();
        for (; pend_r > 0; --pend_r, ph_r ^= 1u) mbar_wait(&bar_r, ph_r);
        for (; pend_h > 0; --pend_h, ph_h ^= 1u) mbar_wait(&bar_h, ph_h);
    }
    if (tid == 0) {
        __threadfence();
        const unsigned t = atomicAdd(a.done, 1u);
        if (t == gridDim.x - 1) {
            *a.step = n0 + a.ksteps;
            *a.done = 0u;
            __threadfence();
        }
    }
}

// A whole small mesh in one CTA: a single tile without a halo (every triangle and edge owned),
// advanced by n steps in one launch with everything in shared memory, by the fused step of
// k_tbf.  Records and fields are read once from global memory; g(t) of the source is evaluated
// in the kernel (the same source_g as the per-chunk table, so the same values).  For meshes
// whose step is a few microseconds of launches: the launch and the barrier latency are its
// whole cost.
struct TBF1Args {
    const int* hdr;
    const int* frec;
    const int* fedge;
    const int2* tsrc;
    const float* Bin;
    const float* Uin;
    float* Bout;
    float* Uout;
    const float* src_c;
    const int32_t* src_grp;
    const double* grp_par;   // per source group: dt, omega0, t0, tau
    long long* step;
    long long n_steps;
};

template <int NT, int TS>
__global__ void __launch_bounds__(NT, 1) k_tbf1(TBF1Args a) {
    constexpr int TLC = TS * NT;
    __shared__ __align__(16) float Bb[2 * TLC];
    __shared__ int spos[TLC];
    const int tid = threadIdx.x;
    const int* h = a.hdr;
    const int nt = h[4], nel = h[5];
    const int* fr = a.frec + 5 * (size_t)h[11];
    const int* fe = a.fedge + 2 * (size_t)h[12];
    const uint32_t bb0 = smem_addr(Bb), bb1 = bb0 + 4u * TLC;
    const long long n0 = *a.step;
    uint32_t r1[TS], r2[TS], r3[TS], srcm = 0;
    float v0[TS], v1[TS], v2[TS], c0[TS], c1[TS], c2[TS], cb[TS], bv[TS];
    auto edge_c = [&](uint32_t e) { return e < (uint32_t)nel ? __ldg(fe + 2 * e + 1) : 0; };
    auto edge_u = [&](uint32_t e) { return e < (uint32_t)nel ? __ldg(a.Uin + __ldg(fe + 2 * e)) : 0.f; };
#pragma unroll
    for (int i = 0; i < TS; ++i) {
        const int l = tid + i * NT;
        if (l < nt) {
            const int* r = fr + 5 * l;
            r1[i] = (uint32_t)__ldg(r + 1);
            r2[i] = (uint32_t)__ldg(r + 2);
            r3[i] = (uint32_t)__ldg(r + 3);
            cb[i] = __int_as_float(__ldg(r + 4));
            bv[i] = __ldg(a.Bin + __ldg(r));
            Bb[l] = bv[i];
            const uint32_t e0 = (r2[i] >> 14) & 0x1FFFu, e1 = r3[i] & 0x1FFFu, e2 = (r3[i] >> 16) & 0x1FFFu;
            const int k0 = edge_c(e0), k1 = edge_c(e1), k2 = edge_c(e2);
            c0[i] = flip(fabsf(__int_as_float(k0)), (r3[i] >> 13) & 1u);
            c1[i] = flip(fabsf(__int_as_float(k1)), (r3[i] >> 14) & 1u);
            c2[i] = flip(fabsf(__int_as_float(k2)), (r3[i] >> 29) & 1u);
            v0[i] = edge_u(e0);
            v1[i] = flip(edge_u(e1), (r2[i] >> 27) & 1u);
            v2[i] = flip(edge_u(e2), (r2[i] >> 28) & 1u);
            const uint32_t f = (k0 < 0 ? 1u : 0u) | (k1 < 0 ? 2u : 0u) | (k2 < 0 ? 4u : 0u);
            if (f && h[9] > 0) {
                const uint32_t e[3] = {e0, e1, e2};
                uint32_t pk = 0;
                for (int q = 0; q < 3; ++q) {
                    if (!((f >> q) & 1u)) continue;
                    int lo = 0, hi = h[9];
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if ((uint32_t)__ldg(&a.tsrc[h[8] + mid].x) < e[q]) lo = mid + 1;
                        else hi = mid;
                    }
                    pk |= (uint32_t)lo << (10 * q);
                }
                spos[l] = (int)pk;
                srcm |= f << (3 * i);
            }
        }
    }
    __syncthreads();
#pragma unroll 1
    for (long long s = 0; s < a.n_steps; ++s) {
        const uint32_t bo = (s & 1) ? bb1 : bb0;
        float* Bn = Bb + ((s & 1) ? 0 : TLC);
#pragma unroll
        for (int i = 0; i < TS; ++i) {
            const int l = tid + i * NT;
            if (l < nt) {
                const float n0v = lds32(bo + (r1[i] & 0xFFFFu));
                const float n1v = lds32(bo + (r1[i] >> 16));
                const float n2v = lds32(bo + (r2[i] & 0x3FFFu));
                const float b = bv[i];
                v0[i] = rn_fma(c0[i], rn_sub(b, n0v), v0[i]);
                v1[i] = rn_fma(c1[i], rn_sub(b, n1v), v1[i]);
                v2[i] = rn_fma(c2[i], rn_sub(b, n2v), v2[i]);
                if (((srcm >> (3 * i)) & 7u) != 0u) {
                    const uint32_t f = (srcm >> (3 * i)) & 7u, pk = (uint32_t)spos[l];
                    for (int q = 0; q < 3; ++q) {
                        if (!((f >> q) & 1u)) continue;
                        const int2 e = __ldg(a.tsrc + h[8] + ((pk >> (10 * q)) & 0x3FFu));
                        const double* par = a.grp_par + 4 * (size_t)__ldg(a.src_grp + e.y);
                        const float g = (float)source_g(n0 + s, par[0], par[1], par[2], par[3]);
                        const float sc = __ldg(a.src_c + e.y);
                        if (q == 0) v0[i] = rn_fma(sc, g, v0[i]);
                        if (q == 1) v1[i] = rn_fma(flip(sc, (r2[i] >> 27) & 1u), g, v1[i]);
                        if (q == 2) v2[i] = rn_fma(flip(sc, (r2[i] >> 28) & 1u), g, v2[i]);
                    }
                }
                bv[i] = rn_fma(cb[i], rn_add(rn_add(v0[i], v1[i]), v2[i]), b);
                Bn[l] = bv[i];
            }
        }
        __syncthreads();
    }
    // write-back: every triangle and edge is owned
    float* Uw = Bb;
#pragma unroll
    for (int i = 0; i < TS; ++i) {
        const int l = tid + i * NT;
        if (l < nt) {
            a.Bout[h[0] + l] = bv[i];
            Uw[(r2[i] >> 14) & 0x1FFFu] = v0[i];
            Uw[r3[i] & 0x1FFFu] = flip(v1[i], (r2[i] >> 27) & 1u);
            Uw[(r3[i] >> 16) & 0x1FFFu] = flip(v2[i], (r2[i] >> 28) & 1u);
        }
    }
    __syncthreads();
    for (int l = tid; l < h[3]; l += NT) a.Uout[h[2] + l] = Uw[l];
    if (tid == 0) *a.step = n0 + a.n_steps;
}

// -s0 dt/S of each fused triangle record (r4) and dt|e|/d with the source flag of each edge
// record, from the mesh's coefficient arrays; the zero-slot and padding records keep 0.
__global__ void k_tbf_fill(int* __restrict__ frec, int64_t n_frec, int* __restrict__ fedge, int64_t n_fedge,
                           const int4* __restrict__ tri, const float* __restrict__ cU) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_frec) {
        const int* r = frec + 5 * i;
        const float c = __int_as_float(tri[r[0]].w);
        frec[5 * i + 4] = __float_as_int(((uint32_t)r[2] >> 29) & 1u ? c : -c);
    }
    if (i < n_fedge) {
        const int g = fedge[2 * i];
        if (g >= 0) fedge[2 * i + 1] = __float_as_int(cU[g]);   // zero slot, padding: gid -1, 0
    }
}

}  // namespace

bool tbf_fits(int max_tri_loc, int max_edge_loc, int max_src) {
    return max_tri_loc <= TbfLayout<512, 8>::TLC && max_edge_loc + 1 <= TbfLayout<512, 8>::ELC &&
           max_src < 1024 && TbfLayout<512, 8>::SMEM <= 227 * 1024 - 1024;
}

cudaError_t launch_tbf_fill(const TBDev& t, const DevMesh& m, cudaStream_t s) {
    const int64_t n = t.n_frec > t.n_fedge ? t.n_frec : t.n_fedge;
    if (n == 0) return cudaSuccess;
    k_tbf_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t.frec, t.n_frec, t.fedge, t.n_fedge, m.tri,
                                                         (const float*)m.cU);
    return cudaGetLastError();
}

bool tbf1_fits(const TBDev& t, const int* hdr_host) {
    // one tile that is the whole mesh (no halo), within one CTA's shared memory
    return t.n_tiles == 1 && t.frec && hdr_host[4] == hdr_host[1] && hdr_host[5] == hdr_host[3] &&
           hdr_host[4] <= 2048 && hdr_host[5] + 1 <= 2 * 2048 && t.max_src < 1024;
}

cudaError_t launch_tbf1(const TBDev& t, const DevMesh& m, long long n_steps, int cur, cudaStream_t s) {
    if (m.plasma || n_steps < 1) return cudaErrorInvalidValue;
    TBF1Args a;
    a.hdr = t.hdr;
    a.frec = t.frec;
    a.fedge = t.fedge;
    a.tsrc = t.tsrc;
    a.Bin = (const float*)t.B[cur];
    a.Uin = (const float*)t.U[cur];
    a.Bout = (float*)t.B[cur ^ 1];
    a.Uout = (float*)t.U[cur ^ 1];
    a.src_c = (const float*)m.src_c;
    a.src_grp = m.src_grp;
    a.grp_par = m.grp_par;
    a.step = m.step;
    a.n_steps = n_steps;
    k_tbf1<512, 4><<<1, 512, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tbf(const TBDev& t, const DevMesh& m, int ksteps, int cur, int gbase, cudaStream_t s) {
    if (ksteps < 1 || ksteps > 15 || m.plasma) return cudaErrorInvalidValue;
    TBFArgs a;
    a.hdr = t.hdr;
    a.frec = t.frec;
    a.fedge = t.fedge;
    a.tsrc = t.tsrc;
    a.Bin = (const float*)t.B[cur];
    a.Uin = (const float*)t.U[cur];
    a.Bout = (float*)t.B[cur ^ 1];
    a.Uout = (float*)t.U[cur ^ 1];
    a.src_c = (const float*)m.src_c;
    a.src_grp = m.src_grp;
    a.gtab = m.gtab;
    a.gstride = m.gtab_size;
    a.gbase = gbase;
    a.step = m.step;
    a.done = t.done;
    a.err = t.done + 1;
    a.ksteps = ksteps;
    a.test_cta = t.test_cta;
    using Lay = TbfLayout<512, 8>;
    auto kern = k_tbf<512, 8>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::SMEM);
    if (e != cudaSuccess) return e;
    const int nt = (int)t.n_tiles;
    const int grid = nt < t.sms ? nt : t.sms;
    kern<<<grid, 512, Lay::SMEM, s>>>(a, nt);
    return cudaGetLastError();
}

}  // namespace ue
