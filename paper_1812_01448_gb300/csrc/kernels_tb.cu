// Temporally blocked leap-frog: one CTA per KD tile advances its owned edges and triangles by
// k steps (eqs. 14-15 with eqs. 3-6) in shared memory, recomputing the k-ring halo that the
// neighbouring tiles own.  The paper's "Divide and conqueror" partitions exchange boundary
// values every step; here the exchange is replaced by redundant halo work inside one launch.
//
// Per launch a tile reads its records (static: 16 B per local triangle, 12 B per local edge,
// plus 4 B per local edge of plasma coefficient) and the fields of its local set from the "in"
// buffers, and writes only the owned values to the "out" buffers (double buffering, so that
// neighbours still read time level n).  Every arithmetic operation repeats the plain kernels'
// sequence of correctly rounded operations (device.cuh rn_* helpers and the shared source_g),
// so the results are bit-identical to the plain two-kernel step.
#include <cuda_runtime.h>

#include "device.cuh"

namespace ue {

namespace {

constexpr int kNT = 512;

struct TBArgs {
    const int* hdr;
    const int4* trec;
    const int* erec;    // 3 ints per local edge record: gid, R | L << 16, bits of cU (sign: source)
    const float* epb;   // plasma coefficient per local edge record
    const int2* tsrc;
    const float* Bin;
    const float* Uin;
    const float* Jin;
    float* Bout;
    float* Uout;
    float* Jout;
    const float* src_c;
    const int32_t* src_grp;
    const double* gtab;
    int gstride;
    int gbase;
    long long* step;
    unsigned* done;
    unsigned* err;      // set when a bounded copy wait of k_tbp runs out
    int ksteps;
    float pa, mdt;
    int test_cta;       // tests only (-1 otherwise): this CTA arms its first record copy for
                        // 16 bytes more than it delivers, so that the wait for it runs out
};


// NT threads; each thread owns local triangle slots tid + i*NT (i < TS) and local edge slots
// tid + i*NT (i < ES), whose records it keeps in registers for all k steps.  In every phase a
// thread takes its slots kG at a time: it issues the group's shared-memory gathers, then
// computes and stores, so that a group's loads are in flight together (kG = 1: slot by slot,
// which measured best for the largest slot counts).
template <int NT, int TS, int ES, int MINB, int kG, bool PLASMA, bool SRC>
__global__ void __launch_bounds__(NT, MINB) k_tb(TBArgs a) {
    extern __shared__ float sm[];
    __shared__ int h[48];
    const int tid = threadIdx.x;
    if (tid < 48) h[tid] = a.hdr[(size_t)blockIdx.x * 48 + tid];
    __syncthreads();
    const int ntl = h[4], nel = h[5];
    float* Bl = sm;
    float* Ul = sm + ntl;
    float* Jl = Ul + nel + 1;

    int tc01[TS], tc2[TS];
    float tcb[TS];
    int erl[ES];
    float ecu[ES], epb[ES];
    const int4* tr = a.trec + h[6];
    const int* er = a.erec + 3 * (size_t)h[7];
#pragma unroll
    for (int i = 0; i < TS; ++i) {
        const int l = tid + i * NT;
        if (l < ntl) {
            const int4 r = __ldg(tr + l);
            tc01[i] = r.y;
            tc2[i] = r.z;
            tcb[i] = __int_as_float(r.w);
            Bl[l] = __ldg(a.Bin + r.x);
        }
    }
#pragma unroll
    for (int i = 0; i < ES; ++i) {
        const int l = tid + i * NT;
        if (l < nel) {
            const int gid = __ldg(er + 3 * l);
            erl[i] = __ldg(er + 3 * l + 1);
            ecu[i] = fabsf(__int_as_float(__ldg(er + 3 * l + 2)));
            Ul[l] = __ldg(a.Uin + gid);
            if constexpr (PLASMA) {
                epb[i] = __ldg(a.epb + h[7] + l);
                Jl[l] = __ldg(a.Jin + gid);
            }
        }
    }
    if (tid == 0) {
        Ul[nel] = 0.f;
        if constexpr (PLASMA) Jl[nel] = 0.f;
    }
    const long long n0 = *a.step;
    __syncthreads();

    for (int s = 1; s <= a.ksteps; ++s) {
        const int lim = a.ksteps - s;
        const int eend = h[32 + lim];
#pragma unroll
        for (int g0 = 0; g0 < ES; g0 += kG) {
            float bR[kG], bL[kG], uo[kG], jo[kG];
#pragma unroll
            for (int q = 0; q < kG; ++q) {
                const int i = g0 + q, l = tid + i * NT;
                if (i < ES && l < eend) {
                    bR[q] = Bl[erl[i] & 0xFFFF];
                    bL[q] = Bl[(unsigned)erl[i] >> 16];
                    uo[q] = Ul[l];
                    if constexpr (PLASMA) jo[q] = Jl[l];
                }
            }
#pragma unroll
            for (int q = 0; q < kG; ++q) {
                const int i = g0 + q, l = tid + i * NT;
                if (i < ES && l < eend) {
                    float un = rn_fma(ecu[i], rn_sub(bR[q], bL[q]), uo[q]);
                    if constexpr (PLASMA) {
                        const float jn = rn_fma(a.pa, jo[q], rn_mul(epb[i], uo[q]));
                        Jl[l] = jn;
                        un = rn_fma(a.mdt, jn, un);
                    }
                    Ul[l] = un;
                }
            }
        }
        if constexpr (SRC) {
            if (h[9] > 0) {
                __syncthreads();
                for (int i = tid; i < h[9]; i += NT) {
                    const int2 q = __ldg(a.tsrc + h[8] + i);
                    if (q.x < eend) {
                        const float g = (float)__ldg(a.gtab + (size_t)__ldg(a.src_grp + q.y) * a.gstride +
                                                     a.gbase + s - 1);
                        Ul[q.x] = rn_fma(__ldg(a.src_c + q.y), g, Ul[q.x]);
                    }
                }
            }
        }
        __syncthreads();
        const int tend = h[16 + lim];
#pragma unroll
        for (int g0 = 0; g0 < TS; g0 += kG) {
            float u0[kG], u1[kG], u2[kG], bo[kG];
#pragma unroll
            for (int q = 0; q < kG; ++q) {
                const int i = g0 + q, l = tid + i * NT;
                if (i < TS && l < tend) {
                    const int c0 = tc01[i] & 0xFFFF, c1 = (unsigned)tc01[i] >> 16, c2 = tc2[i];
                    u0[q] = Ul[c0 >> 1];
                    u1[q] = Ul[c1 >> 1];
                    u2[q] = Ul[c2 >> 1];
                    bo[q] = Bl[l];
                }
            }
#pragma unroll
            for (int q = 0; q < kG; ++q) {
                const int i = g0 + q, l = tid + i * NT;
                if (i < TS && l < tend) {
                    const int c0 = tc01[i], c1 = (unsigned)tc01[i] >> 16, c2 = tc2[i];
                    const float x0 = (c0 & 1) ? -u0[q] : u0[q];
                    const float x1 = (c1 & 1) ? -u1[q] : u1[q];
                    const float x2 = (c2 & 1) ? -u2[q] : u2[q];
                    Bl[l] = rn_fma(-tcb[i], rn_add(rn_add(x0, x1), x2), bo[q]);
                }
            }
        }
        __syncthreads();
    }
    const int nto = h[1], neo = h[3];
#pragma unroll
    for (int i = 0; i < TS; ++i) {
        const int l = tid + i * NT;
        if (l < nto) a.Bout[h[0] + l] = Bl[l];
    }
#pragma unroll
    for (int i = 0; i < ES; ++i) {
        const int l = tid + i * NT;
        if (l < neo) {
            a.Uout[h[2] + l] = Ul[l];
            if constexpr (PLASMA) a.Jout[h[2] + l] = Jl[l];
        }
    }
    // the last CTA to finish advances the step counter (every CTA has read it by then)
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

// Shared-memory-record form: the tile's records are staged in shared memory next to its
// fields, so that registers stay few and 1024 threads (or two CTAs) fit per SM.  Threads
// stride over the local elements, two at a time (gathers of both issued before either store).
template <bool PLASMA, bool SRC>
__global__ void __launch_bounds__(1024, 1) k_tbs(TBArgs a) {
    constexpr int NT = 1024;
    extern __shared__ float sm[];
    __shared__ int h[48];
    const int tid = threadIdx.x;
    if (tid < 48) h[tid] = a.hdr[(size_t)blockIdx.x * 48 + tid];
    __syncthreads();
    const int ntl = h[4], nel = h[5];
    float* Bl = sm;
    float* Ul = Bl + ntl;
    float* Jl = Ul + nel + 1;
    int2* Tc = reinterpret_cast<int2*>(Ul + (PLASMA ? 2 * (nel + 1) : nel + 1) + 1);   // 8-B aligned below
    Tc = reinterpret_cast<int2*>((reinterpret_cast<uintptr_t>(Tc) + 7) & ~uintptr_t(7));
    float* Tb = reinterpret_cast<float*>(Tc + ntl);
    int* Erl = reinterpret_cast<int*>(Tb + ntl);
    float* Ecu = reinterpret_cast<float*>(Erl + nel);
    float* Epb = Ecu + nel;
    const int4* tr = a.trec + h[6];
    const int* er = a.erec + 3 * (size_t)h[7];
    for (int l = tid; l < ntl; l += NT) {
        const int4 r = __ldg(tr + l);
        Tc[l] = make_int2(r.y, r.z);
        Tb[l] = __int_as_float(r.w);
        Bl[l] = __ldg(a.Bin + r.x);
    }
    for (int l = tid; l < nel; l += NT) {
        const int gid = __ldg(er + 3 * l);
        Erl[l] = __ldg(er + 3 * l + 1);
        Ecu[l] = fabsf(__int_as_float(__ldg(er + 3 * l + 2)));
        Ul[l] = __ldg(a.Uin + gid);
        if constexpr (PLASMA) {
            Epb[l] = __ldg(a.epb + h[7] + l);
            Jl[l] = __ldg(a.Jin + gid);
        }
    }
    if (tid == 0) {
        Ul[nel] = 0.f;
        if constexpr (PLASMA) Jl[nel] = 0.f;
    }
    const long long n0 = *a.step;
    __syncthreads();
    for (int s = 1; s <= a.ksteps; ++s) {
        const int lim = a.ksteps - s;
        const int eend = h[32 + lim];
        for (int l0 = tid; l0 < eend; l0 += 2 * NT) {
            const int l1 = l0 + NT;
            const bool v1 = l1 < eend;
            const int r0 = Erl[l0], r1 = v1 ? Erl[l1] : 0;
            const float a0 = Bl[r0 & 0xFFFF], b0 = Bl[(unsigned)r0 >> 16], u0 = Ul[l0];
            const float a1 = Bl[r1 & 0xFFFF], b1 = Bl[(unsigned)r1 >> 16], u1 = v1 ? Ul[l1] : 0.f;
            float j0 = 0.f, j1 = 0.f;
            if constexpr (PLASMA) {
                j0 = Jl[l0];
                if (v1) j1 = Jl[l1];
            }
            float n0v = rn_fma(Ecu[l0], rn_sub(a0, b0), u0);
            if constexpr (PLASMA) {
                const float jn = rn_fma(a.pa, j0, rn_mul(Epb[l0], u0));
                Jl[l0] = jn;
                n0v = rn_fma(a.mdt, jn, n0v);
            }
            Ul[l0] = n0v;
            if (v1) {
                float n1v = rn_fma(Ecu[l1], rn_sub(a1, b1), u1);
                if constexpr (PLASMA) {
                    const float jn = rn_fma(a.pa, j1, rn_mul(Epb[l1], u1));
                    Jl[l1] = jn;
                    n1v = rn_fma(a.mdt, jn, n1v);
                }
                Ul[l1] = n1v;
            }
        }
        if constexpr (SRC) {
            if (h[9] > 0) {
                __syncthreads();
                for (int i = tid; i < h[9]; i += NT) {
                    const int2 q = __ldg(a.tsrc + h[8] + i);
                    if (q.x < eend) {
                        const float g = (float)__ldg(a.gtab + (size_t)__ldg(a.src_grp + q.y) * a.gstride +
                                                     a.gbase + s - 1);
                        Ul[q.x] = rn_fma(__ldg(a.src_c + q.y), g, Ul[q.x]);
                    }
                }
            }
        }
        __syncthreads();
        const int tend = h[16 + lim];
        for (int l0 = tid; l0 < tend; l0 += 2 * NT) {
            const int l1 = l0 + NT;
            const bool v1 = l1 < tend;
            const int2 c0 = Tc[l0];
            const int2 c1 = v1 ? Tc[l1] : make_int2(nel << 1 | (nel << 17), nel << 1);
            const int p0 = c0.x & 0xFFFF, q0 = (unsigned)c0.x >> 16, w0 = c0.y;
            const int p1 = c1.x & 0xFFFF, q1 = (unsigned)c1.x >> 16, w1 = c1.y;
            const float x0 = Ul[p0 >> 1], y0 = Ul[q0 >> 1], z0 = Ul[w0 >> 1], bo0 = Bl[l0];
            const float x1 = Ul[p1 >> 1], y1 = Ul[q1 >> 1], z1 = Ul[w1 >> 1];
            const float bo1 = v1 ? Bl[l1] : 0.f;
            const float s0 = rn_add(rn_add((p0 & 1) ? -x0 : x0, (q0 & 1) ? -y0 : y0), (w0 & 1) ? -z0 : z0);
            Bl[l0] = rn_fma(-Tb[l0], s0, bo0);
            if (v1) {
                const float s1 = rn_add(rn_add((p1 & 1) ? -x1 : x1, (q1 & 1) ? -y1 : y1), (w1 & 1) ? -z1 : z1);
                Bl[l1] = rn_fma(-Tb[l1], s1, bo1);
            }
        }
        __syncthreads();
    }
    for (int l = tid; l < h[1]; l += NT) a.Bout[h[0] + l] = Bl[l];
    for (int l = tid; l < h[3]; l += NT) {
        a.Uout[h[2] + l] = Ul[l];
        if constexpr (PLASMA) a.Jout[h[2] + l] = Jl[l];
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

// Pipelined persistent form: one CTA per SM walks the tiles blockIdx.x, blockIdx.x + gridDim.x,
// ...  Global loads run ahead of the steps:
// - headers: a ring of three; tile i+2's header is copied (TMA bulk copy) while tile i steps;
// - records: tile i+1's records are copied (TMA bulk copies) into a staging area as soon as
//   tile i has moved its own records from there into registers;
// - fields: after step min(3, k) of tile i, tile i+1's fields are gathered (4-byte cp.async)
//   into the second field buffer.
// A launch of kk < k_max steps stages and gathers only the rings it reads: triangles of level
// <= kk and edges of level <= kk - 1.
//
// Each thread keeps, for its slots (local element tid + i*NT), the element's current value (B,
// U, and J in plasma media) and its record in registers; shared memory holds the values that
// other threads gather.  So a half-step per element is its gathers, the arithmetic and one
// store.  Records are turned into byte offsets of the gathered values once per tile, and the
// signs of eq. 4 into the coefficients: with x_q = s_q U_q,
//   rn(rn(x0 + x1) + x2) = s0 rn(rn(U0 + s0 s1 U1) + s0 s2 U2)
// because round-to-nearest is odd (rn(-y) = -rn(y)), so
//   B - (dt/S) rn(rn(x0 + x1) + x2) = fma(-s0 dt/S, rn(rn(U0 + s0 s1 U1) + s0 s2 U2), B)
// rounds exactly as the plain kernel's select-and-add does; the signs s0 s1 and s0 s2 ride in
// bits 31 and 30 of the third gather offset and flip the gathered values' sign bits.  Gathers of G slots are issued
// before any of their stores.  The field buffers sit at compile-time offsets (capacity TS*NT
// triangles and ES*NT edges); a gather is one shift or mask, one add to the buffer's 32-bit
// shared address and one shared load.
// Dynamic shared memory: two field buffers of FB floats (B at 0, U at TLC, J at JOFF), then
// the staging records (TLC triangle records, ELC edge records, ELC plasma coefficients).
template <int NT, int TS, int ES, bool PLASMA>
struct TbpLayout {
    static constexpr int TLC = TS * NT;                      // local triangle capacity
    static constexpr int ELC = ES * NT;                      // local edge capacity
    static constexpr int UOFF = TLC;                         // U in a field buffer (floats)
    static constexpr int JOFF = TLC + ELC + 4;               // J in a field buffer (plasma)
    static constexpr int FB = PLASMA ? JOFF + ELC : TLC + ELC + 4;
    static constexpr size_t TSTAGE = 2 * 4 * (size_t)FB;     // byte offsets in shared memory
    static constexpr size_t ESTAGE = TSTAGE + 16 * (size_t)TLC;
    static constexpr size_t PSTAGE = ESTAGE + 12 * (size_t)ELC;
    static constexpr size_t SMEM = PSTAGE + (PLASMA ? 4 * (size_t)ELC : 0);
    static_assert(4 * (TLC + ELC + 1) < 65536, "byte offsets must fit 16 bits");
    static_assert(FB % 4 == 0 && ELC % 4 == 0, "16-byte aligned buffers and staging");
};

// Shared-memory load at a 32-bit shared address (the buffer's address plus a byte offset).  The
// gathers of a phase read values that a barrier separates from their stores, so the loads may
// move freely among the phase's own stores (which go to other elements).
__device__ __forceinline__ float lds_at(uint32_t base, unsigned off) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(base + off));
    return v;
}

template <int NT, int TS, int ES, int G, bool PLASMA, bool SRC>
__global__ void __launch_bounds__(NT, 1) k_tbp(TBArgs a, int n_tiles) {
    using Lay = TbpLayout<NT, TS, ES, PLASMA>;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ __align__(16) int hs[3][48];
    __shared__ __align__(8) uint64_t bar_h, bar_r;
    const int tid = threadIdx.x;
    const int stride = gridDim.x;
    const int kk = a.ksteps;
    float* F0 = reinterpret_cast<float*>(smraw);
    int4* tstage = reinterpret_cast<int4*>(smraw + Lay::TSTAGE);
    int* estage = reinterpret_cast<int*>(smraw + Lay::ESTAGE);
    float* pstage = reinterpret_cast<float*>(smraw + Lay::PSTAGE);
    if (tid == 0) {
        mbar_init(&bar_h, 1);
        mbar_init(&bar_r, 1);
        fence_mbar_init();
    }
    __syncthreads();
    long long n0 = 0;   // the step counter, read once the previous launch has finished
    uint32_t ph_h = 0, ph_r = 0;
    int pend_h = 0, pend_r = 0;   // bulk copies issued and not yet waited for (uniform)
    bool ok = true;
    // a wait that runs out ends this CTA's work: every thread agrees on it before any staged
    // value is used, and the copies in flight are waited for (bounded) before the CTA exits
    auto wait_bar = [&](uint64_t* bar, uint32_t& ph) {
        if (!mbar_wait(bar, ph)) ok = false;
        ph ^= 1u;
        if (bar == &bar_h) --pend_h;
        else --pend_r;
        ok = __syncthreads_and(ok ? 1 : 0) != 0;
        return ok;
    };
    // local triangles of level <= kk, local edges of level <= kk - 1 (header layout in
    // tiles_host.cpp)
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
            const uint32_t ne4 = (uint32_t)(n_edge(h) + 3) & ~3u;
            const uint32_t tb = 16u * (uint32_t)n_tri(h), eb = 12u * ne4, pbb = PLASMA ? 4u * ne4 : 0u;
            fence_proxy_async();
            mbar_expect_tx(&bar_r, tb + eb + pbb + (extra ? 16u : 0u));
            if (tb) bulk_copy_g2s(tstage, a.trec + h[6], tb, &bar_r);
            if (eb) bulk_copy_g2s(estage, a.erec + 3 * (size_t)h[7], eb, &bar_r);
            if (PLASMA && pbb) bulk_copy_g2s(pstage, a.epb + h[7], pbb, &bar_r);
        }
    };
    auto issue_fields = [&](int slot, float* Fn) {
        const int* h = hs[slot];
        const int nt = n_tri(h), ne = n_edge(h);
#pragma unroll
        for (int i = 0; i < TS; ++i) {
            const int l = tid + i * NT;
            if (l < nt) cp_async4(Fn + l, a.Bin + tstage[l].x);
        }
#pragma unroll
        for (int i = 0; i < ES; ++i) {
            const int l = tid + i * NT;
            if (l < ne) {
                const int g = estage[3 * l];
                cp_async4(Fn + Lay::UOFF + l, a.Uin + g);
                if constexpr (PLASMA) cp_async4(Fn + Lay::JOFF + l, a.Jin + g);
            }
        }
        if (tid == 0) Fn[Lay::UOFF + h[5]] = 0.f;   // the zero slot of boundary edges
        cp_async_commit();
    };
    int tile = blockIdx.x, it = 0;
    // prologue: first tile's header, records and fields; the second tile's header
    if (tile < n_tiles) {
        issue_header(tile, 0);
        if (wait_bar(&bar_h, ph_h)) {
            issue_records(0);
            if (tile + stride < n_tiles) issue_header(tile + stride, 1);
            if (wait_bar(&bar_r, ph_r)) {
                // headers and records are static: the fields and the step counter come from the
                // previous launch, which may still be finishing (programmatic dependent launch)
                grid_dependency_wait();
                n0 = *a.step;
                issue_fields(0, F0);
                cp_async_wait_all();
                if (tile + stride < n_tiles) wait_bar(&bar_h, ph_h);
            }
        }
    }
    if (tile >= n_tiles || !ok) {
        grid_dependency_wait();
        n0 = *a.step;
    }
    if (!ok) tile = n_tiles;
    __syncthreads();
    // per slot: triangle gather offsets (U0 | U1 << 16, U2 | signs s0 s1, s0 s2 in bits 31, 30),
    // -s0 dt/S and B;
    // edge gather offsets (B_lo | B_hi << 16), +-dt|e|/d and U (plasma: pb and J)
    unsigned toff[TS], toff2[TS];
    float tcb[TS], tb[TS];
    unsigned erl[ES];
    float ecu[ES], eu[ES], epb[ES], ej[ES];
    unsigned srcm = 0;

    for (int cur = 0; tile < n_tiles; tile += stride, ++it, cur ^= 1) {
        float* Fc = F0 + cur * Lay::FB;
        float* Fn = F0 + (cur ^ 1) * Lay::FB;
        const uint32_t Fcb = smem_addr(Fc);
        const bool has_next = tile + stride < n_tiles, has_next2 = tile + 2 * stride < n_tiles;
        // this CTA's last tile: the next launch may start its static loads on SMs that free up
        if (!has_next && tid == 0) grid_dependents_launch();
        const int slot = it % 3, slot1 = (it + 1) % 3, slot2 = (it + 2) % 3;
        const int* h = hs[slot];
        const int nt_upd = h[16 + kk - 1], ne = n_edge(h);
#pragma unroll
        for (int i = 0; i < TS; ++i) {
            const int l = tid + i * NT;
            if (l < nt_upd) {
                const int4 r = tstage[l];
                const unsigned c0 = (unsigned)r.y & 0xFFFFu, c1 = (unsigned)r.y >> 16, c2 = (unsigned)r.z;
                toff[i] = (4u * (Lay::UOFF + (c0 >> 1))) | ((4u * (Lay::UOFF + (c1 >> 1))) << 16);
                toff2[i] = (4u * (Lay::UOFF + (c2 >> 1))) | (((c0 ^ c1) & 1u) << 31) | (((c0 ^ c2) & 1u) << 30);
                const float cb = __int_as_float(r.w);
                tcb[i] = (c0 & 1u) ? cb : -cb;
                tb[i] = Fc[l];
            }
        }
        if constexpr (SRC) srcm = 0;
#pragma unroll
        for (int i = 0; i < ES; ++i) {
            const int l = tid + i * NT;
            if (l < ne) {
                // the edge's triangles in slot order (lo, hi): one gather of a warp then reads
                // the lower-numbered triangles of 32 consecutive edges and the other the higher
                // ones, two narrow windows of slots with fewer bank conflicts than R and L,
                // which mix both; where R is the higher slot the coefficient changes sign,
                // since rn(B_lo - B_hi) = -rn(B_R - B_L) exactly
                const int cub = estage[3 * l + 2];
                const unsigned w = (unsigned)estage[3 * l + 1], R = w & 0xFFFFu, L = w >> 16;
                erl[i] = (R < L ? (R | (L << 16)) : (L | (R << 16))) << 2;
                const float c = fabsf(__int_as_float(cub));
                ecu[i] = R > L ? -c : c;
                if constexpr (SRC) srcm |= (cub < 0 ? 1u : 0u) << i;
                eu[i] = Fc[Lay::UOFF + l];
                if constexpr (PLASMA) {
                    epb[i] = pstage[l];
                    ej[i] = Fc[Lay::JOFF + l];
                }
            }
        }
        __syncthreads();   // the staging area is free for the next tile's records
        if (has_next) issue_records(slot1);
        if (has_next2) issue_header(tile + 2 * stride, slot2);
        const int s_fields = kk < 3 ? kk : 3;
#pragma unroll 1
        for (int s = 1; s <= kk; ++s) {
            const int lim = kk - s;
            const int eend = h[32 + lim], tend = h[16 + lim];
            // E half-step (eq. 3; eqs. 5-6 in plasma media)
#pragma unroll
            for (int g0 = 0; g0 < ES; g0 += G) {
                float blo[G], bhi[G];
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    const int i = g0 + q;
                    if (i < ES && tid + i * NT < eend) {
                        blo[q] = lds_at(Fcb, erl[i] & 0xFFFFu);
                        bhi[q] = lds_at(Fcb, erl[i] >> 16);
                    }
                }
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    const int i = g0 + q;
                    if (i < ES && tid + i * NT < eend) {
                        const float uo = eu[i];
                        float un = rn_fma(ecu[i], rn_sub(blo[q], bhi[q]), uo);
                        if constexpr (PLASMA) {
                            const float jn = rn_fma(a.pa, ej[i], rn_mul(epb[i], uo));
                            ej[i] = jn;
                            un = rn_fma(a.mdt, jn, un);
                        }
                        eu[i] = un;
                        Fc[Lay::UOFF + tid + i * NT] = un;
                    }
                }
            }
            if constexpr (SRC) {
                if (h[9] > 0) {
                    __syncthreads();
                    for (int i = tid; i < h[9]; i += NT) {
                        const int2 q = __ldg(a.tsrc + h[8] + i);
                        if (q.x < eend) {
                            const float g = (float)__ldg(a.gtab + (size_t)__ldg(a.src_grp + q.y) * a.gstride +
                                                         a.gbase + s - 1);
                            Fc[Lay::UOFF + q.x] = rn_fma(__ldg(a.src_c + q.y), g, Fc[Lay::UOFF + q.x]);
                        }
                    }
                }
            }
            __syncthreads();
            if constexpr (SRC) {
                // source edges take their value back from shared memory
                if (srcm) {
#pragma unroll
                    for (int i = 0; i < ES; ++i)
                        if (((srcm >> i) & 1u) && tid + i * NT < eend) eu[i] = Fc[Lay::UOFF + tid + i * NT];
                }
            }
            // B half-step (eq. 4)
#pragma unroll
            for (int g0 = 0; g0 < TS; g0 += G) {
                float u0[G], u1[G], u2[G];
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    const int i = g0 + q;
                    if (i < TS && tid + i * NT < tend) {
                        u0[q] = lds_at(Fcb, toff[i] & 0xFFFFu);
                        u1[q] = lds_at(Fcb, toff[i] >> 16);
                        u2[q] = lds_at(Fcb, toff2[i] & 0xFFFFu);
                    }
                }
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    const int i = g0 + q;
                    if (i < TS && tid + i * NT < tend) {
                        const float x1 = __int_as_float(__float_as_int(u1[q]) ^ (int)(toff2[i] & 0x80000000u));
                        const float x2 = __int_as_float(__float_as_int(u2[q]) ^ (int)((toff2[i] << 1) & 0x80000000u));
                        const float t = rn_add(rn_add(u0[q], x1), x2);
                        tb[i] = rn_fma(tcb[i], t, tb[i]);
                        Fc[tid + i * NT] = tb[i];
                    }
                }
            }
            __syncthreads();
            if (has_next && s == s_fields) {
                if (!wait_bar(&bar_r, ph_r)) break;
                issue_fields(slot1, Fn);
            }
        }
        if (!ok) break;
        // owned values, from registers
        const int nto = h[1], neo = h[3];
#pragma unroll
        for (int i = 0; i < TS; ++i) {
            const int l = tid + i * NT;
            if (l < nto) a.Bout[h[0] + l] = tb[i];
        }
#pragma unroll
        for (int i = 0; i < ES; ++i) {
            const int l = tid + i * NT;
            if (l < neo) {
                a.Uout[h[2] + l] = eu[i];
                if constexpr (PLASMA) a.Jout[h[2] + l] = ej[i];
            }
        }
        if (has_next) cp_async_wait_all();
        if (has_next2 && !wait_bar(&bar_h, ph_h)) break;
        __syncthreads();
    }
    if (!ok) {
        // this CTA's tiles were not advanced: report it, and let its copies in flight land
        // before the CTA's shared memory goes (each wait bounded)
        atomicOr(a.err, 1u);
        cp_async_wait_all();
        for (; pend_r > 0; --pend_r, ph_r ^= 1u) mbar_wait(&bar_r, ph_r);
        for (; pend_h > 0; --pend_h, ph_h ^= 1u) mbar_wait(&bar_h, ph_h);
    }
    // the last CTA to finish advances the step counter (every CTA has read it by then)
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

// Fill the coefficient slots of the tile records from the global coefficient arrays: dt/S of
// each triangle record, dt|e|/d of each edge record with the source flag kept in its sign bit,
// and the plasma coefficient (pb may be NULL).  Padding records carry gid 0.
__global__ void k_tb_fill(int4* __restrict__ trec, int64_t n_trec, int* __restrict__ erec,
                          float* __restrict__ epb, int64_t n_erec, const int4* __restrict__ tri,
                          const float* __restrict__ cU, const float* __restrict__ pb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_trec) trec[i].w = tri[trec[i].x].w;
    if (i < n_erec) {
        const int g = erec[3 * i];
        erec[3 * i + 2] = __float_as_int(cU[g]);
        if (pb) epb[i] = pb[g];
    }
}

template <int NT, int TS, int ES, int MINB, int G, bool PLASMA, bool SRC>
cudaError_t launch_tb_t(const TBArgs& a, int n_tiles, size_t smem, cudaStream_t s) {
    auto kern = k_tb<NT, TS, ES, MINB, G, PLASMA, SRC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<n_tiles, NT, smem, s>>>(a);
    return cudaGetLastError();
}

// gathers issued together per group of slots in k_tbp (2 measured best: 1.5% faster than 1;
// 3 and 4 slower)
constexpr int kTbpGroup = 2;

template <int NT, int TS, int ES, bool PLASMA, bool SRC>
cudaError_t launch_tbp_t(const TBArgs& a, int n_tiles, int grid, cudaStream_t s) {
    auto kern = k_tbp<NT, TS, ES, kTbpGroup, PLASMA, SRC>;
    const size_t smem = TbpLayout<NT, TS, ES, PLASMA>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // programmatic dependent launch: this launch may begin while the previous kernel of the
    // stream finishes its last tiles; it waits for that kernel before it reads any field
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a, n_tiles);
}

// One form with the source branch for meshes with and without a source (the branch is one
// uniform test per step; the form without it needs more registers than the 128 a thread has).
template <int NT, int TS, int ES, bool PLASMA>
cudaError_t launch_tbp_s(const TBArgs& a, bool, int n_tiles, int grid, cudaStream_t s) {
    return launch_tbp_t<NT, TS, ES, PLASMA, true>(a, n_tiles, grid, s);
}

template <bool PLASMA, bool SRC>
cudaError_t launch_tbs_t(const TBArgs& a, int n_tiles, size_t smem, cudaStream_t s) {
    auto kern = k_tbs<PLASMA, SRC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<n_tiles, 1024, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NT, int TS, int ES, int MINB, int G>
cudaError_t launch_tb_ps(const TBArgs& a, bool plasma, bool src, int n_tiles, size_t smem,
                         cudaStream_t s) {
    if (plasma) return src ? launch_tb_t<NT, TS, ES, MINB, G, true, true>(a, n_tiles, smem, s)
                           : launch_tb_t<NT, TS, ES, MINB, G, true, false>(a, n_tiles, smem, s);
    return src ? launch_tb_t<NT, TS, ES, MINB, G, false, true>(a, n_tiles, smem, s)
               : launch_tb_t<NT, TS, ES, MINB, G, false, false>(a, n_tiles, smem, s);
}

// Opt-in shared memory per CTA, less the static shared memory of the kernels.
constexpr size_t kSmemMax = 227 * 1024 - 1024;

// The k_tbp slot configuration (triangle slots, edge slots) for tiles of at most TL local
// triangles and EL local edges, or (0, 0) when none fits (k_tb then runs).
void tbp_config(int TL, int EL, bool plasma, int& ts, int& es) {
    ts = es = 0;
    auto fits = [&](int a, int b, size_t smem) { return TL <= a * kNT && EL <= b * kNT && smem <= kSmemMax; };
    if (!plasma) {
        if (fits(4, 6, TbpLayout<kNT, 4, 6, false>::SMEM)) ts = 4, es = 6;
        else if (fits(6, 9, TbpLayout<kNT, 6, 9, false>::SMEM)) ts = 6, es = 9;
        else if (fits(8, 12, TbpLayout<kNT, 8, 12, false>::SMEM)) ts = 8, es = 12;
    } else {
        if (fits(4, 6, TbpLayout<kNT, 4, 6, true>::SMEM)) ts = 4, es = 6;
        else if (fits(6, 9, TbpLayout<kNT, 6, 9, true>::SMEM)) ts = 6, es = 9;
    }
}

}  // namespace

int tb_threads() { return kNT; }

size_t tbs_smem(int ntl, int nel, bool plasma) {
    return 4 * ((size_t)ntl + nel + 1) + (plasma ? 4 * ((size_t)nel + 1) : 0) + 8 +
           12 * (size_t)ntl + (plasma ? 12 : 8) * (size_t)nel;
}

bool tb_fits(int max_tri_loc, int max_edge_loc, int threads) {
    // 1024 threads: records in shared memory (227 KB per CTA, plasma included)
    if (threads == 1024) return tbs_smem(max_tri_loc, max_edge_loc, true) <= 227 * 1024;
    return max_tri_loc <= 8 * kNT && max_edge_loc <= 12 * kNT;
}

bool tb_pipelined(int max_tri_loc, int max_edge_loc, int threads, bool plasma) {
    int ts = 0, es = 0;
    tbp_config(max_tri_loc, max_edge_loc, plasma, ts, es);
    return threads != 1024 && ts > 0;
}

cudaError_t launch_tb_fill(const TBDev& t, const DevMesh& m, cudaStream_t s) {
    const int64_t n = t.n_trec > t.n_erec ? t.n_trec : t.n_erec;
    if (n == 0) return cudaSuccess;
    // the plasma coefficients once their array exists (made when the plasma is baked)
    const float* pb = (m.plasma && t.epb) ? (const float*)m.pb : nullptr;
    k_tb_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t.trec, t.n_trec, t.erec, t.epb, t.n_erec,
                                                        m.tri, (const float*)m.cU, pb);
    return cudaGetLastError();
}

int tb_kernel_used(const TBDev& t, const DevMesh& m) {
    if (t.n_tiles == 0) return UE_TBK_NONE;
    if (t.threads == 1024) return UE_TBK_SHARED_RECORDS;
    if (!m.plasma && t.frec && t.sms > 0 && tbf_fits(t.max_tri_loc, t.max_edge_loc, t.max_src)) return UE_TBK_FUSED;
    int ts = 0, es = 0;
    tbp_config(t.max_tri_loc, t.max_edge_loc, m.plasma, ts, es);
    if (t.sms > 0 && ts > 0) return UE_TBK_SPLIT_PIPELINED;
    return UE_TBK_SPLIT;
}

cudaError_t launch_tb(const TBDev& t, const DevMesh& m, int ksteps, int cur, int gbase,
                      cudaStream_t s) {
    TBArgs a;
    a.hdr = t.hdr;
    a.trec = t.trec;
    a.erec = t.erec;
    a.epb = t.epb;
    a.tsrc = t.tsrc;
    a.Bin = (const float*)t.B[cur];
    a.Uin = (const float*)t.U[cur];
    a.Jin = (const float*)t.J[cur];
    a.Bout = (float*)t.B[cur ^ 1];
    a.Uout = (float*)t.U[cur ^ 1];
    a.Jout = (float*)t.J[cur ^ 1];
    a.src_c = (const float*)m.src_c;
    a.src_grp = m.src_grp;
    a.gtab = m.gtab;
    a.gstride = m.gtab_size;
    a.gbase = gbase;
    a.step = m.step;
    a.done = t.done;
    a.err = t.done + 1;
    a.ksteps = ksteps;
    a.pa = (float)m.pa;
    a.mdt = (float)(-m.dt);
    a.test_cta = t.test_cta;
    const bool src = m.n_src > 0;
    if (ksteps < 1 || ksteps > 15) return cudaErrorInvalidValue;
    if (m.plasma && !t.epb) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * ((size_t)t.max_tri_loc + t.max_edge_loc + 1 +
                                         (m.plasma ? (size_t)t.max_edge_loc + 1 : 0));
    if (t.threads == 1024) {
        const size_t sm2 = tbs_smem(t.max_tri_loc, t.max_edge_loc, m.plasma);
        if (m.plasma) return src ? launch_tbs_t<true, true>(a, (int)t.n_tiles, sm2, s)
                                 : launch_tbs_t<true, false>(a, (int)t.n_tiles, sm2, s);
        return src ? launch_tbs_t<false, true>(a, (int)t.n_tiles, sm2, s)
                   : launch_tbs_t<false, false>(a, (int)t.n_tiles, sm2, s);
    }
    // vacuum media: the fused triangle-centric form when its records exist and the tiles fit
    if (!m.plasma && t.frec && t.sms > 0 && tbf_fits(t.max_tri_loc, t.max_edge_loc, t.max_src))
        return launch_tbf(t, m, ksteps, cur, gbase, s);
    // pipelined persistent form when two field buffers and the staging records fit
    int ts = 0, es = 0;
    tbp_config(t.max_tri_loc, t.max_edge_loc, m.plasma, ts, es);
    if (t.sms > 0 && ts > 0) {
        const int nt = (int)t.n_tiles;
        const int grid = nt < t.sms ? nt : t.sms;
        if (m.plasma) {
            if (ts == 4) return launch_tbp_s<kNT, 4, 6, true>(a, src, nt, grid, s);
            return launch_tbp_s<kNT, 6, 9, true>(a, src, nt, grid, s);
        }
        if (ts == 4) return launch_tbp_s<kNT, 4, 6, false>(a, src, nt, grid, s);
        if (ts == 6) return launch_tbp_s<kNT, 6, 9, false>(a, src, nt, grid, s);
        return launch_tbp_s<kNT, 8, 12, false>(a, src, nt, grid, s);
    }
    if (t.max_tri_loc <= 4 * kNT && t.max_edge_loc <= 6 * kNT)
        return launch_tb_ps<kNT, 4, 6, 2, 3>(a, m.plasma, src, (int)t.n_tiles, smem, s);
    if (t.max_tri_loc <= 6 * kNT && t.max_edge_loc <= 9 * kNT)
        return launch_tb_ps<kNT, 6, 9, 1, 3>(a, m.plasma, src, (int)t.n_tiles, smem, s);
    return launch_tb_ps<kNT, 8, 12, 1, 1>(a, m.plasma, src, (int)t.n_tiles, smem, s);
}

}  // namespace ue
