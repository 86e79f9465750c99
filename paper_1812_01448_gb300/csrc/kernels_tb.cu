// Temporally blocked leap-frog: one CTA per KD tile advances its owned edges and triangles by
// k steps (eqs. 14-15 with eqs. 3-6) in shared memory, recomputing the k-ring halo that the
// neighbouring tiles own.  The paper's "Divide and conqueror" partitions exchange boundary
// values every step; here the exchange is replaced by redundant halo work inside one launch.
//
// Per launch a tile reads its records (static, 16 B per local triangle and per local edge) and
// the fields of its local set from the "in" buffers, and writes only the owned values to the
// "out" buffers (double buffering, so that neighbours still read time level n).  Every
// arithmetic operation repeats the plain kernels' sequence exactly (device.cuh rn_* helpers
// and the shared source_g), so the results are bit-identical to the plain two-kernel step.
#include <cuda_runtime.h>

#include "device.cuh"

namespace ue {

namespace {

constexpr int kNT = 512;

struct TBArgs {
    const int* hdr;
    const int4* trec;
    const int4* erec;
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
    const int4* er = a.erec + h[7];
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
            const int4 r = __ldg(er + l);
            erl[i] = r.y;
            ecu[i] = __int_as_float(r.z);
            Ul[l] = __ldg(a.Uin + r.x);
            if constexpr (PLASMA) {
                epb[i] = __int_as_float(r.w);
                Jl[l] = __ldg(a.Jin + r.x);
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
    const int4* er = a.erec + h[7];
    for (int l = tid; l < ntl; l += NT) {
        const int4 r = __ldg(tr + l);
        Tc[l] = make_int2(r.y, r.z);
        Tb[l] = __int_as_float(r.w);
        Bl[l] = __ldg(a.Bin + r.x);
    }
    for (int l = tid; l < nel; l += NT) {
        const int4 r = __ldg(er + l);
        Erl[l] = r.y;
        Ecu[l] = __int_as_float(r.z);
        Ul[l] = __ldg(a.Uin + r.x);
        if constexpr (PLASMA) {
            Epb[l] = __int_as_float(r.w);
            Jl[l] = __ldg(a.Jin + r.x);
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

// Pipelined persistent form (no plasma): one CTA per SM walks the tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...  Global loads run ahead of the steps:
// - headers: a ring of three; tile i+2's header is copied (TMA bulk copy) while tile i steps;
// - records: tile i+1's records are copied (TMA bulk copies) into a staging area as soon as
//   tile i has moved its own records from there into registers;
// - fields: after step min(3, k) of tile i, tile i+1's fields are gathered (4-byte cp.async)
//   into the second field buffer.
// So a tile's loads overlap the previous tile's steps instead of stalling the SM.  Each thread
// keeps its slots' records in registers for the k steps and repeats k_tb's arithmetic slot by
// slot, so the results are bit-identical.
// Dynamic shared memory: two field buffers of FB floats (B at 0, U at TL), then the staging
// records (TL triangle records, EL edge records).
template <int NT, int TS, int ES, bool SRC>
__global__ void __launch_bounds__(NT, 1) k_tbp(TBArgs a, int n_tiles, int TL, int EL) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ __align__(16) int hs[3][48];
    __shared__ __align__(8) uint64_t bar_h, bar_r;
    const int tid = threadIdx.x;
    const int FB = (TL + EL + 1 + 3) & ~3;
    const int stride = gridDim.x;
    float* F0 = reinterpret_cast<float*>(smraw);
    int4* tstage = reinterpret_cast<int4*>(F0 + 2 * FB);
    int4* estage = tstage + TL;
    if (tid == 0) {
        mbar_init(&bar_h, 1);
        mbar_init(&bar_r, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const long long n0 = *a.step;
    uint32_t ph_h = 0, ph_r = 0;
    bool ok = true;
    auto wait_bar = [&](uint64_t* bar, uint32_t& ph) {
        if (!mbar_wait(bar, ph)) ok = false;
        ph ^= 1u;
    };
    auto issue_header = [&](int t, int slot) {
        if (tid == 0) {
            fence_proxy_async();
            bulk_g2s(hs[slot], a.hdr + (size_t)t * 48, 48 * sizeof(int), &bar_h);
        }
    };
    auto issue_records = [&](int slot) {
        if (tid == 0) {
            const uint32_t tb = 16u * (uint32_t)hs[slot][4], eb = 16u * (uint32_t)hs[slot][5];
            fence_proxy_async();
            mbar_expect_tx(&bar_r, tb + eb);
            if (tb) bulk_copy_g2s(tstage, a.trec + hs[slot][6], tb, &bar_r);
            if (eb) bulk_copy_g2s(estage, a.erec + hs[slot][7], eb, &bar_r);
        }
    };
    auto issue_fields = [&](int slot, int b) {
        const int ntl = hs[slot][4], nel = hs[slot][5];
        float* Bn = F0 + b * FB;
        float* Un = Bn + TL;
#pragma unroll
        for (int i = 0; i < TS; ++i) {
            const int l = tid + i * NT;
            if (l < ntl) cp_async4(Bn + l, a.Bin + tstage[l].x);
        }
#pragma unroll
        for (int i = 0; i < ES; ++i) {
            const int l = tid + i * NT;
            if (l < nel) cp_async4(Un + l, a.Uin + estage[l].x);
        }
        if (tid == 0) Un[nel] = 0.f;
        cp_async_commit();
    };
    int tile = blockIdx.x, it = 0, cur = 0;
    // prologue: first tile's header, records and fields; the second tile's header
    if (tile < n_tiles) {
        issue_header(tile, 0);
        wait_bar(&bar_h, ph_h);
        issue_records(0);
        if (tile + stride < n_tiles) issue_header(tile + stride, 1);
        wait_bar(&bar_r, ph_r);
        issue_fields(0, 0);
        cp_async_wait_all();
        if (tile + stride < n_tiles) wait_bar(&bar_h, ph_h);
    }
    __syncthreads();
    int tc01[TS], tc2[TS];
    float tcb[TS];
    int erl[ES];
    float ecu[ES];
    for (; tile < n_tiles; tile += stride, ++it) {
        const bool has_next = tile + stride < n_tiles, has_next2 = tile + 2 * stride < n_tiles;
        const int slot = it % 3, slot1 = (it + 1) % 3, slot2 = (it + 2) % 3;
        const int* h = hs[slot];
        float* Bl = F0 + cur * FB;
        float* Ul = Bl + TL;
        const int ntl = h[4], nel = h[5];
#pragma unroll
        for (int i = 0; i < TS; ++i) {
            const int l = tid + i * NT;
            if (l < ntl) {
                const int4 r = tstage[l];
                tc01[i] = r.y;
                tc2[i] = r.z;
                tcb[i] = __int_as_float(r.w);
            }
        }
#pragma unroll
        for (int i = 0; i < ES; ++i) {
            const int l = tid + i * NT;
            if (l < nel) {
                const int4 r = estage[l];
                erl[i] = r.y;
                ecu[i] = __int_as_float(r.z);
            }
        }
        __syncthreads();   // the staging area is free for the next tile's records
        if (has_next) issue_records(slot1);
        if (has_next2) issue_header(tile + 2 * stride, slot2);
        const int s_fields = a.ksteps < 3 ? a.ksteps : 3;
        for (int s = 1; s <= a.ksteps; ++s) {
            const int lim = a.ksteps - s;
            const int eend = h[32 + lim];
#pragma unroll
            for (int i = 0; i < ES; ++i) {
                const int l = tid + i * NT;
                if (l < eend) {
                    const float bR = Bl[erl[i] & 0xFFFF];
                    const float bL = Bl[(unsigned)erl[i] >> 16];
                    Ul[l] = rn_fma(ecu[i], rn_sub(bR, bL), Ul[l]);
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
            for (int i = 0; i < TS; ++i) {
                const int l = tid + i * NT;
                if (l < tend) {
                    const int c0 = tc01[i], c1 = (unsigned)tc01[i] >> 16, c2 = tc2[i];
                    const float u0 = Ul[(c0 & 0xFFFF) >> 1], u1 = Ul[c1 >> 1], u2 = Ul[c2 >> 1];
                    const float x0 = (c0 & 1) ? -u0 : u0;
                    const float x1 = (c1 & 1) ? -u1 : u1;
                    const float x2 = (c2 & 1) ? -u2 : u2;
                    Bl[l] = rn_fma(-tcb[i], rn_add(rn_add(x0, x1), x2), Bl[l]);
                }
            }
            __syncthreads();
            if (has_next && s == s_fields) {
                wait_bar(&bar_r, ph_r);
                issue_fields(slot1, cur ^ 1);
            }
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
            if (l < neo) a.Uout[h[2] + l] = Ul[l];
        }
        if (has_next) cp_async_wait_all();
        if (has_next2) wait_bar(&bar_h, ph_h);
        __syncthreads();
        cur ^= 1;
    }
    if (!ok) atomicOr(a.err, 1u);
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

// Fill the coefficient slots of the tile records from the global coefficient arrays.
__global__ void k_tb_fill(int4* __restrict__ trec, int64_t n_trec, int4* __restrict__ erec,
                          int64_t n_erec, const int4* __restrict__ tri, const float* __restrict__ cU,
                          const float* __restrict__ pb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_trec) trec[i].w = tri[trec[i].x].w;
    if (i < n_erec) {
        const int g = erec[i].x;
        erec[i].z = __float_as_int(fabsf(cU[g]));   // without the source flag
        erec[i].w = pb ? __float_as_int(pb[g]) : 0;
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

template <int NT, int TS, int ES, bool SRC>
cudaError_t launch_tbp_t(const TBArgs& a, int n_tiles, int grid, int TL, int EL, size_t smem,
                         cudaStream_t s) {
    auto kern = k_tbp<NT, TS, ES, SRC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, NT, smem, s>>>(a, n_tiles, TL, EL);
    return cudaGetLastError();
}

template <int NT, int TS, int ES>
cudaError_t launch_tbp_s(const TBArgs& a, bool src, int n_tiles, int grid, int TL, int EL,
                         size_t smem, cudaStream_t s) {
    return src ? launch_tbp_t<NT, TS, ES, true>(a, n_tiles, grid, TL, EL, smem, s)
               : launch_tbp_t<NT, TS, ES, false>(a, n_tiles, grid, TL, EL, smem, s);
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

}  // namespace

int tb_threads() { return kNT; }

// Register-slot configurations, smallest first: (threads, triangle slots, edge slots, CTAs
// per SM the register budget is sized for).
size_t tbs_smem(int ntl, int nel, bool plasma) {
    return 4 * ((size_t)ntl + nel + 1) + (plasma ? 4 * ((size_t)nel + 1) : 0) + 8 +
           12 * (size_t)ntl + (plasma ? 12 : 8) * (size_t)nel;
}

// k_tbp: two field buffers and the staging records, within the opt-in shared memory per CTA
// (static shared memory of the kernel aside).
constexpr size_t kTbpSmemMax = 227 * 1024 - 512;
size_t tbp_smem(int tl, int el) {
    const size_t fb = ((size_t)tl + el + 1 + 3) & ~(size_t)3;
    return 2 * 4 * fb + 16 * ((size_t)tl + el);
}

bool tb_fits(int max_tri_loc, int max_edge_loc, int threads) {
    // 1024 threads: records in shared memory (227 KB per CTA, plasma included)
    if (threads == 1024) return tbs_smem(max_tri_loc, max_edge_loc, true) <= 227 * 1024;
    return max_tri_loc <= 8 * kNT && max_edge_loc <= 12 * kNT;
}

cudaError_t launch_tb_fill(const TBDev& t, const DevMesh& m, cudaStream_t s) {
    const int64_t n = t.n_trec > t.n_erec ? t.n_trec : t.n_erec;
    if (n == 0) return cudaSuccess;
    k_tb_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t.trec, t.n_trec, t.erec, t.n_erec, m.tri,
                                                        (const float*)m.cU,
                                                        m.plasma ? (const float*)m.pb : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_tb(const TBDev& t, const DevMesh& m, int ksteps, int cur, int gbase,
                      cudaStream_t s) {
    TBArgs a;
    a.hdr = t.hdr;
    a.trec = t.trec;
    a.erec = t.erec;
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
    const bool src = m.n_src > 0;
    const size_t smem = sizeof(float) * ((size_t)t.max_tri_loc + t.max_edge_loc + 1 +
                                         (m.plasma ? (size_t)t.max_edge_loc + 1 : 0));
    if (t.threads == 1024) {
        const size_t sm2 = tbs_smem(t.max_tri_loc, t.max_edge_loc, m.plasma);
        if (m.plasma) return src ? launch_tbs_t<true, true>(a, (int)t.n_tiles, sm2, s)
                                 : launch_tbs_t<true, false>(a, (int)t.n_tiles, sm2, s);
        return src ? launch_tbs_t<false, true>(a, (int)t.n_tiles, sm2, s)
                   : launch_tbs_t<false, false>(a, (int)t.n_tiles, sm2, s);
    }
    // pipelined persistent form when two field buffers and the staging records fit
    const size_t smem_p = tbp_smem(t.max_tri_loc, t.max_edge_loc);
    if (!m.plasma && t.sms > 0 && smem_p <= kTbpSmemMax) {
        const int TL = t.max_tri_loc, EL = t.max_edge_loc, nt = (int)t.n_tiles;
        const int grid = nt < t.sms ? nt : t.sms;
        if (TL <= 4 * kNT && EL <= 6 * kNT) return launch_tbp_s<kNT, 4, 6>(a, src, nt, grid, TL, EL, smem_p, s);
        if (TL <= 6 * kNT && EL <= 9 * kNT) return launch_tbp_s<kNT, 6, 9>(a, src, nt, grid, TL, EL, smem_p, s);
        return launch_tbp_s<kNT, 8, 12>(a, src, nt, grid, TL, EL, smem_p, s);
    }
    if (t.max_tri_loc <= 4 * kNT && t.max_edge_loc <= 6 * kNT)
        return launch_tb_ps<kNT, 4, 6, 2, 3>(a, m.plasma, src, (int)t.n_tiles, smem, s);
    if (t.max_tri_loc <= 6 * kNT && t.max_edge_loc <= 9 * kNT)
        return launch_tb_ps<kNT, 6, 9, 1, 3>(a, m.plasma, src, (int)t.n_tiles, smem, s);
    return launch_tb_ps<kNT, 8, 12, 1, 1>(a, m.plasma, src, (int)t.n_tiles, smem, s);
}

}  // namespace ue
