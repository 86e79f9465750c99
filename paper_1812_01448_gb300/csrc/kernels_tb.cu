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
    const double* gtab;
    int gbase;
    long long* step;
    unsigned* done;
    int ksteps;
    float pa, mdt;
    double dt, w0, t0, tau;
};

template <int TS, int ES, bool PLASMA, bool SRC>
__global__ void __launch_bounds__(kNT, 1) k_tb(TBArgs a) {
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
        const int l = tid + i * kNT;
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
        const int l = tid + i * kNT;
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
        for (int i = 0; i < ES; ++i) {
            const int l = tid + i * kNT;
            if (l < eend) {
                const int rl = erl[i];
                const float b = rn_sub(Bl[rl & 0xFFFF], Bl[(unsigned)rl >> 16]);
                const float u = Ul[l];
                float un = rn_fma(ecu[i], b, u);
                if constexpr (PLASMA) {
                    const float jn = rn_fma(a.pa, Jl[l], rn_mul(epb[i], u));
                    Jl[l] = jn;
                    un = rn_fma(a.mdt, jn, un);
                }
                Ul[l] = un;
            }
        }
        if constexpr (SRC) {
            if (h[9] > 0) {
                __syncthreads();
                const float g = (float)__ldg(a.gtab + a.gbase + s - 1);
                for (int i = tid; i < h[9]; i += kNT) {
                    const int2 q = __ldg(a.tsrc + h[8] + i);
                    if (q.x < eend) Ul[q.x] = rn_fma(__ldg(a.src_c + q.y), g, Ul[q.x]);
                }
            }
        }
        __syncthreads();
        const int tend = h[16 + lim];
#pragma unroll
        for (int i = 0; i < TS; ++i) {
            const int l = tid + i * kNT;
            if (l < tend) {
                const int c0 = tc01[i] & 0xFFFF, c1 = (unsigned)tc01[i] >> 16, c2 = tc2[i];
                float u0 = Ul[c0 >> 1], u1 = Ul[c1 >> 1], u2 = Ul[c2 >> 1];
                if (c0 & 1) u0 = -u0;
                if (c1 & 1) u1 = -u1;
                if (c2 & 1) u2 = -u2;
                const float sum = rn_add(rn_add(u0, u1), u2);
                Bl[l] = rn_fma(-tcb[i], sum, Bl[l]);
            }
        }
        __syncthreads();
    }
    const int nto = h[1], neo = h[3];
#pragma unroll
    for (int i = 0; i < TS; ++i) {
        const int l = tid + i * kNT;
        if (l < nto) a.Bout[h[0] + l] = Bl[l];
    }
#pragma unroll
    for (int i = 0; i < ES; ++i) {
        const int l = tid + i * kNT;
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

template <int TS, int ES, bool PLASMA, bool SRC>
cudaError_t launch_tb_t(const TBArgs& a, int n_tiles, size_t smem, cudaStream_t s) {
    auto kern = k_tb<TS, ES, PLASMA, SRC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<n_tiles, kNT, smem, s>>>(a);
    return cudaGetLastError();
}

template <int TS, int ES>
cudaError_t launch_tb_ps(const TBArgs& a, bool plasma, bool src, int n_tiles, size_t smem,
                         cudaStream_t s) {
    if (plasma) return src ? launch_tb_t<TS, ES, true, true>(a, n_tiles, smem, s)
                           : launch_tb_t<TS, ES, true, false>(a, n_tiles, smem, s);
    return src ? launch_tb_t<TS, ES, false, true>(a, n_tiles, smem, s)
               : launch_tb_t<TS, ES, false, false>(a, n_tiles, smem, s);
}

}  // namespace

int tb_threads() { return kNT; }

bool tb_fits(int max_tri_loc, int max_edge_loc) {
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
    a.gtab = m.gtab;
    a.gbase = gbase;
    a.step = m.step;
    a.done = t.done;
    a.ksteps = ksteps;
    a.pa = (float)m.pa;
    a.mdt = (float)(-m.dt);
    a.dt = m.dt;
    a.w0 = m.w0;
    a.t0 = m.t0;
    a.tau = m.tau;
    const bool src = m.n_src > 0;
    const size_t smem = sizeof(float) * ((size_t)t.max_tri_loc + t.max_edge_loc + 1 +
                                         (m.plasma ? (size_t)t.max_edge_loc + 1 : 0));
    if (t.max_tri_loc <= 4 * kNT && t.max_edge_loc <= 6 * kNT)
        return launch_tb_ps<4, 6>(a, m.plasma, src, (int)t.n_tiles, smem, s);
    return launch_tb_ps<8, 12>(a, m.plasma, src, (int)t.n_tiles, smem, s);
}

}  // namespace ue
