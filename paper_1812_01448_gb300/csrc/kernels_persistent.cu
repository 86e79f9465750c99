// Persistent cooperative leap-frog: one cooperative launch runs n steps.  Its CTAs stride over
// the interior edges (E half-step of eq. 3, with the current of eqs. 5-6 and the source) and,
// after a grid barrier, over the triangles (B half-step of eq. 4), then meet at a second
// barrier.  Element arithmetic is the plain kernels' sequence, so results are bit-identical.
//
// The grid barrier is timed: a CTA that waits longer than `budget` clock cycles (or sees the
// error word set) records UE_ERR_TIMEOUT's cause in the error word and returns, so a missing
// CTA ends the launch instead of hanging it.  `skip_cta` (>= 0) makes one CTA return at once;
// it exists to test that path.  Values written by other CTAs in this launch (the gathered B
// and U) are read through L2 (ld.global.cg), never from a possibly stale L1 line.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "device.cuh"

namespace ue {

namespace {

struct PArgs {
    const int4* rl4;
    const float* cU;
    float* U;
    float* B;
    const float* pb;
    float* J;
    float pa, mdt;
    const int4* tri;
    int64_t n_vec_e, n_vec_t;
    // source
    const int2* hash;
    unsigned bits;
    const float* src_c;
    const int32_t* src_grp;
    const double* gtab;
    int gstride;
    bool has_src;
    long long* step;
    int n_steps;
    // barrier
    unsigned* count;
    unsigned* gen;
    int* err;
    long long budget;
    int skip_cta;
};

__device__ bool grid_barrier(const PArgs& a) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned* gen = a.gen;
        volatile int* err = a.err;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(a.count, 1u);
        if (arrived == gridDim.x - 1) {
            *a.count = 0u;
            __threadfence();
            atomicAdd(a.gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (*err != 0) {
                    ok = 0;
                    break;
                }
                if (clock64() - t0 > a.budget) {
                    atomicExch(a.err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ float src_term(const PArgs& a, int k, float u, int s) {
    const unsigned size = 1u << a.bits;
    unsigned h = ((unsigned)k * 2654435761u) >> (32 - a.bits);
    int2 e = __ldg(a.hash + h);
    for (unsigned p = 1; e.x != k && p < size; ++p) {
        h = (h + 1) & (size - 1);
        e = __ldg(a.hash + h);
    }
    if (e.x != k) return u;
    const double g = __ldg(a.gtab + (size_t)__ldg(a.src_grp + e.y) * a.gstride + s);
    return rn_fma(__ldg(a.src_c + e.y), (float)g, u);
}

template <bool PLASMA>
__global__ void __launch_bounds__(256) k_persistent(PArgs a) {
    if ((int)blockIdx.x == a.skip_cta) return;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int s = 0; s < a.n_steps; ++s) {
        for (int64_t v = tid; v < a.n_vec_e; v += stride) {
            const int4 ra = __ldg(a.rl4 + 2 * v), rb = __ldg(a.rl4 + 2 * v + 1);
            const int R[4] = {ra.x, ra.z, rb.x, rb.z};
            const int L[4] = {ra.y, ra.w, rb.y, rb.w};
            const float4 c4 = __ldg(reinterpret_cast<const float4*>(a.cU) + v);
            const float c[4] = {c4.x, c4.y, c4.z, c4.w};
            const float4 u4 = reinterpret_cast<const float4*>(a.U)[v];
            const float u[4] = {u4.x, u4.y, u4.z, u4.w};
            float un[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) un[i] = rn_fma(fabsf(c[i]), rn_sub(__ldcg(a.B + R[i]), __ldcg(a.B + L[i])), u[i]);
            if constexpr (PLASMA) {
                const float4 j4 = reinterpret_cast<const float4*>(a.J)[v];
                const float4 p4 = __ldg(reinterpret_cast<const float4*>(a.pb) + v);
                float jj[4] = {j4.x, j4.y, j4.z, j4.w};
                const float p[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    jj[i] = rn_fma(a.pa, jj[i], rn_mul(p[i], u[i]));
                    un[i] = rn_fma(a.mdt, jj[i], un[i]);
                }
                reinterpret_cast<float4*>(a.J)[v] = make_float4(jj[0], jj[1], jj[2], jj[3]);
            }
            if (a.has_src) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (__float_as_uint(c[i]) >> 31) un[i] = src_term(a, (int)(4 * v + i), un[i], s);
            }
            reinterpret_cast<float4*>(a.U)[v] = make_float4(un[0], un[1], un[2], un[3]);
        }
        if (!grid_barrier(a)) return;
        for (int64_t v = tid; v < a.n_vec_t; v += stride) {
            float4 b4 = reinterpret_cast<float4*>(a.B)[v];
            float bo[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int4 t = __ldg(a.tri + 4 * v + i);
                float u0 = __ldcg(a.U + (t.x >> 1)), u1 = __ldcg(a.U + (t.y >> 1)), u2 = __ldcg(a.U + (t.z >> 1));
                if (t.x & 1) u0 = -u0;
                if (t.y & 1) u1 = -u1;
                if (t.z & 1) u2 = -u2;
                bo[i] = rn_fma(-__int_as_float(t.w), rn_add(rn_add(u0, u1), u2), bo[i]);
            }
            reinterpret_cast<float4*>(a.B)[v] = make_float4(bo[0], bo[1], bo[2], bo[3]);
        }
        if (tid == 0) *a.step += 1;
        if (!grid_barrier(a)) return;
    }
}

}  // namespace

int persistent_grid(int device) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent<false>, 256, 0);
    int per2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k_persistent<true>, 256, 0);
    if (per2 < per) per = per2;
    return sms * (per > 0 ? per : 1);
}

// n steps in one cooperative launch; `sync` = {count, gen} and err must be zeroed by the caller.
cudaError_t launch_persistent(const DevMesh& m, int n_steps, unsigned* sync, int* err,
                              long long budget, int skip_cta, int grid, cudaStream_t s) {
    PArgs a;
    a.rl4 = (const int4*)m.rl;
    a.cU = (const float*)m.cU;
    a.U = (float*)m.U;
    a.B = (float*)m.B;
    a.pb = (const float*)m.pb;
    a.J = (float*)m.J;
    a.pa = (float)m.pa;
    a.mdt = (float)(-m.dt);
    a.tri = m.tri;
    a.n_vec_e = m.n_ei_pad / 4;
    a.n_vec_t = m.n_t_pad / 4;
    a.hash = m.src_hash;
    a.bits = (unsigned)m.src_bits;
    a.src_c = (const float*)m.src_c;
    a.src_grp = m.src_grp;
    a.gtab = m.gtab;
    a.gstride = m.gtab_size;
    a.has_src = m.n_src > 0;
    a.step = m.step;
    a.n_steps = n_steps;
    a.count = sync;
    a.gen = sync + 1;
    a.err = err;
    a.budget = budget;
    a.skip_cta = skip_cta;
    void* args[] = {&a};
    const void* fn = m.plasma ? (const void*)k_persistent<true> : (const void*)k_persistent<false>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(256), args, 0, s);
}

}  // namespace ue
