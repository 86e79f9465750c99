// The leap-frog step (eqs. 14-15): the E half-step of eq. 3 (eq. 6 with the current of eq. 5
// in plasma media) over interior edges, an optional soft source, then the B half-step of
// eq. 4 over triangles.  Plain form: one thread per edge, then one thread per triangle.
//
// Stored variables are circulations U_i = |e_i| E_i (and J_i = |e_i| j_i), so that
//   E half-step:  U_i += (dt |e_i| / d_i) (B_R - B_L)            [eq. 3 times dt |e_i|]
//   plasma:       J_i  = pa J_i + pb_i U_i;  U_i -= dt J_i        [eqs. 5-6, trapezoidal in nu]
//   B half-step:  B_j -= (dt / S_j) (s_0 U_0 + s_1 U_1 + s_2 U_2) [eq. 4]
// with the sign s(j,q) carried in bit 0 of the edge code and boundary edges pointing at a
// zero slot (U[n_ei] = 0).  Every operation is explicitly rounded (device.cuh).
#include <cuda_runtime.h>

#include "device.cuh"

namespace ue {

namespace {

constexpr int kThreads = 256;

template <typename T, bool PLASMA>
__global__ void __launch_bounds__(kThreads)
k_edge_half(const int2* __restrict__ rl, const T* __restrict__ cU, const T* __restrict__ B,
            T* __restrict__ U, const T* __restrict__ pb, T* __restrict__ J, T pa, T mdt,
            int64_t n_ei) {
    const int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (k >= n_ei) return;
    const int2 e = __ldg(rl + k);
    const T b = rn_sub(__ldg(B + e.x), __ldg(B + e.y));
    const T u = U[k];
    T un = rn_fma(__ldg(cU + k), b, u);
    if constexpr (PLASMA) {
        const T jn = rn_fma(pa, J[k], rn_mul(__ldg(pb + k), u));
        J[k] = jn;
        un = rn_fma(mdt, jn, un);
    }
    U[k] = un;
}

// Soft source on its edges: U += dt |e| a g(t), t = (step + 1/2) dt, g in FP64.
template <typename T>
__global__ void k_source(const int32_t* __restrict__ sk, const T* __restrict__ sc, int64_t n,
                         T* __restrict__ U, const long long* __restrict__ step, double dt,
                         double w0, double t0, double tau) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const T g = (T)source_g(*step, dt, w0, t0, tau);
    const int k = sk[i];
    U[k] = rn_fma(sc[i], g, U[k]);
}

template <typename T>
__device__ __forceinline__ T signed_load(const T* __restrict__ U, int code) {
    const T u = __ldg(U + (code >> 1));
    return (code & 1) ? -u : u;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_tri_half(const int4* __restrict__ tri, const double* __restrict__ cB64,
           const T* __restrict__ U, T* __restrict__ B, int64_t n_t, long long* __restrict__ step) {
    const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (j == 0) *step += 1;
    if (j >= n_t) return;
    const int4 t = __ldg(tri + j);
    const T s = rn_add(rn_add(signed_load(U, t.x), signed_load(U, t.y)), signed_load(U, t.z));
    T c;
    if constexpr (sizeof(T) == 4) c = __int_as_float(t.w);
    else c = __ldg(cB64 + j);
    B[j] = rn_fma(-c, s, B[j]);
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

template <typename T>
void edge_half_t(const DevMesh& m, cudaStream_t s) {
    if (m.n_ei == 0) return;
    if (m.plasma)
        k_edge_half<T, true><<<blocks_for(m.n_ei), kThreads, 0, s>>>(
            m.rl, (const T*)m.cU, (const T*)m.B, (T*)m.U, (const T*)m.pb, (T*)m.J, (T)m.pa,
            (T)(-m.dt), m.n_ei);
    else
        k_edge_half<T, false><<<blocks_for(m.n_ei), kThreads, 0, s>>>(
            m.rl, (const T*)m.cU, (const T*)m.B, (T*)m.U, nullptr, nullptr, (T)0, (T)0, m.n_ei);
}

template <typename T>
void source_t(const DevMesh& m, cudaStream_t s) {
    if (m.n_src > 0)
        k_source<T><<<blocks_for(m.n_src), kThreads, 0, s>>>(m.src_k, (const T*)m.src_c, m.n_src,
                                                             (T*)m.U, m.step, m.dt, m.w0, m.t0, m.tau);
}

template <typename T>
void tri_half_t(const DevMesh& m, cudaStream_t s) {
    k_tri_half<T><<<blocks_for(m.n_t), kThreads, 0, s>>>(m.tri, (const double*)m.cB,
                                                         (const T*)m.U, (T*)m.B, m.n_t, m.step);
}

}  // namespace

cudaError_t launch_step_part(const DevMesh& m, int part, cudaStream_t s) {
    const bool f64 = m.precision == UE_PREC_FP64;
    switch (part) {
        case 0: f64 ? edge_half_t<double>(m, s) : edge_half_t<float>(m, s); break;
        case 1: f64 ? source_t<double>(m, s) : source_t<float>(m, s); break;
        default: f64 ? tri_half_t<double>(m, s) : tri_half_t<float>(m, s); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_step_plain(const DevMesh& m, cudaStream_t s) {
    for (int p = 0; p < 3; ++p) {
        cudaError_t e = launch_step_part(m, p, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ue
