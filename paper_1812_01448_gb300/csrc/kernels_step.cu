// The leap-frog step (eqs. 14-15): the E half-step of eq. 3 (eq. 6 with the current of eq. 5
// in plasma media, plus the soft source) over interior edges, then the B half-step of eq. 4
// over triangles.  Plain form: two kernels per step, four elements per thread with 16-byte
// loads of the streamed arrays, so that each thread keeps several independent gathers in
// flight.
//
// Stored variables are circulations U_i = |e_i| E_i (and J_i = |e_i| j_i), so that
//   E half-step:  U_i += (dt |e_i| / d_i) (B_R - B_L)            [eq. 3 times dt |e_i|]
//   plasma:       J_i  = pa J_i + pb_i U_i;  U_i -= dt J_i        [eqs. 5-6, trapezoidal in nu]
//   source:       U_i += (dt |e_i| a_i) g(t_n)                    [g from a per-chunk table]
//   B half-step:  B_j -= (dt / S_j) (s_0 U_0 + s_1 U_1 + s_2 U_2) [eq. 4]
// The sign s(j,q) is bit 0 of the edge code; boundary edges point at a slot that stays 0.
// Source edges carry the sign bit of their coefficient dt|e|/d (always > 0) as a flag and find
// their source coefficient through a small open-addressing table.  Arrays are padded to a
// multiple of four with neutral entries (R = L = 0 and zero coefficients; triangle codes on
// the zero slot).  Every operation is explicitly rounded (device.cuh).
#include <cuda_runtime.h>

#include "device.cuh"
#include "frame.cuh"

namespace ue {

namespace {

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ void ld4(const T* __restrict__ p, T (&x)[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
        x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
    }
}

// load/store of read-write arrays (not through the read-only path)
template <typename T>
__device__ __forceinline__ void ldw4(const T* p, T (&x)[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else {
        const double2 a = reinterpret_cast<const double2*>(p)[0];
        const double2 b = reinterpret_cast<const double2*>(p)[1];
        x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
    }
}

template <typename T>
__device__ __forceinline__ void st4(T* p, const T (&x)[4]) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
    } else {
        reinterpret_cast<double2*>(p)[0] = make_double2(x[0], x[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(x[2], x[3]);
    }
}

__device__ __forceinline__ bool flagged(float c) { return __float_as_uint(c) >> 31; }
__device__ __forceinline__ bool flagged(double c) {
    return (unsigned long long)__double_as_longlong(c) >> 63;
}

template <typename T>
struct SrcArgs {
    const int2* hash;       // {edge id, source index}, empty slots have edge id -1
    unsigned bits;          // table size 2^bits
    const T* c;             // dt |e| a per source index
    const int32_t* grp;     // group of each source index
    const double* g;        // g(t) per group and step of the current chunk
    int stride;             // table entries per group
    int s;                  // this step's index in the chunk table
};

template <typename T>
__device__ __forceinline__ T source_term(const SrcArgs<T>& src, int k, T u) {
    const unsigned size = 1u << src.bits;
    unsigned h = ((unsigned)k * 2654435761u) >> (32 - src.bits);
    int2 e = __ldg(src.hash + h);
    // linear probing; a flagged edge is always in the table, the bound only guards the loop
    for (unsigned p = 1; e.x != k && p < size; ++p) {
        h = (h + 1) & (size - 1);
        e = __ldg(src.hash + h);
    }
    if (e.x != k) return u;
    const double g = __ldg(src.g + (size_t)__ldg(src.grp + e.y) * src.stride + src.s);
    return rn_fma(__ldg(src.c + e.y), (T)g, u);
}

// FRAME: blocks from nb_mesh on run a PML frame's sides and interface edges (frame.cuh); they
// write only the frame's arrays and the interface slots, which no mesh thread touches.
template <typename T, bool PLASMA, bool SRC, bool FRAME>
__global__ void __launch_bounds__(kThreads)
k_edge_half(const int4* __restrict__ rl4, const T* __restrict__ cU, const T* __restrict__ B,
            T* __restrict__ U, const T* __restrict__ pb, T* __restrict__ J, T pa, T mdt,
            int64_t n_vec, SrcArgs<T> src, FrameDev f, int64_t nb_mesh) {
    if constexpr (FRAME) {
        if ((int64_t)blockIdx.x >= nb_mesh) {
            frame_edge_thread<T>(f, B, U, ((int64_t)blockIdx.x - nb_mesh) * kThreads + threadIdx.x);
            return;
        }
    }
    const int64_t v = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (v >= n_vec) return;
    const int4 ra = __ldg(rl4 + 2 * v), rb = __ldg(rl4 + 2 * v + 1);
    const int R[4] = {ra.x, ra.z, rb.x, rb.z};
    const int L[4] = {ra.y, ra.w, rb.y, rb.w};
    T c[4], u[4], b[4], un[4];
    ld4(cU + 4 * v, c);
    ldw4(U + 4 * v, u);
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = rn_sub(__ldg(B + R[i]), __ldg(B + L[i]));
#pragma unroll
    for (int i = 0; i < 4; ++i) un[i] = rn_fma(fabs(c[i]), b[i], u[i]);
    if constexpr (PLASMA) {
        T jj[4], p[4];
        ldw4(J + 4 * v, jj);
        ld4(pb + 4 * v, p);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            jj[i] = rn_fma(pa, jj[i], rn_mul(p[i], u[i]));
            un[i] = rn_fma(mdt, jj[i], un[i]);
        }
        st4(J + 4 * v, jj);
    }
    if constexpr (SRC) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (flagged(c[i])) un[i] = source_term(src, (int)(4 * v + i), un[i]);
    }
    st4(U + 4 * v, un);
}

template <typename T>
__device__ __forceinline__ T signed_load(const T* __restrict__ U, int code) {
    const T u = __ldg(U + (code >> 1));
    return (code & 1) ? -u : u;
}

// FRAME: blocks from nb_mesh on update a PML frame's cells (frame.cuh).
template <typename T, bool FRAME>
__global__ void __launch_bounds__(kThreads)
k_tri_half(const int4* __restrict__ tri, const double* __restrict__ cB64,
           const T* __restrict__ U, T* __restrict__ B, int64_t n_vec, long long* __restrict__ step,
           FrameDev f, int64_t nb_mesh) {
    if constexpr (FRAME) {
        if ((int64_t)blockIdx.x >= nb_mesh) {
            frame_cell_thread<T>(f, U, ((int64_t)blockIdx.x - nb_mesh) * kThreads + threadIdx.x);
            return;
        }
    }
    const int64_t v = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (v == 0) *step += 1;
    if (v >= n_vec) return;
    int4 t[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) t[i] = __ldg(tri + 4 * v + i);
    T bo[4];
    ldw4(B + 4 * v, bo);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const T s = rn_add(rn_add(signed_load(U, t[i].x), signed_load(U, t[i].y)),
                           signed_load(U, t[i].z));
        T c;
        if constexpr (sizeof(T) == 4) c = __int_as_float(t[i].w);
        else c = __ldg(cB64 + 4 * v + i);
        bo[i] = rn_fma(-c, s, bo[i]);
    }
    st4(B + 4 * v, bo);
}

// g(t_n) of every source group for the next `count` steps, n = *step + i.
__global__ void k_gtab(double* __restrict__ g, const long long* __restrict__ step, int count,
                       int stride, const double* __restrict__ par, int n_grp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int grp = blockIdx.y;
    if (i < count && grp < n_grp)
        g[(size_t)grp * stride + i] = source_g(*step + i, par[4 * grp], par[4 * grp + 1],
                                               par[4 * grp + 2], par[4 * grp + 3]);
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

template <typename T, bool PLASMA>
void edge_half_p(const DevMesh& m, int s_index, cudaStream_t s) {
    const int64_t n_vec = m.n_ei_pad / 4;
    SrcArgs<T> src{m.src_hash, (unsigned)m.src_bits, (const T*)m.src_c, m.src_grp, m.gtab,
                   m.gtab_size, s_index};
    const T pa = PLASMA ? (T)m.pa : (T)0, mdt = PLASMA ? (T)(-m.dt) : (T)0;
    const int64_t nb = blocks_for(n_vec);
    // a frame adds its blocks to the same launch (its sides and the outer edges are vacuum)
    const FrameDev f = m.frame ? *m.frame : FrameDev();
    const int64_t nbf = m.frame ? blocks_for(f.n_fc + f.n_if) : 0;
    const unsigned grid = (unsigned)(nb + nbf);
    const int4* rl = (const int4*)m.rl;
    if (nbf > 0) {
        if (m.n_src > 0)
            k_edge_half<T, PLASMA, true, true><<<grid, kThreads, 0, s>>>(
                rl, (const T*)m.cU, (const T*)m.B, (T*)m.U, (const T*)m.pb, (T*)m.J, pa, mdt, n_vec, src, f, nb);
        else
            k_edge_half<T, PLASMA, false, true><<<grid, kThreads, 0, s>>>(
                rl, (const T*)m.cU, (const T*)m.B, (T*)m.U, (const T*)m.pb, (T*)m.J, pa, mdt, n_vec, src, f, nb);
    } else if (m.n_src > 0) {
        k_edge_half<T, PLASMA, true, false><<<grid, kThreads, 0, s>>>(
            rl, (const T*)m.cU, (const T*)m.B, (T*)m.U, (const T*)m.pb, (T*)m.J, pa, mdt, n_vec, src, f, nb);
    } else {
        k_edge_half<T, PLASMA, false, false><<<grid, kThreads, 0, s>>>(
            rl, (const T*)m.cU, (const T*)m.B, (T*)m.U, (const T*)m.pb, (T*)m.J, pa, mdt, n_vec, src, f, nb);
    }
}

template <typename T>
void tri_half_t(const DevMesh& m, cudaStream_t s) {
    const int64_t n_vec = m.n_t_pad / 4;
    const int64_t nb = blocks_for(n_vec);
    if (m.frame) {
        const int64_t nbf = blocks_for(m.frame->n_fc);
        k_tri_half<T, true><<<(unsigned)(nb + nbf), kThreads, 0, s>>>(
            m.tri, (const double*)m.cB, (const T*)m.U, (T*)m.B, n_vec, m.step, *m.frame, nb);
    } else {
        k_tri_half<T, false><<<(unsigned)nb, kThreads, 0, s>>>(m.tri, (const double*)m.cB, (const T*)m.U,
                                                              (T*)m.B, n_vec, m.step, FrameDev(), nb);
    }
}

}  // namespace

cudaError_t launch_gtab(const DevMesh& m, int count, cudaStream_t s) {
    if (m.n_src == 0 || count <= 0) return cudaSuccess;
    k_gtab<<<dim3((count + 63) / 64, m.n_grp), 64, 0, s>>>(m.gtab, m.step, count, m.gtab_size,
                                                          m.grp_par, m.n_grp);
    return cudaGetLastError();
}

cudaError_t launch_step_part(const DevMesh& m, int part, int s_index, cudaStream_t s) {
    const bool f64 = m.precision == UE_PREC_FP64;
    if (part == 0) {
        if (f64) m.plasma ? edge_half_p<double, true>(m, s_index, s) : edge_half_p<double, false>(m, s_index, s);
        else m.plasma ? edge_half_p<float, true>(m, s_index, s) : edge_half_p<float, false>(m, s_index, s);
    } else {
        f64 ? tri_half_t<double>(m, s) : tri_half_t<float>(m, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_steps_plain(const DevMesh& m, int count, cudaStream_t s) {
    cudaError_t e = launch_gtab(m, count, s);
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        e = launch_step_part(m, 0, i, s);
        if (e == cudaSuccess) e = launch_step_part(m, 1, i, s);
    }
    return e;
}

}  // namespace ue
