// The leap-frog step (eqs. 14-15): the E half-step of eq. 3 (eq. 6 with the current of eq. 5
// in plasma media, plus the soft source) over interior edges, then the B half-step of eq. 4
// over triangles.  Plain form: two kernels per step, four elements per thread, so that each
// thread keeps several independent gathers in flight.
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

// Each warp takes 4 x 32 consecutive elements, element 32 i + lane of its run of 128 in pass i:
// every load instruction of the warp reads 32 consecutive records (coalesced), and its gathers
// come from 32 neighbouring elements, whose neighbours are close in the stored order.
constexpr int kPer = 4;

__device__ __forceinline__ int64_t run_base() {
    return ((int64_t)blockIdx.x * kThreads + (threadIdx.x & ~31u)) * kPer + (threadIdx.x & 31u);
}

// FRAME: blocks from nb_mesh on run a PML frame's sides and interface edges (frame.cuh); they
// write only the frame's arrays and the interface slots, which no mesh thread touches.
template <typename T, bool PLASMA, bool SRC, bool FRAME>
__global__ void __launch_bounds__(kThreads)
k_edge_half(const int2* __restrict__ rl, const T* __restrict__ cU, const T* __restrict__ B,
            T* __restrict__ U, const T* __restrict__ pb, T* __restrict__ J, T pa, T mdt,
            int64_t n_pad, SrcArgs<T> src, FrameDev f, int64_t nb_mesh) {
    // launched as a programmatic dependent of the previous kernel: wait for it, then let the
    // next kernel's blocks take the places this grid leaves free
    grid_dependency_wait();
    grid_dependents_launch();
    if constexpr (FRAME) {
        if ((int64_t)blockIdx.x >= nb_mesh) {
            frame_edge_thread<T>(f, B, U, ((int64_t)blockIdx.x - nb_mesh) * kThreads + threadIdx.x);
            return;
        }
    }
    const int64_t e0 = run_base();
    if (e0 >= n_pad) return;
    int2 r[kPer];
    T c[kPer], u[kPer], b[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int64_t e = e0 + 32 * i;
        const bool in = e < n_pad;
        r[i] = in ? __ldg(rl + e) : make_int2(0, 0);
        c[i] = in ? __ldg(cU + e) : (T)0;
        u[i] = in ? U[e] : (T)0;
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) b[i] = rn_sub(__ldg(B + r[i].x), __ldg(B + r[i].y));
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int64_t e = e0 + 32 * i;
        if (e >= n_pad) break;
        T un = rn_fma(fabs(c[i]), b[i], u[i]);
        if constexpr (PLASMA) {
            const T jj = rn_fma(pa, J[e], rn_mul(__ldg(pb + e), u[i]));
            un = rn_fma(mdt, jj, un);
            J[e] = jj;
        }
        if constexpr (SRC) {
            if (flagged(c[i])) un = source_term(src, (int)e, un);
        }
        U[e] = un;
    }
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
           const T* __restrict__ U, T* __restrict__ B, int64_t n_pad, long long* __restrict__ step,
           FrameDev f, int64_t nb_mesh) {
    grid_dependency_wait();
    grid_dependents_launch();
    if constexpr (FRAME) {
        if ((int64_t)blockIdx.x >= nb_mesh) {
            frame_cell_thread<T>(f, U, ((int64_t)blockIdx.x - nb_mesh) * kThreads + threadIdx.x);
            return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *step += 1;
    const int64_t j0 = run_base();
    if (j0 >= n_pad) return;
    int4 t[kPer];
    T bo[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int64_t j = j0 + 32 * i;
        const bool in = j < n_pad;
        t[i] = in ? __ldg(tri + j) : make_int4(0, 0, 0, 0);
        bo[i] = in ? B[j] : (T)0;
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int64_t j = j0 + 32 * i;
        const T s = rn_add(rn_add(signed_load(U, t[i].x), signed_load(U, t[i].y)),
                           signed_load(U, t[i].z));
        if (j >= n_pad) break;
        T c;
        if constexpr (sizeof(T) == 4) c = __int_as_float(t[i].w);
        else c = __ldg(cB64 + j);
        B[j] = rn_fma(-c, s, bo[i]);
    }
}

// g(t_n) of every source group for the next `count` steps, n = *step + i.
__global__ void k_gtab(double* __restrict__ g, const long long* __restrict__ step, int count,
                       int stride, const double* __restrict__ par, int n_grp) {
    grid_dependents_launch();   // the next kernel waits for this one before it reads the table
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int grp = blockIdx.y;
    if (i < count && grp < n_grp)
        g[(size_t)grp * stride + i] = source_g(*step + i, par[4 * grp], par[4 * grp + 1],
                                               par[4 * grp + 2], par[4 * grp + 3]);
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// A launch that may begin while the previous kernel of the stream finishes (programmatic
// dependent launch); the kernel waits for that kernel before it reads anything it wrote.
template <typename... P, typename... A>
cudaError_t launch_dep(void (*kern)(P...), unsigned grid, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, ((P)args)...);
}
inline unsigned blocks_for_runs(int64_t n_pad) { return blocks_for((n_pad + kPer - 1) / kPer); }

template <typename T, bool PLASMA>
cudaError_t edge_half_p(const DevMesh& m, int s_index, cudaStream_t s) {
    const int64_t n_pad = m.n_ei_pad;
    SrcArgs<T> src{m.src_hash, (unsigned)m.src_bits, (const T*)m.src_c, m.src_grp, m.gtab,
                   m.gtab_size, s_index};
    const T pa = PLASMA ? (T)m.pa : (T)0, mdt = PLASMA ? (T)(-m.dt) : (T)0;
    const int64_t nb = blocks_for_runs(n_pad);
    // a frame adds its blocks to the same launch (its sides and the outer edges are vacuum)
    const FrameDev f = m.frame ? *m.frame : FrameDev();
    const int64_t nbf = m.frame ? blocks_for(f.n_fc + f.n_if) : 0;
    const unsigned grid = (unsigned)(nb + nbf);
    const int2* rl = (const int2*)m.rl;
    auto kern = nbf > 0 ? (m.n_src > 0 ? k_edge_half<T, PLASMA, true, true> : k_edge_half<T, PLASMA, false, true>)
                        : (m.n_src > 0 ? k_edge_half<T, PLASMA, true, false> : k_edge_half<T, PLASMA, false, false>);
    return launch_dep(kern, grid, s, rl, (const T*)m.cU, (const T*)m.B, (T*)m.U, (const T*)m.pb, (T*)m.J, pa,
                      mdt, n_pad, src, f, nb);
}

template <typename T>
cudaError_t tri_half_t(const DevMesh& m, cudaStream_t s) {
    const int64_t n_pad = m.n_t_pad;
    const int64_t nb = blocks_for_runs(n_pad);
    if (m.frame) {
        const int64_t nbf = blocks_for(m.frame->n_fc);
        return launch_dep(k_tri_half<T, true>, (unsigned)(nb + nbf), s, m.tri, (const double*)m.cB,
                          (const T*)m.U, (T*)m.B, n_pad, m.step, *m.frame, nb);
    }
    return launch_dep(k_tri_half<T, false>, (unsigned)nb, s, m.tri, (const double*)m.cB, (const T*)m.U, (T*)m.B,
                      n_pad, m.step, FrameDev(), nb);
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
    cudaError_t e;
    if (part == 0) {
        if (f64) e = m.plasma ? edge_half_p<double, true>(m, s_index, s) : edge_half_p<double, false>(m, s_index, s);
        else e = m.plasma ? edge_half_p<float, true>(m, s_index, s) : edge_half_p<float, false>(m, s_index, s);
    } else {
        e = f64 ? tri_half_t<double>(m, s) : tri_half_t<float>(m, s);
    }
    return e != cudaSuccess ? e : cudaGetLastError();
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
