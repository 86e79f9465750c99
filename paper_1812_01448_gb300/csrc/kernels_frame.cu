// PML frame around a mesh with a rectangular outer boundary (the paper's conclusion: a
// triangle mesh tied to a structured frame of rectangular cells that carries PML layers):
// interface geometry and field transfer.  The frame's share of each half-step runs in extra
// blocks of the plain step's kernels (frame.cuh, kernels_step.cu).
#include <cuda_runtime.h>

#include <cmath>

#include "frame.cuh"

namespace ue {

namespace {

constexpr int kThreads = 256;

unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// Interface geometry: d = (O_tri - C_e) . n_in + h/2, ic = |e| / d, icU = dt |e| / d.
template <typename T>
__global__ void k_frame_geom(FrameDev f, const double* __restrict__ O, const double* __restrict__ iface,
                             double dt) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= f.n_if) return;
    const double* g = iface + 6 * k;
    const int32_t code = f.itri[k];
    const int64_t t = code >= 0 ? code : ~code;
    const double cx = 0.5 * (g[0] + g[2]), cy = 0.5 * (g[1] + g[3]);
    const double ex = g[2] - g[0], ey = g[3] - g[1];
    const double el = sqrt(ex * ex + ey * ey);
    const double d = (O[2 * t] - cx) * g[4] + (O[2 * t + 1] - cy) * g[5] + 0.5 * f.h;
    f.ic[k] = el / d;
    ((T*)f.icU)[k] = (T)(dt * el / d);
}

template <typename T>
__global__ void k_frame_iface_out(FrameDev f, const T* __restrict__ U, const int64_t* __restrict__ iedge,
                                  const double* __restrict__ ielen, double* __restrict__ E) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < f.n_if) E[iedge[k]] = (double)U[f.u_off + k] / ielen[k];
}

template <typename T>
__global__ void k_frame_iface_in(FrameDev f, T* __restrict__ U, const int64_t* __restrict__ iedge,
                                 const double* __restrict__ ielen, const double* __restrict__ E) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < f.n_if) U[f.u_off + k] = (T)(E[iedge[k]] * ielen[k]);
}

template <typename T>
__global__ void k_frame_out(FrameDev f, double* __restrict__ B, double* __restrict__ Ex,
                            double* __restrict__ Ey) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (B && t < f.n_fc) B[t] = (double)cellB<T>(f, t);
    const int64_t nh = (int64_t)f.NX * (f.NY + 1), nv = (int64_t)(f.NX + 1) * f.NY;
    if (Ex && t < nh) {
        const int I = (int)(t % f.NX), J = (int)(t / f.NX);
        const bool unk = frame_is_cell(f, I, J - 1) && frame_is_cell(f, I, J);
        Ex[t] = unk ? (double)((const T*)f.H)[t] / f.h : 0.0;
    }
    if (Ey && t < nv) {
        const int I = (int)(t % (f.NX + 1)), J = (int)(t / (f.NX + 1));
        const bool unk = frame_is_cell(f, I - 1, J) && frame_is_cell(f, I, J);
        Ey[t] = unk ? (double)((const T*)f.V)[t] / f.h : 0.0;
    }
}

__global__ void k_region_coeff(int4* __restrict__ rtri, float* __restrict__ rcU, const int32_t* __restrict__ tgid,
                               const int32_t* __restrict__ egid, const char* __restrict__ upd, int64_t nt,
                               int64_t ne, const int4* __restrict__ tri, const float* __restrict__ cU) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nt) rtri[i].w = upd[i] ? tri[tgid[i]].w : 0;
    if (i < ne) rcU[i] = cU[egid[i]];
}

// rJ / J may be NULL (no plasma)
__global__ void k_region_gather(float* __restrict__ rB, float* __restrict__ rU, float* __restrict__ rJ,
                                const int32_t* __restrict__ tgid, const int32_t* __restrict__ egid, int64_t nt,
                                int64_t ne, const float* __restrict__ B, const float* __restrict__ U,
                                const float* __restrict__ J) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nt) rB[i] = B[tgid[i]];
    if (i < ne) {
        rU[i] = U[egid[i]];
        if (rJ) rJ[i] = J[egid[i]];
    }
}

__global__ void k_region_scatter(const float* __restrict__ rB, const float* __restrict__ rU,
                                 const float* __restrict__ rJ, const int32_t* __restrict__ tgid,
                                 const int32_t* __restrict__ egid, int64_t nt, int64_t ne, float* __restrict__ B,
                                 float* __restrict__ U, float* __restrict__ J) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nt) B[tgid[i]] = rB[i];
    if (i < ne) {
        U[egid[i]] = rU[i];
        if (rJ) J[egid[i]] = rJ[i];
    }
}

__global__ void k_region_pb(float* __restrict__ rpb, const int32_t* __restrict__ egid, int64_t ne,
                            const float* __restrict__ pb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ne) rpb[i] = pb[egid[i]];
}

template <typename T>
__global__ void k_frame_state(FrameDev f, double* __restrict__ Bx, double* __restrict__ By,
                              double* __restrict__ Ex, double* __restrict__ Ey, bool write) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    T* bx = (T*)f.Bx;
    T* by = (T*)f.By;
    T* H = (T*)f.H;
    T* V = (T*)f.V;
    if (t < f.n_fc) {
        if (write) {
            bx[t] = (T)Bx[t];
            by[t] = (T)By[t];
        } else {
            Bx[t] = (double)bx[t];
            By[t] = (double)by[t];
        }
    }
    const int64_t nh = (int64_t)f.NX * (f.NY + 1), nv = (int64_t)(f.NX + 1) * f.NY;
    if (t < nh) {
        const int I = (int)(t % f.NX), J = (int)(t / f.NX);
        const bool unk = frame_is_cell(f, I, J - 1) && frame_is_cell(f, I, J);
        if (write) {
            if (unk) H[t] = (T)(Ex[t] * f.h);
        } else {
            Ex[t] = unk ? (double)H[t] / f.h : 0.0;
        }
    }
    if (t < nv) {
        const int I = (int)(t % (f.NX + 1)), J = (int)(t / (f.NX + 1));
        const bool unk = frame_is_cell(f, I - 1, J) && frame_is_cell(f, I, J);
        if (write) {
            if (unk) V[t] = (T)(Ey[t] * f.h);
        } else {
            Ey[t] = unk ? (double)V[t] / f.h : 0.0;
        }
    }
}

}  // namespace

cudaError_t launch_frame_state(const FrameDev& f, bool f64, double* Bx, double* By, double* Ex, double* Ey,
                               bool write, cudaStream_t s) {
    int64_t n = f.n_fc;
    const int64_t nh = (int64_t)f.NX * (f.NY + 1), nv = (int64_t)(f.NX + 1) * f.NY;
    if (nh > n) n = nh;
    if (nv > n) n = nv;
    if (f64) k_frame_state<double><<<blocks_for(n), kThreads, 0, s>>>(f, Bx, By, Ex, Ey, write);
    else k_frame_state<float><<<blocks_for(n), kThreads, 0, s>>>(f, Bx, By, Ex, Ey, write);
    return cudaGetLastError();
}

cudaError_t launch_region_coeff(const RegionDev& r, const int4* tri, const float* cU, cudaStream_t s) {
    const int64_t n = r.dm.n_t > r.dm.n_ei ? r.dm.n_t : r.dm.n_ei;
    if (n == 0) return cudaSuccess;
    k_region_coeff<<<blocks_for(n), kThreads, 0, s>>>(r.dm.tri, (float*)r.dm.cU, r.tgid, r.egid, r.upd, r.dm.n_t,
                                                      r.dm.n_ei, tri, cU);
    return cudaGetLastError();
}

cudaError_t launch_region_gather(const RegionDev& r, const float* B, const float* U, const float* J,
                                 cudaStream_t s) {
    const int64_t n = r.dm.n_t > r.dm.n_ei ? r.dm.n_t : r.dm.n_ei;
    if (n == 0) return cudaSuccess;
    float* rJ = r.dm.plasma ? (float*)r.dm.J : nullptr;
    k_region_gather<<<blocks_for(n), kThreads, 0, s>>>((float*)r.dm.B, (float*)r.dm.U, rJ, r.tgid, r.egid,
                                                       r.dm.n_t, r.dm.n_ei, B, U, J);
    return cudaGetLastError();
}

cudaError_t launch_region_scatter(const RegionDev& r, float* B, float* U, float* J, cudaStream_t s) {
    const int64_t n = r.n_own_t > r.n_own_e ? r.n_own_t : r.n_own_e;
    if (n == 0) return cudaSuccess;
    const float* rJ = r.dm.plasma ? (const float*)r.dm.J : nullptr;
    k_region_scatter<<<blocks_for(n), kThreads, 0, s>>>((const float*)r.dm.B, (const float*)r.dm.U, rJ, r.tgid,
                                                        r.egid, r.n_own_t, r.n_own_e, B, U, J);
    return cudaGetLastError();
}

cudaError_t launch_region_pb(const RegionDev& r, const float* pb, cudaStream_t s) {
    if (r.dm.n_ei == 0) return cudaSuccess;
    k_region_pb<<<blocks_for(r.dm.n_ei), kThreads, 0, s>>>((float*)r.dm.pb, r.egid, r.dm.n_ei, pb);
    return cudaGetLastError();
}

cudaError_t launch_frame_geom(const FrameDev& f, const double* O, const double* iface, double dt,
                              bool f64, cudaStream_t s) {
    if (f.n_if == 0) return cudaSuccess;
    if (f64) k_frame_geom<double><<<blocks_for(f.n_if), kThreads, 0, s>>>(f, O, iface, dt);
    else k_frame_geom<float><<<blocks_for(f.n_if), kThreads, 0, s>>>(f, O, iface, dt);
    return cudaGetLastError();
}

cudaError_t launch_frame_iface_out(const FrameDev& f, const DevMesh& m, const int64_t* iedge,
                                   const double* ielen, double* E_caller, cudaStream_t s) {
    if (f.n_if == 0) return cudaSuccess;
    if (m.precision == UE_PREC_FP64)
        k_frame_iface_out<double><<<blocks_for(f.n_if), kThreads, 0, s>>>(f, (const double*)m.U, iedge, ielen, E_caller);
    else
        k_frame_iface_out<float><<<blocks_for(f.n_if), kThreads, 0, s>>>(f, (const float*)m.U, iedge, ielen, E_caller);
    return cudaGetLastError();
}

cudaError_t launch_frame_iface_in(const FrameDev& f, const DevMesh& m, const int64_t* iedge,
                                  const double* ielen, const double* E_caller, cudaStream_t s) {
    if (f.n_if == 0) return cudaSuccess;
    if (m.precision == UE_PREC_FP64)
        k_frame_iface_in<double><<<blocks_for(f.n_if), kThreads, 0, s>>>(f, (double*)m.U, iedge, ielen, E_caller);
    else
        k_frame_iface_in<float><<<blocks_for(f.n_if), kThreads, 0, s>>>(f, (float*)m.U, iedge, ielen, E_caller);
    return cudaGetLastError();
}

cudaError_t launch_frame_out(const FrameDev& f, bool f64, double* B, double* Ex, double* Ey,
                             cudaStream_t s) {
    int64_t n = f.n_fc;
    const int64_t nh = (int64_t)f.NX * (f.NY + 1), nv = (int64_t)(f.NX + 1) * f.NY;
    if (nh > n) n = nh;
    if (nv > n) n = nv;
    if (f64) k_frame_out<double><<<blocks_for(n), kThreads, 0, s>>>(f, B, Ex, Ey);
    else k_frame_out<float><<<blocks_for(n), kThreads, 0, s>>>(f, B, Ex, Ey);
    return cudaGetLastError();
}

}  // namespace ue
