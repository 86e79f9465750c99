// Power iteration for rho(M) that allocates no device memory (ue_power_iteration_static).
//
// Some callers cannot allocate device memory while they run: code inside a fixed memory
// budget that was reserved up front, plug-ins hosted by a process that owns the allocator, or
// callers that must not take cudaMalloc's implicit synchronisation.  This entry point keeps its
// work vectors in one file-scope device array instead of asking for memory.  The caller still
// owns the inputs and the output.
//
// The array is sized for at most UE_STATIC_MAX_TRIS triangles and UE_STATIC_MAX_EDGES interior
// edges (about 8.4 MB); every GPU that loads the library holds it until the process exits.
// All calls share it, so calls that overlap on the GPU (other streams, other host threads)
// race on it.  Each call re-initialises everything it reads, including the zero slot used for
// boundary edges, so a call never depends on what an earlier one left there.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "device.cuh"

namespace ue {

namespace {

constexpr int kThreads = 256;
constexpr int64_t kMaxTris = UE_STATIC_MAX_TRIS;
constexpr int64_t kMaxEdges = UE_STATIC_MAX_EDGES;
constexpr int64_t kMaxBlocks = (kMaxTris + kThreads - 1) / kThreads;
// v[n_t] | w[n_t] | g[n_ei + 1] | block partials[2 * blocks] | sums[2] | bad-index flag
constexpr int64_t kScratch = 2 * kMaxTris + (kMaxEdges + 1) + 2 * kMaxBlocks + 3;

static __device__ __align__(256) double g_pi_scratch[kScratch];

// SplitMix64 (Steele, Lea, Flood 2014), the published mixing function.
__device__ __forceinline__ uint64_t sm64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void s_init(double* __restrict__ w, const int64_t* __restrict__ caller, uint32_t seed,
                       double* __restrict__ g, double* __restrict__ bad, int64_t n_t, int64_t n_ei) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n_t) {
        const uint64_t z = sm64(((uint64_t)seed << 32) + (uint64_t)caller[j]);
        w[j] = (double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0;
    }
    if (j == 0) {
        g[n_ei] = 0.0;   // boundary edges read this slot
        *bad = 0.0;
    }
}

// Indices that leave the caller's arrays are not followed: the element is skipped and the
// flag set, and the call returns UE_ERR_ARG.
__global__ void s_edge(const int2* __restrict__ rl, const double* __restrict__ elen,
                       const double* __restrict__ d, const double* __restrict__ v,
                       double* __restrict__ g, double* __restrict__ bad, int64_t n_t, int64_t n_ei) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_ei) return;
    const int2 e = rl[k];
    if (e.x < 0 || e.x >= n_t || e.y < 0 || e.y >= n_t) {
        *bad = 1.0;
        g[k] = 0.0;
        return;
    }
    g[k] = elen[k] * (v[e.x] - v[e.y]) / d[k];
}

// w = K v (K = -L_E L_B) and per-block sums of S v w and S w w, fixed-order tree.
__global__ void s_tri(const int32_t* __restrict__ code, const double* __restrict__ S,
                      const double* __restrict__ g, const double* __restrict__ v,
                      double* __restrict__ w, double* __restrict__ part, double* __restrict__ bad,
                      int64_t n_t, int64_t n_ei, int norm_only) {
    __shared__ double a[kThreads], b[kThreads];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double vw = 0.0, ww = 0.0;
    if (j < n_t) {
        if (norm_only) {
            ww = S[j] * v[j] * v[j];
        } else {
            int c0 = code[3 * j], c1 = code[3 * j + 1], c2 = code[3 * j + 2];
            if (c0 < 0 || (c0 >> 1) > n_ei || c1 < 0 || (c1 >> 1) > n_ei || c2 < 0 || (c2 >> 1) > n_ei) {
                *bad = 1.0;
                c0 = c1 = c2 = (int)(2 * n_ei);   // the zero slot
            }
            double x0 = g[c0 >> 1], x1 = g[c1 >> 1], x2 = g[c2 >> 1];
            if (c0 & 1) x0 = -x0;
            if (c1 & 1) x1 = -x1;
            if (c2 & 1) x2 = -x2;
            const double x = (x0 + x1 + x2) / S[j];
            w[j] = x;
            vw = S[j] * v[j] * x;
            ww = S[j] * x * x;
        }
    }
    a[threadIdx.x] = vw;
    b[threadIdx.x] = ww;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            a[threadIdx.x] += a[threadIdx.x + o];
            b[threadIdx.x] += b[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a[0];
        part[2 * blockIdx.x + 1] = b[0];
    }
}

__global__ void s_reduce(const double* __restrict__ part, int64_t nb, double* __restrict__ sums) {
    __shared__ double a[kThreads], b[kThreads];
    double x = 0.0, y = 0.0;
    for (int64_t i = threadIdx.x; i < nb; i += kThreads) {
        x += part[2 * i];
        y += part[2 * i + 1];
    }
    a[threadIdx.x] = x;
    b[threadIdx.x] = y;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            a[threadIdx.x] += a[threadIdx.x + o];
            b[threadIdx.x] += b[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sums[0] = a[0];
        sums[1] = b[0];
    }
}

__global__ void s_scale(const double* __restrict__ w, const double* __restrict__ sums,
                        double* __restrict__ v, int64_t n_t) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n_t) v[j] = w[j] / sqrt(sums[1]);
}

// Device address of the scratch array on the current device.  Looked up on every call (the
// lookup allocates nothing), so that a module reloaded after a device reset is found at its
// new address.  In host code the array's name is only a host-side handle.
cudaError_t scratch_address(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_pi_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double*>(p);
    return cudaSuccess;
}

}  // namespace

int power_iteration_static(const int32_t* edge_tri, const double* elen, const double* d,
                           const int32_t* tri_code, const double* S, const int64_t* tri_caller,
                           int64_t n_t, int64_t n_ei, int iters, uint32_t seed, cudaStream_t s,
                           double* rho, std::string& err) {
    if (n_t < 1 || n_t > kMaxTris || n_ei < 0 || n_ei > kMaxEdges) {
        err = "ue_power_iteration_static: sizes must satisfy 1 <= n_tris <= " +
              std::to_string(kMaxTris) + " and 0 <= n_interior_edges <= " + std::to_string(kMaxEdges);
        return UE_ERR_ARG;
    }
    if (iters < 1 || !edge_tri || !elen || !d || !tri_code || !S || !tri_caller || !rho) {
        err = "ue_power_iteration_static: null pointer or iters < 1";
        return UE_ERR_ARG;
    }
    double* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        err = std::string("ue_power_iteration_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return UE_ERR_CUDA;
    }
    const int64_t nb = (n_t + kThreads - 1) / kThreads;
    double* v = base;
    double* w = v + n_t;
    double* g = w + n_t;
    double* part = g + (n_ei + 1);
    double* sums = part + 2 * nb;
    double* bad = sums + 2;
    const unsigned bt = (unsigned)nb;
    const unsigned be = (unsigned)((n_ei + kThreads) / kThreads);
    const int2* rl = reinterpret_cast<const int2*>(edge_tri);
    s_init<<<bt, kThreads, 0, s>>>(w, tri_caller, seed, g, bad, n_t, n_ei);
    s_tri<<<bt, kThreads, 0, s>>>(tri_code, S, g, w, nullptr, part, bad, n_t, n_ei, 1);   // norm only
    s_reduce<<<1, kThreads, 0, s>>>(part, nb, sums);
    s_scale<<<bt, kThreads, 0, s>>>(w, sums, v, n_t);
    for (int it = 0; it < iters; ++it) {
        if (n_ei > 0) s_edge<<<be, kThreads, 0, s>>>(rl, elen, d, v, g, bad, n_t, n_ei);
        s_tri<<<bt, kThreads, 0, s>>>(tri_code, S, g, v, w, part, bad, n_t, n_ei, 0);
        s_reduce<<<1, kThreads, 0, s>>>(part, nb, sums);
        if (it + 1 < iters) s_scale<<<bt, kThreads, 0, s>>>(w, sums, v, n_t);
    }
    double h[3] = {0, 0, 0};
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        err = std::string("ue_power_iteration_static: ") + cudaGetErrorString(e);
        return UE_ERR_CUDA;
    }
    if (h[2] != 0.0) {
        err = "ue_power_iteration_static: an edge_tri entry lies outside [0, n_tris) or a tri_code "
              "entry outside [0, 2 n_interior_edges + 1]";
        return UE_ERR_ARG;
    }
    *rho = std::sqrt(h[0] > 0 ? h[0] : 0.0);
    return UE_OK;
}

}  // namespace ue
