// The highest eigenmodes of the semi-discrete system by the "complex time" method with
// deflation (Section 2).
//
// With t -> i t the modes grow like exp(omega t), so repeated application of K = -L_E L_B to
// a vector, normalised each time, converges to the top mode; the paper finds the next modes
// the same way while keeping the ones already found from growing back.  Here the m columns of
// a block are advanced together: V <- K V, then the block is made S-orthonormal again
// (Cholesky QR: G = W^T S W = R^T R, V = W R^{-1}).  Column i is thereby kept clear of the
// directions of columns 0..i-1 at every step, which is the deflation applied to all columns at
// once.  A final Rayleigh-Ritz step on the block (eigenvectors of V^T S K V) gives the modes.
// Everything is FP64.  Blocks of vectors are row-major [n_t][m]: a triangle's m values are
// contiguous, so each gather reads one contiguous row.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "device.cuh"

namespace ue {

namespace {

constexpr int kMdThreads = 256;

// SplitMix64 (Steele, Lea, Flood 2014), published constants.
__device__ __forceinline__ uint64_t md_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

unsigned md_blocks(int64_t n) { return (unsigned)((n + kMdThreads - 1) / kMdThreads); }

// c_k = |e_k| / d_k and 1/S_j (FP64 divisions once, not per product)
__global__ void k_md_prep(const double* __restrict__ elen, const double* __restrict__ d,
                          const double* __restrict__ S, double* __restrict__ c,
                          double* __restrict__ invS, int64_t n_ei, int64_t n_t) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_ei) c[i] = elen[i] / d[i];
    if (i < n_t) invS[i] = 1.0 / S[i];
}

// V[j][col] uniform in [-1, 1), keyed by the caller id of triangle j and the column
__global__ void k_md_init(double* __restrict__ V, const int64_t* __restrict__ perm, uint32_t seed,
                          int64_t n_t, int m) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_t * m) return;
    const int64_t j = i / m;
    const int col = (int)(i - j * m);
    const uint64_t z = md_splitmix64(((uint64_t)seed << 32) + (uint64_t)perm[j] * (uint64_t)m + (uint64_t)col);
    V[i] = (double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0;
}

// g[k][col] = c_k (V[R][col] - V[L][col]); row n_ei of g is the zero row of boundary edges
__global__ void k_md_edge(const int2* __restrict__ rl, const double* __restrict__ c,
                          const double* __restrict__ V, double* __restrict__ g, int64_t n_ei, int m) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_ei * m) return;
    const int64_t k = i / m;
    const int col = (int)(i - k * m);
    const int2 e = rl[k];
    g[i] = c[k] * (V[(int64_t)e.x * m + col] - V[(int64_t)e.y * m + col]);
}

// W[j][col] = (1/S_j) sum_q s(j,q) g[k_q][col]  (K V)
__global__ void k_md_tri(const int4* __restrict__ tri, const double* __restrict__ invS,
                         const double* __restrict__ g, double* __restrict__ W, int64_t n_t, int m) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_t * m) return;
    const int64_t j = i / m;
    const int col = (int)(i - j * m);
    const int4 q = tri[j];
    double a = g[(int64_t)(q.x >> 1) * m + col], b = g[(int64_t)(q.y >> 1) * m + col],
           e = g[(int64_t)(q.z >> 1) * m + col];
    if (q.x & 1) a = -a;
    if (q.y & 1) b = -b;
    if (q.z & 1) e = -e;
    W[i] = (a + b + e) * invS[j];
}

// Block partials of the upper triangle of G[a][b] = sum_j S_j X[j][a] Y[j][b] (a <= b; G is
// symmetric for X = Y, and for Y = K X up to rounding): rows in tiles of kMdRows staged in
// shared memory, each thread owning the pairs tid, tid + 256, ... (m <= 32: at most 3 pairs of
// the 528).  Pair p enumerates (a, b) row by row.
constexpr int kMdRows = 32, kMdMaxM = 32;
__global__ void __launch_bounds__(kMdThreads) k_md_gram(const double* __restrict__ S,
                                                        const double* __restrict__ X,
                                                        const double* __restrict__ Y, int64_t n_t,
                                                        int m, double* __restrict__ part) {
    __shared__ double xs[kMdRows][kMdMaxM + 1], ys[kMdRows][kMdMaxM + 1];
    const int tid = threadIdx.x, npair = m * (m + 1) / 2;
    int pa[3], pb[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        int p = tid + u * kMdThreads, a = 0;
        while (a < m && p >= m - a) {
            p -= m - a;
            ++a;
        }
        pa[u] = a;
        pb[u] = a + p;
    }
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t r0 = (int64_t)blockIdx.x * kMdRows; r0 < n_t; r0 += (int64_t)gridDim.x * kMdRows) {
        const int rows = (int)(n_t - r0 < kMdRows ? n_t - r0 : kMdRows);
        __syncthreads();
        for (int e = tid; e < kMdRows * m; e += kMdThreads) {
            const int r = e / m, col = e - r * m;
            double x = 0.0, y = 0.0;
            if (r < rows) {
                const int64_t j = r0 + r;
                x = S[j] * X[j * m + col];
                y = Y[j * m + col];
            }
            xs[r][col] = x;
            ys[r][col] = y;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            if (tid + u * kMdThreads < npair) {
                const int a = pa[u], b = pb[u];
                double s = acc[u];
                for (int r = 0; r < kMdRows; ++r) s = fma(xs[r][a], ys[r][b], s);
                acc[u] = s;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        const int p = tid + u * kMdThreads;
        if (p < npair) part[(int64_t)blockIdx.x * npair + p] = acc[u];
    }
}

// G[p] = sum over blocks of part[b][p], in block order (deterministic)
__global__ void k_md_sum(const double* __restrict__ part, int nb, int npair, double* __restrict__ G) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npair) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * npair + p];
    G[p] = s;
}

// V[j][col] = sum_a W[j][a] T[a][col] (T is m x m, row-major; upper: T[a][col] = 0 for
// a > col).  One thread per row: the row sits in registers, T (zero-padded to MW x MW) in
// shared memory is read by every thread of a warp at the same address, and the sums are
// unrolled at compile time, so the triangle below the diagonal costs nothing.
template <int MW, bool UPPER>
__global__ void __launch_bounds__(kMdThreads) k_md_apply(const double* __restrict__ W,
                                                         const double* __restrict__ T,
                                                         double* __restrict__ V, int64_t n_t, int m) {
    __shared__ double ts[MW * MW];
    for (int e = threadIdx.x; e < MW * MW; e += blockDim.x) {
        const int r = e / MW, c = e - r * MW;
        ts[e] = (r < m && c < m) ? T[r * m + c] : 0.0;
    }
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_t) return;
    const double* w = W + j * m;
    double x[MW];
#pragma unroll
    for (int a = 0; a < MW; ++a) x[a] = a < m ? w[a] : 0.0;
    double* v = V + j * m;
#pragma unroll
    for (int col = 0; col < MW; ++col) {
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < (UPPER ? col + 1 : MW); ++a) s = fma(x[a], ts[a * MW + col], s);
        if (col < m) v[col] = s;
    }
}

template <bool UPPER>
void md_apply(const double* W, const double* T, double* V, int64_t n_t, int m, cudaStream_t s) {
    const unsigned g = md_blocks(n_t);
    if (m <= 8) k_md_apply<8, UPPER><<<g, kMdThreads, 0, s>>>(W, T, V, n_t, m);
    else if (m <= 16) k_md_apply<16, UPPER><<<g, kMdThreads, 0, s>>>(W, T, V, n_t, m);
    else if (m <= 24) k_md_apply<24, UPPER><<<g, kMdThreads, 0, s>>>(W, T, V, n_t, m);
    else k_md_apply<32, UPPER><<<g, kMdThreads, 0, s>>>(W, T, V, n_t, m);
}

// out[col * n_t + perm[j]] = V[j][col] for col < n_out (caller triangle order)
__global__ void k_md_scatter(const double* __restrict__ V, const int64_t* __restrict__ perm,
                             double* __restrict__ out, int64_t n_t, int m, int n_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_t * n_out) return;
    const int col = (int)(i / n_t);
    const int64_t j = i - (int64_t)col * n_t;
    out[(int64_t)col * n_t + perm[j]] = V[j * m + col];
}

// One step of the Chebyshev recurrence on blocks: Y1 = a (W - c Y) + b Y0, with W = K Y.
__global__ void k_md_cheb(const double* __restrict__ W, const double* __restrict__ Y,
                          const double* __restrict__ Y0, double* __restrict__ Y1, double a, double c,
                          double b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double y = a * (W[i] - c * Y[i]);
    Y1[i] = Y0 ? fma(b, Y0[i], y) : y;
}

// Gershgorin bound of S^(1/2) K S^(-1/2) (the S-symmetric form of K, same eigenvalues): row j
// has K_jj = sum_q c_q / S_j and off-diagonal c_q / sqrt(S_j S_k) for the triangle k across
// interior edge q; the largest row sum bounds lambda_max from above.  Positive doubles order
// like their bit patterns, so the maximum is an integer atomic.
__global__ void k_md_gersh(const int4* __restrict__ tri, const int2* __restrict__ rl,
                           const double* __restrict__ c, const double* __restrict__ S,
                           int64_t n_t, int64_t n_ei, unsigned long long* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_t) return;
    const int4 q = tri[j];
    const int code[3] = {q.x, q.y, q.z};
    const double sj = S[j];
    double row = 0.0;
    for (int k = 0; k < 3; ++k) {
        const int64_t e = code[k] >> 1;
        if (e >= n_ei) continue;
        const int2 t = rl[e];
        const int64_t o = t.x == j ? t.y : t.x;
        row += c[e] / sj + c[e] / sqrt(sj * S[o]);
    }
    atomicMax(out, (unsigned long long)__double_as_longlong(row));
}

// ---- host: small dense algebra on m x m matrices (m <= 32) --------------------------------

// upper-triangular R with G = R^T R; false if G is not positive definite
bool cholesky_upper(const std::vector<double>& G, int m, std::vector<double>& R) {
    R.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) {
        double s = G[(size_t)i * m + i];
        for (int k = 0; k < i; ++k) s -= R[(size_t)k * m + i] * R[(size_t)k * m + i];
        if (!(s > 0.0)) return false;
        const double rii = std::sqrt(s);
        R[(size_t)i * m + i] = rii;
        for (int j = i + 1; j < m; ++j) {
            double t = 0.5 * (G[(size_t)i * m + j] + G[(size_t)j * m + i]);
            for (int k = 0; k < i; ++k) t -= R[(size_t)k * m + i] * R[(size_t)k * m + j];
            R[(size_t)i * m + j] = t / rii;
        }
    }
    return true;
}

// inverse of an upper-triangular matrix (back substitution, column by column)
void upper_inverse(const std::vector<double>& R, int m, std::vector<double>& T) {
    T.assign((size_t)m * m, 0.0);
    for (int c = 0; c < m; ++c) {
        for (int i = c; i >= 0; --i) {
            double s = i == c ? 1.0 : 0.0;
            for (int k = i + 1; k <= c; ++k) s -= R[(size_t)i * m + k] * T[(size_t)k * m + c];
            T[(size_t)i * m + c] = s / R[(size_t)i * m + i];
        }
    }
}

// eigenpairs of a symmetric matrix by cyclic Jacobi rotations: values in lam, vectors as the
// columns of Q (row-major), sorted by decreasing eigenvalue
void jacobi_eigen(std::vector<double> A, int m, std::vector<double>& lam, std::vector<double>& Q) {
    Q.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                const double v = A[(size_t)i * m + j] * A[(size_t)i * m + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = A[(size_t)p * m + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q];
                const double theta = 0.5 * (aqq - app) / apq;
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < m; ++k) {   // A <- A J (columns p, q)
                    const double akp = A[(size_t)k * m + p], akq = A[(size_t)k * m + q];
                    A[(size_t)k * m + p] = cs * akp - sn * akq;
                    A[(size_t)k * m + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < m; ++k) {   // A <- J^T A (rows p, q)
                    const double apk = A[(size_t)p * m + k], aqk = A[(size_t)q * m + k];
                    A[(size_t)p * m + k] = cs * apk - sn * aqk;
                    A[(size_t)q * m + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < m; ++k) {   // Q <- Q J
                    const double qkp = Q[(size_t)k * m + p], qkq = Q[(size_t)k * m + q];
                    Q[(size_t)k * m + p] = cs * qkp - sn * qkq;
                    Q[(size_t)k * m + q] = sn * qkp + cs * qkq;
                }
            }
    }
    std::vector<int> ord(m);
    for (int i = 0; i < m; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return A[(size_t)a * m + a] > A[(size_t)b * m + b]; });
    std::vector<double> Qs((size_t)m * m);
    lam.resize(m);
    for (int c = 0; c < m; ++c) {
        lam[c] = A[(size_t)ord[c] * m + ord[c]];
        for (int k = 0; k < m; ++k) Qs[(size_t)k * m + c] = Q[(size_t)k * m + ord[c]];
    }
    Q = Qs;
}

}  // namespace

int modes_block_size(int n_modes) { return std::min(kMdMaxM, 2 * n_modes); }

size_t modes_work_doubles(int64_t n_t, int64_t n_ei, int m) {
    const int64_t nb = std::min<int64_t>(152 * 4, (n_t + kMdRows - 1) / kMdRows);
    return (size_t)(2 * n_t * m + (n_ei + 1) * m + n_ei + n_t + nb * (int64_t)m * (m + 1) / 2 + 2 * m * m + 8);
}

cudaError_t modes_run(const int2* rl, const int4* tri, const double* elen, const double* d,
                      const double* S, const int64_t* perm, int64_t n_t, int64_t n_ei, int n_modes,
                      int iters, uint32_t seed, double* work, double* omega, double* B_dev,
                      bool* lost_rank, cudaStream_t s) {
    const int m = modes_block_size(n_modes);
    const int npair = m * m, nup = m * (m + 1) / 2;
    const int nb = (int)std::min<int64_t>(152 * 4, (n_t + kMdRows - 1) / kMdRows);
    double* V = work;
    double* W = V + n_t * m;
    double* g = W + n_t * m;
    double* c = g + (n_ei + 1) * m;
    double* invS = c + n_ei;
    double* part = invS + n_t;
    double* G = part + (int64_t)nb * nup;
    double* T = G + npair;
    *lost_rank = false;
    cudaError_t e;
    if ((e = cudaMemsetAsync(g + n_ei * m, 0, sizeof(double) * m, s)) != cudaSuccess) return e;
    k_md_prep<<<md_blocks(std::max(n_ei, n_t)), kMdThreads, 0, s>>>(elen, d, S, c, invS, n_ei, n_t);
    k_md_init<<<md_blocks(n_t * m), kMdThreads, 0, s>>>(V, perm, seed, n_t, m);
    std::vector<double> Gu(nup), Gh(npair), R, Th;
    auto apply_K = [&](const double* X, double* Y) {
        if (n_ei > 0) k_md_edge<<<md_blocks(n_ei * m), kMdThreads, 0, s>>>(rl, c, X, g, n_ei, m);
        k_md_tri<<<md_blocks(n_t * m), kMdThreads, 0, s>>>(tri, invS, g, Y, n_t, m);
    };
    auto gram = [&](const double* X, const double* Y) -> cudaError_t {
        k_md_gram<<<nb, kMdThreads, 0, s>>>(S, X, Y, n_t, m, part);
        k_md_sum<<<(nup + 255) / 256, 256, 0, s>>>(part, nb, nup, G);
        cudaError_t e2 = cudaMemcpyAsync(Gu.data(), G, sizeof(double) * nup, cudaMemcpyDeviceToHost, s);
        if (e2 != cudaSuccess) return e2;
        if ((e2 = cudaStreamSynchronize(s)) != cudaSuccess) return e2;
        for (int a = 0, p = 0; a < m; ++a)
            for (int b = a; b < m; ++b, ++p) Gh[(size_t)a * m + b] = Gh[(size_t)b * m + a] = Gu[p];
        return cudaSuccess;
    };
    auto orthonormalize = [&](const double* X, double* Y) -> cudaError_t {   // Y = X R^{-1}
        cudaError_t e2 = gram(X, X);
        if (e2 != cudaSuccess) return e2;
        if (!cholesky_upper(Gh, m, R)) {
            *lost_rank = true;
            return cudaSuccess;
        }
        upper_inverse(R, m, Th);
        if ((e2 = cudaMemcpyAsync(T, Th.data(), sizeof(double) * npair, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return e2;
        md_apply<true>(X, T, Y, n_t, m, s);
        return cudaGetLastError();
    };
    // start: the random block made S-orthonormal (into W, then copied back by the first step)
    if ((e = orthonormalize(V, W)) != cudaSuccess || *lost_rank) return e;
    std::swap(V, W);
    for (int it = 0; it < iters; ++it) {
        apply_K(V, W);                                   // W = K V
        if ((e = orthonormalize(W, V)) != cudaSuccess || *lost_rank) return e;   // V = W R^{-1}
    }
    // Rayleigh-Ritz: H = V^T S K V, its eigenvectors rotate V into the modes
    apply_K(V, W);
    if ((e = gram(V, W)) != cudaSuccess) return e;
    std::vector<double> lam, Q;
    jacobi_eigen(Gh, m, lam, Q);
    for (int i = 0; i < n_modes; ++i) omega[i] = std::sqrt(std::max(lam[i], 0.0));
    if (B_dev) {
        if ((e = cudaMemcpyAsync(T, Q.data(), sizeof(double) * npair, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return e;
        md_apply<false>(V, T, W, n_t, m, s);
        k_md_scatter<<<md_blocks(n_t * n_modes), kMdThreads, 0, s>>>(W, perm, B_dev, n_t, m, n_modes);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

size_t modes_low_work_doubles(int64_t n_t, int64_t n_ei, int m) {
    return modes_work_doubles(n_t, n_ei, m) + 2 * (size_t)n_t * m + 8;
}

// The lowest n_modes eigenpairs of K by Chebyshev-filtered subspace iteration: each outer
// iteration applies to the block the degree-`degree` Chebyshev polynomial that stays within
// [-1, 1] on [lo, hi] (hi a certified Gershgorin bound of lambda_max, lo the block's largest
// Ritz value) and grows fast below lo, then makes the block S-orthonormal (Cholesky QR) and
// rotates it by Rayleigh-Ritz.  The columns beyond n_modes guard the convergence.  Omegas
// ascending; B_dev as in modes_run.
cudaError_t modes_low_run(const int2* rl, const int4* tri, const double* elen, const double* d,
                          const double* S, const int64_t* perm, int64_t n_t, int64_t n_ei, int n_modes,
                          int iters, int degree, uint32_t seed, double* work, double* omega,
                          double* B_dev, bool* lost_rank, cudaStream_t s) {
    const int m = modes_block_size(n_modes);
    const int npair = m * m, nup = m * (m + 1) / 2;
    const int nb = (int)std::min<int64_t>(152 * 4, (n_t + kMdRows - 1) / kMdRows);
    double* V = work;
    double* W = V + n_t * m;
    double* g = W + n_t * m;
    double* c = g + (n_ei + 1) * m;
    double* invS = c + n_ei;
    double* part = invS + n_t;
    double* G = part + (int64_t)nb * nup;
    double* T = G + npair;
    double* Y0 = work + modes_work_doubles(n_t, n_ei, m);
    double* Y1 = Y0 + n_t * m;
    unsigned long long* gmax = reinterpret_cast<unsigned long long*>(Y1 + n_t * m);
    *lost_rank = false;
    cudaError_t e;
    if ((e = cudaMemsetAsync(g + n_ei * m, 0, sizeof(double) * m, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(gmax, 0, 8, s)) != cudaSuccess) return e;
    k_md_prep<<<md_blocks(std::max(n_ei, n_t)), kMdThreads, 0, s>>>(elen, d, S, c, invS, n_ei, n_t);
    k_md_gersh<<<md_blocks(n_t), kMdThreads, 0, s>>>(tri, rl, c, S, n_t, n_ei, gmax);
    k_md_init<<<md_blocks(n_t * m), kMdThreads, 0, s>>>(V, perm, seed, n_t, m);
    unsigned long long hb = 0;
    if ((e = cudaMemcpyAsync(&hb, gmax, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    double hi;
    std::memcpy(&hi, &hb, 8);
    hi *= 1.0 + 1e-12;
    std::vector<double> Gu(nup), Gh(npair), R, Th, lam, Q;
    auto apply_K = [&](const double* X, double* Y) {
        if (n_ei > 0) k_md_edge<<<md_blocks(n_ei * m), kMdThreads, 0, s>>>(rl, c, X, g, n_ei, m);
        k_md_tri<<<md_blocks(n_t * m), kMdThreads, 0, s>>>(tri, invS, g, Y, n_t, m);
    };
    auto gram = [&](const double* X, const double* Y) -> cudaError_t {
        k_md_gram<<<nb, kMdThreads, 0, s>>>(S, X, Y, n_t, m, part);
        k_md_sum<<<(nup + 255) / 256, 256, 0, s>>>(part, nb, nup, G);
        cudaError_t e2 = cudaMemcpyAsync(Gu.data(), G, sizeof(double) * nup, cudaMemcpyDeviceToHost, s);
        if (e2 != cudaSuccess) return e2;
        if ((e2 = cudaStreamSynchronize(s)) != cudaSuccess) return e2;
        for (int a = 0, p = 0; a < m; ++a)
            for (int b = a; b < m; ++b, ++p) Gh[(size_t)a * m + b] = Gh[(size_t)b * m + a] = Gu[p];
        return cudaSuccess;
    };
    auto orthonormalize = [&](const double* X, double* Y) -> cudaError_t {   // Y = X R^{-1}
        cudaError_t e2 = gram(X, X);
        if (e2 != cudaSuccess) return e2;
        if (!cholesky_upper(Gh, m, R)) {
            *lost_rank = true;
            return cudaSuccess;
        }
        upper_inverse(R, m, Th);
        if ((e2 = cudaMemcpyAsync(T, Th.data(), sizeof(double) * npair, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return e2;
        md_apply<true>(X, T, Y, n_t, m, s);
        return cudaGetLastError();
    };
    // The block always lives in V (the work space's first n_t * m values), W is scratch; the
    // filter's recurrence rotates among V, Y0 and Y1.
    const int64_t n = n_t * m;
    auto copy_to_V = [&](const double* X) -> cudaError_t {
        return X == V ? cudaSuccess : cudaMemcpyAsync(V, X, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    };
    // V -> its Ritz vectors (V^T S K V diagonal), lam ascending
    auto rayleigh_ritz = [&]() -> cudaError_t {
        apply_K(V, W);
        cudaError_t e2 = gram(V, W);
        if (e2 != cudaSuccess) return e2;
        jacobi_eigen(Gh, m, lam, Q);
        std::reverse(lam.begin(), lam.end());
        for (int r = 0; r < m; ++r) std::reverse(Q.begin() + (size_t)r * m, Q.begin() + (size_t)(r + 1) * m);
        if ((e2 = cudaMemcpyAsync(T, Q.data(), sizeof(double) * npair, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return e2;
        md_apply<false>(V, T, W, n_t, m, s);
        return copy_to_V(W);
    };
    if ((e = orthonormalize(V, W)) != cudaSuccess || *lost_rank) return e;
    if ((e = copy_to_V(W)) != cudaSuccess) return e;
    if ((e = rayleigh_ritz()) != cudaSuccess) return e;
    std::vector<double> prev(n_modes, -1.0);
    for (int it = 0; it < iters; ++it) {
        // the interval to damp: [lo, hi], lo the block's largest Ritz value (at least a small
        // fraction of hi, so that the first filters, on a random block, damp only the top)
        const double lo = std::max(lam[m - 1], 1e-3 * hi);
        const double cc = 0.5 * (hi + lo), ee = 0.5 * (hi - lo);
        // scaled three-term recurrence: T_k((x - cc)/ee) / T_k((0 - cc)/ee) (Zhou and Saad)
        const double sig1 = ee / (0.0 - cc);
        double sig = sig1;
        apply_K(V, W);
        k_md_cheb<<<md_blocks(n), kMdThreads, 0, s>>>(W, V, nullptr, Y1, sig1 / ee, cc, 0.0, n);
        double* Yp = V;    // T_{k-1}
        double* Yc = Y1;   // T_k
        double* Yn = Y0;
        for (int k = 2; k <= degree; ++k) {
            const double sn = 1.0 / (2.0 / sig1 - sig);
            apply_K(Yc, W);
            k_md_cheb<<<md_blocks(n), kMdThreads, 0, s>>>(W, Yc, Yp, Yn, 2.0 * sn / ee, cc, -sig * sn, n);
            sig = sn;
            double* t = Yp;
            Yp = Yc;
            Yc = Yn;
            Yn = t;
        }
        if ((e = orthonormalize(Yc, W)) != cudaSuccess || *lost_rank) return e;
        if ((e = copy_to_V(W)) != cudaSuccess) return e;
        if ((e = rayleigh_ritz()) != cudaSuccess) return e;
        bool done = true;
        for (int i = 0; i < n_modes; ++i) {
            if (std::fabs(lam[i] - prev[i]) > 1e-15 * hi) done = false;
            prev[i] = lam[i];
        }
        if (done && it > 0) break;
    }
    for (int i = 0; i < n_modes; ++i) omega[i] = std::sqrt(std::max(lam[i], 0.0));
    if (B_dev) k_md_scatter<<<md_blocks(n_t * n_modes), kMdThreads, 0, s>>>(V, perm, B_dev, n_t, m, n_modes);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

}  // namespace ue
