// Features (per triangle, stored order; lengths over sqrt(S_j), ratios as logarithms):
// angles opposite the three edges, log(|e_q|/sqrt S), log(d_q/sqrt S) (4 on a boundary edge),
// log(S_neighbour/S) (0 on a boundary edge).
//
// Learned spectral radius: features, the 12-64-64-1 MLP (forward on BF16 tensor cores with
// FP32 accumulation, or an FP32 debug path), its backward pass on the argmax rows, Adam, the
// per-mesh max aggregation, and the certified bracket used to accept a prediction.
//
// The paper fixes dt by the highest mode, dt < 2/omega_max (eq. 20), found by the "complex
// time" power iteration (Section 2).  The network predicts a correction z_j per triangle from
// scale-free geometry on top of base_j = log sqrt(K_jj) (K = -L_E L_B): rho_hat =
// max_j exp(z_j + base_j).  A prediction is used only inside the bracket
// [1.05 rho_lo, rho_hi]: rho_lo from max_j K_jj and a Rayleigh quotient of K^5 delta_j* near
// the argmax triangle, rho_hi from Gershgorin on S^{1/2} K S^{-1/2} (K = -L_E L_B).
//
// Parameter layout (floats): W1 [64x12] row-major, b1 [64], W2 [64x64] row-major, b2 [64],
// w3 [64], b3 [1]  (5,057 values).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "device.cuh"

namespace ue {

namespace {

constexpr int kH = 64, kD = 12;
constexpr int kOffW1 = 0, kOffB1 = kH * kD, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH, kNParams = kOffB3 + 1;
static_assert(kNParams == 5057, "parameter count");

// ---------------------------------------------------------------------------------------
// features (FP64 geometry, FP32 output) and the per-triangle bracket terms
// ---------------------------------------------------------------------------------------
__global__ void k_features(const double* __restrict__ xy, const int32_t* __restrict__ tn,
                           const int32_t* __restrict__ code, const int2* __restrict__ rl,
                           const double* __restrict__ elen, const double* __restrict__ d,
                           const double* __restrict__ S, int64_t n_t, int64_t n_ei,
                           float* __restrict__ X, float* __restrict__ base,
                           double* __restrict__ kdiag, double* __restrict__ gersh) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_t) return;
    double px[3], py[3];
    for (int q = 0; q < 3; ++q) {
        const int v = tn[3 * j + q];
        px[q] = xy[2 * v];
        py[q] = xy[2 * v + 1];
    }
    const double Sj = S[j];
    const double rs = 1.0 / sqrt(Sj);
    double kd = 0.0, off = 0.0;
    float f[kD];
    for (int q = 0; q < 3; ++q) {
        const int a = q, b = (q + 1) % 3, o = (q + 2) % 3;
        const double ux = px[a] - px[o], uy = py[a] - py[o], vx = px[b] - px[o], vy = py[b] - py[o];
        f[q] = (float)atan2(fabs(ux * vy - uy * vx), ux * vx + uy * vy);
        f[3 + q] = (float)log(hypot(px[b] - px[a], py[b] - py[a]) * rs);
        const int c = code[3 * j + q];
        const int64_t k = c >> 1;
        if (k < n_ei) {
            const int2 e = rl[k];
            const int64_t nb = e.x == j ? e.y : e.x;
            const double w = elen[k] / d[k];
            f[6 + q] = (float)log(d[k] * rs);
            f[9 + q] = (float)log(S[nb] / Sj);
            kd += w;
            off += w / sqrt(Sj * S[nb]);
        } else {
            f[6 + q] = 4.f;    // boundary: a dual so long the edge adds nothing to K
            f[9 + q] = 0.f;
        }
    }
    for (int i = 0; i < kD; ++i) X[j * kD + i] = f[i];
    base[j] = kd > 0.0 ? (float)(0.5 * log(kd / Sj)) : -1e30f;   // log sqrt(K_jj)
    kdiag[j] = kd / Sj;
    gersh[j] = kd / Sj + off;
}

// ---------------------------------------------------------------------------------------
// forward, BF16 tensor cores: one warp per 16 rows, mma.sync m16n8k16 (row.col), FP32 accum.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

constexpr int kW1S = 16 + 8;     // smem row stride (bf16) of W1 padded to K = 16
constexpr int kW2S = 64 + 8;     // smem row stride (bf16) of W2

__global__ void __launch_bounds__(128) k_mlp_fwd_bf16(const float* __restrict__ P,
                                                      const float* __restrict__ X, int64_t n,
                                                      float* __restrict__ z) {
    __shared__ __nv_bfloat16 w1[kH * kW1S];
    __shared__ __nv_bfloat16 w2[kH * kW2S];
    __shared__ float bias1[kH], bias2[kH], w3[kH];
    for (int i = threadIdx.x; i < kH * kW1S; i += blockDim.x) {
        const int r = i / kW1S, c = i % kW1S;
        w1[i] = __float2bfloat16_rn(c < kD ? P[kOffW1 + r * kD + c] : 0.f);
    }
    for (int i = threadIdx.x; i < kH * kW2S; i += blockDim.x) {
        const int r = i / kW2S, c = i % kW2S;
        w2[i] = __float2bfloat16_rn(c < kH ? P[kOffW2 + r * kH + c] : 0.f);
    }
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        bias1[i] = P[kOffB1 + i];
        bias2[i] = P[kOffB2 + i];
        w3[i] = P[kOffW3 + i];
    }
    const float b3 = P[kOffB3];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile * 16 < n;
         tile += warps) {
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        auto xv = [&](int64_t r, int c) { return (r < n && c < kD) ? __ldg(X + r * kD + c) : 0.f; };
        const uint32_t a0 = pack_bf16(xv(r0, 2 * t), xv(r0, 2 * t + 1));
        const uint32_t a1 = pack_bf16(xv(r1, 2 * t), xv(r1, 2 * t + 1));
        const uint32_t a2 = pack_bf16(xv(r0, 2 * t + 8), xv(r0, 2 * t + 9));
        const uint32_t a3 = pack_bf16(xv(r1, 2 * t + 8), xv(r1, 2 * t + 9));
        // layer 1: [16 x 16] x [16 x 64]
        float h1[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int col = nt * 8 + 2 * t;
            h1[nt][0] = h1[nt][1] = h1[nt][2] = h1[nt][3] = 0.f;
            const __nv_bfloat16* wr = w1 + (nt * 8 + g) * kW1S;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wr + 2 * t);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wr + 2 * t + 8);
            mma_bf16(h1[nt], a0, a1, a2, a3, b0, b1);
            h1[nt][0] = fmaxf(h1[nt][0] + bias1[col], 0.f);
            h1[nt][1] = fmaxf(h1[nt][1] + bias1[col + 1], 0.f);
            h1[nt][2] = fmaxf(h1[nt][2] + bias1[col], 0.f);
            h1[nt][3] = fmaxf(h1[nt][3] + bias1[col + 1], 0.f);
        }
        // layer 2: [16 x 64] x [64 x 64]; C fragments of layer 1 are A fragments here
        float h2[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) h2[nt][0] = h2[nt][1] = h2[nt][2] = h2[nt][3] = 0.f;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const uint32_t c0 = pack_bf16(h1[2 * kt][0], h1[2 * kt][1]);
            const uint32_t c1 = pack_bf16(h1[2 * kt][2], h1[2 * kt][3]);
            const uint32_t c2 = pack_bf16(h1[2 * kt + 1][0], h1[2 * kt + 1][1]);
            const uint32_t c3 = pack_bf16(h1[2 * kt + 1][2], h1[2 * kt + 1][3]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const __nv_bfloat16* wr = w2 + (nt * 8 + g) * kW2S + kt * 16;
                const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wr + 2 * t);
                const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wr + 2 * t + 8);
                mma_bf16(h2[nt], c0, c1, c2, c3, b0, b1);
            }
        }
        // layer 3 (FP32): z = w3 . relu(a2 + b2) + b3, rows r0 and r1
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int col = nt * 8 + 2 * t;
            s0 += w3[col] * fmaxf(h2[nt][0] + bias2[col], 0.f) + w3[col + 1] * fmaxf(h2[nt][1] + bias2[col + 1], 0.f);
            s1 += w3[col] * fmaxf(h2[nt][2] + bias2[col], 0.f) + w3[col + 1] * fmaxf(h2[nt][3] + bias2[col + 1], 0.f);
        }
        s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
        s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
        if (t == 0) {
            if (r0 < n) z[r0] = s0 + b3;
            if (r1 < n) z[r1] = s1 + b3;
        }
    }
}

// Fused inference for one mesh: features -> BF16 MLP -> z_j + base_j, with per-block maxima
// of that score (and its row), of K_jj and of the Gershgorin row bound.  One warp handles 16
// triangles at a time: lanes 0..15 build one triangle's features each (FP64 geometry) in
// shared memory, then the warp runs the same tensor-core layers as k_mlp_fwd_bf16.  No
// feature array is written.  part[4 * block] = {best score, row (as double), max K_jj, max
// Gershgorin bound}.
__device__ __forceinline__ void triangle_features(const double* __restrict__ xy,
                                                  const int32_t* __restrict__ tn,
                                                  const int32_t* __restrict__ code,
                                                  const int2* __restrict__ rl,
                                                  const double* __restrict__ elen,
                                                  const double* __restrict__ d,
                                                  const double* __restrict__ S, int64_t j,
                                                  int64_t n_ei, float* f, double& kdiag,
                                                  double& gersh) {
    double px[3], py[3];
    for (int q = 0; q < 3; ++q) {
        const int v = tn[3 * j + q];
        px[q] = xy[2 * v];
        py[q] = xy[2 * v + 1];
    }
    const double Sj = S[j];
    const double rs = 1.0 / sqrt(Sj);
    double kd = 0.0, off = 0.0;
    for (int q = 0; q < 3; ++q) {
        const int a = q, b = (q + 1) % 3, o = (q + 2) % 3;
        const double ux = px[a] - px[o], uy = py[a] - py[o], vx = px[b] - px[o], vy = py[b] - py[o];
        f[q] = (float)atan2(fabs(ux * vy - uy * vx), ux * vx + uy * vy);
        f[3 + q] = (float)log(hypot(px[b] - px[a], py[b] - py[a]) * rs);
        const int c = code[3 * j + q];
        const int64_t k = c >> 1;
        if (k < n_ei) {
            const int2 e = rl[k];
            const int64_t nb = e.x == j ? e.y : e.x;
            const double w = elen[k] / d[k];
            f[6 + q] = (float)log(d[k] * rs);
            f[9 + q] = (float)log(S[nb] / Sj);
            kd += w;
            off += w / sqrt(Sj * S[nb]);
        } else {
            f[6 + q] = 4.f;
            f[9 + q] = 0.f;
        }
    }
    kdiag = kd / Sj;
    gersh = kd / Sj + off;
    f[12] = kd > 0.0 ? (float)(0.5 * log(kd / Sj)) : -1e30f;   // base = log sqrt(K_jj)
}

__global__ void __launch_bounds__(128) k_rho_infer(const float* __restrict__ P,
                                                   const double* __restrict__ xy,
                                                   const int32_t* __restrict__ tn,
                                                   const int32_t* __restrict__ code,
                                                   const int2* __restrict__ rl,
                                                   const double* __restrict__ elen,
                                                   const double* __restrict__ d,
                                                   const double* __restrict__ S, int64_t n,
                                                   int64_t n_ei, double* __restrict__ part) {
    __shared__ __nv_bfloat16 w1[kH * kW1S];
    __shared__ __nv_bfloat16 w2[kH * kW2S];
    __shared__ float bias1[kH], bias2[kH], w3[kH];
    __shared__ float feat[4][16][13];
    __shared__ double red[4][4];
    for (int i = threadIdx.x; i < kH * kW1S; i += blockDim.x) {
        const int r = i / kW1S, c = i % kW1S;
        w1[i] = __float2bfloat16_rn(c < kD ? P[kOffW1 + r * kD + c] : 0.f);
    }
    for (int i = threadIdx.x; i < kH * kW2S; i += blockDim.x) {
        const int r = i / kW2S, c = i % kW2S;
        w2[i] = __float2bfloat16_rn(c < kH ? P[kOffW2 + r * kH + c] : 0.f);
    }
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        bias1[i] = P[kOffB1 + i];
        bias2[i] = P[kOffB2 + i];
        w3[i] = P[kOffW3 + i];
    }
    const float b3 = P[kOffB3];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float (*F)[13] = feat[warp];
    double best = -1e300, arg = -1.0, kmax = 0.0, gmax = 0.0;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; tile * 16 < n; tile += warps) {
        if (lane < 16) {
            const int64_t j = tile * 16 + lane;
            if (j < n) {
                double kd, ge;
                triangle_features(xy, tn, code, rl, elen, d, S, j, n_ei, F[lane], kd, ge);
                kmax = fmax(kmax, kd);
                gmax = fmax(gmax, ge);
            } else {
                for (int i = 0; i < 12; ++i) F[lane][i] = 0.f;
                F[lane][12] = -1e30f;
            }
        }
        __syncwarp();
        auto xv = [&](int r, int c) { return c < kD ? F[r][c] : 0.f; };
        const uint32_t a0 = pack_bf16(xv(g, 2 * t), xv(g, 2 * t + 1));
        const uint32_t a1 = pack_bf16(xv(g + 8, 2 * t), xv(g + 8, 2 * t + 1));
        const uint32_t a2 = pack_bf16(xv(g, 2 * t + 8), xv(g, 2 * t + 9));
        const uint32_t a3 = pack_bf16(xv(g + 8, 2 * t + 8), xv(g + 8, 2 * t + 9));
        float h1[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int col = nt * 8 + 2 * t;
            h1[nt][0] = h1[nt][1] = h1[nt][2] = h1[nt][3] = 0.f;
            const __nv_bfloat16* wr = w1 + (nt * 8 + g) * kW1S;
            mma_bf16(h1[nt], a0, a1, a2, a3, *reinterpret_cast<const uint32_t*>(wr + 2 * t),
                     *reinterpret_cast<const uint32_t*>(wr + 2 * t + 8));
            h1[nt][0] = fmaxf(h1[nt][0] + bias1[col], 0.f);
            h1[nt][1] = fmaxf(h1[nt][1] + bias1[col + 1], 0.f);
            h1[nt][2] = fmaxf(h1[nt][2] + bias1[col], 0.f);
            h1[nt][3] = fmaxf(h1[nt][3] + bias1[col + 1], 0.f);
        }
        float h2[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) h2[nt][0] = h2[nt][1] = h2[nt][2] = h2[nt][3] = 0.f;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const uint32_t c0 = pack_bf16(h1[2 * kt][0], h1[2 * kt][1]);
            const uint32_t c1 = pack_bf16(h1[2 * kt][2], h1[2 * kt][3]);
            const uint32_t c2 = pack_bf16(h1[2 * kt + 1][0], h1[2 * kt + 1][1]);
            const uint32_t c3 = pack_bf16(h1[2 * kt + 1][2], h1[2 * kt + 1][3]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const __nv_bfloat16* wr = w2 + (nt * 8 + g) * kW2S + kt * 16;
                mma_bf16(h2[nt], c0, c1, c2, c3, *reinterpret_cast<const uint32_t*>(wr + 2 * t),
                         *reinterpret_cast<const uint32_t*>(wr + 2 * t + 8));
            }
        }
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int col = nt * 8 + 2 * t;
            s0 += w3[col] * fmaxf(h2[nt][0] + bias2[col], 0.f) + w3[col + 1] * fmaxf(h2[nt][1] + bias2[col + 1], 0.f);
            s1 += w3[col] * fmaxf(h2[nt][2] + bias2[col], 0.f) + w3[col + 1] * fmaxf(h2[nt][3] + bias2[col + 1], 0.f);
        }
        s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
        s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
        if (t == 0) {
            const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
            const double v0 = (double)(s0 + b3 + F[g][12]), v1 = (double)(s1 + b3 + F[g + 8][12]);
            if (r0 < n && v0 > best) { best = v0; arg = (double)r0; }
            if (r1 < n && v1 > best) { best = v1; arg = (double)r1; }
        }
        __syncwarp();
    }
    // warp then block maxima (ties: smaller row)
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o), oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (ob > best || (ob == best && oa >= 0 && (arg < 0 || oa < arg))) { best = ob; arg = oa; }
        kmax = fmax(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    }
    if (lane == 0) {
        red[warp][0] = best;
        red[warp][1] = arg;
        red[warp][2] = kmax;
        red[warp][3] = gmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 4; ++w) {
            if (red[w][0] > red[0][0] || (red[w][0] == red[0][0] && red[w][1] >= 0 && (red[0][1] < 0 || red[w][1] < red[0][1]))) {
                red[0][0] = red[w][0];
                red[0][1] = red[w][1];
            }
            red[0][2] = fmax(red[0][2], red[w][2]);
            red[0][3] = fmax(red[0][3], red[w][3]);
        }
        for (int i = 0; i < 4; ++i) part[4 * blockIdx.x + i] = red[0][i];
    }
}

// out = {best score, row, max K_jj, max Gershgorin} over the block partials; row also as int64.
__global__ void k_rho_reduce(const double* __restrict__ part, int nb, double* __restrict__ out,
                             int64_t* __restrict__ arg) {
    if (threadIdx.x != 0) return;
    double b = -1e300, a = -1.0, k = 0.0, g = 0.0;
    for (int i = 0; i < nb; ++i) {
        const double pb = part[4 * i], pa = part[4 * i + 1];
        if (pb > b || (pb == b && pa >= 0 && (a < 0 || pa < a))) { b = pb; a = pa; }
        k = fmax(k, part[4 * i + 2]);
        g = fmax(g, part[4 * i + 3]);
    }
    out[0] = b;
    out[1] = a;
    out[2] = k;
    out[3] = g;
    *arg = (int64_t)a;
}

// FP32 debug forward: one thread per row, CUDA cores.
__global__ void k_mlp_fwd_f32(const float* __restrict__ P, const float* __restrict__ X, int64_t n,
                              float* __restrict__ z) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float x[kD], h1[kH];
    for (int i = 0; i < kD; ++i) x[i] = X[r * kD + i];
    for (int o = 0; o < kH; ++o) {
        float a = P[kOffB1 + o];
        for (int i = 0; i < kD; ++i) a = fmaf(P[kOffW1 + o * kD + i], x[i], a);
        h1[o] = fmaxf(a, 0.f);
    }
    float s = P[kOffB3];
    for (int o = 0; o < kH; ++o) {
        float a = P[kOffB2 + o];
        for (int i = 0; i < kH; ++i) a = fmaf(P[kOffW2 + o * kH + i], h1[i], a);
        s = fmaf(P[kOffW3 + o], fmaxf(a, 0.f), s);
    }
    z[r] = s;
}

// ---------------------------------------------------------------------------------------
// backward for selected rows: per-row gradient rows (deterministic), reduced in fixed order.
// bf16 = 1 repeats the forward's BF16 rounding of x, W1, W2 and h1.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float rb(float x, int bf16) {
    return bf16 ? __bfloat162float(__float2bfloat16_rn(x)) : x;
}

__global__ void __launch_bounds__(64) k_mlp_bwd_rows(const float* __restrict__ P,
                                                     const float* __restrict__ X,
                                                     const int64_t* __restrict__ rows,
                                                     const float* __restrict__ dz, int bf16,
                                                     float* __restrict__ G) {
    const int64_t m = blockIdx.x;
    const int o = threadIdx.x;   // hidden unit
    __shared__ float x[kD], h1[kH], d2[kH];
    const int64_t r = rows[m];
    if (o < kD) x[o] = rb(X[r * kD + o], bf16);
    __syncthreads();
    float a1 = P[kOffB1 + o];
    for (int i = 0; i < kD; ++i) a1 += rb(P[kOffW1 + o * kD + i], bf16) * x[i];
    h1[o] = rb(fmaxf(a1, 0.f), bf16);
    __syncthreads();
    float a2 = P[kOffB2 + o];
    for (int i = 0; i < kH; ++i) a2 += rb(P[kOffW2 + o * kH + i], bf16) * h1[i];
    const float g = dz[m];
    float* Gm = G + m * (int64_t)kNParams;
    const float h2 = fmaxf(a2, 0.f);
    Gm[kOffW3 + o] = g * h2;
    if (o == 0) Gm[kOffB3] = g;
    const float dd2 = a2 > 0.f ? g * P[kOffW3 + o] : 0.f;
    d2[o] = dd2;
    Gm[kOffB2 + o] = dd2;
    for (int i = 0; i < kH; ++i) Gm[kOffW2 + o * kH + i] = dd2 * h1[i];
    __syncthreads();
    float d1 = 0.f;
    for (int i = 0; i < kH; ++i) d1 += d2[i] * rb(P[kOffW2 + i * kH + o], bf16);
    d1 = a1 > 0.f ? d1 : 0.f;
    Gm[kOffB1 + o] = d1;
    for (int i = 0; i < kD; ++i) Gm[kOffW1 + o * kD + i] = d1 * x[i];
}

__global__ void k_colsum(const float* __restrict__ G, int64_t m, float* __restrict__ g) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kNParams) return;
    float s = 0.f;
    for (int64_t i = 0; i < m; ++i) s += G[i * kNParams + p];
    g[p] = s;
}

// Adam (Kingma & Ba 2015) with bias correction.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mi = b1 * m[i] + (1.f - b1) * g[i];
    const float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Per segment (mesh): best = max_j (z_j + base_j) and its row (first on ties).
__global__ void k_seg_argmax(const float* __restrict__ z, const float* __restrict__ base,
                             const int64_t* __restrict__ off, int n_seg, float* __restrict__ best,
                             int64_t* __restrict__ arg) {
    const int s = blockIdx.x;
    if (s >= n_seg) return;
    __shared__ float bv[256];
    __shared__ int64_t bi[256];
    float v = -INFINITY;
    int64_t a = -1;
    for (int64_t j = off[s] + threadIdx.x; j < off[s + 1]; j += blockDim.x) {
        const float x = z[j] + base[j];
        if (x > v) {
            v = x;
            a = j;
        }
    }
    bv[threadIdx.x] = v;
    bi[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const float w = bv[threadIdx.x + o];
            const int64_t wi = bi[threadIdx.x + o];
            if (w > bv[threadIdx.x] || (w == bv[threadIdx.x] && wi >= 0 && (bi[threadIdx.x] < 0 || wi < bi[threadIdx.x]))) {
                bv[threadIdx.x] = w;
                bi[threadIdx.x] = wi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        best[s] = bv[0];
        arg[s] = bi[0];
    }
}

// Loss per mesh (best - target)^2 and dL/dz of its argmax row: 2 (best - target).
__global__ void k_rho_loss(const float* __restrict__ best, const float* __restrict__ target,
                           int n_seg, float* __restrict__ dz, float* __restrict__ loss) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_seg) return;
    const float r = best[s] - target[s];
    dz[s] = 2.f * r;
    loss[s] = r * r;
}

// max of a double array (block partials, then one block).
__global__ void k_max_parts(const double* __restrict__ a, int64_t n, double* __restrict__ part) {
    __shared__ double s[256];
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, a[i]);
    s[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// Rayleigh quotient of v = K^p delta_j0 (p = 5), computed on the 6-ring neighbourhood of j0
// (exact: K couples edge neighbours only).  One block; out = {lambda lower bound}.
constexpr int kRing = 6, kLoc = 512;
__global__ void k_local_rq(const int32_t* __restrict__ code, const int2* __restrict__ rl,
                           const double* __restrict__ elen, const double* __restrict__ d,
                           const double* __restrict__ S, int64_t n_ei, const int64_t* __restrict__ j0p,
                           double* __restrict__ out) {
    __shared__ int64_t ids[kLoc];
    __shared__ int nb[kLoc][3];
    __shared__ double w[kLoc][3];
    __shared__ double sv[kLoc], v[kLoc], kv[kLoc];
    __shared__ int n_loc, ring_end[kRing + 2];
    __shared__ double red[2][256];
    const int tid = threadIdx.x;
    if (tid == 0) {
        // breadth-first rings; linear search keeps this small and deterministic
        ids[0] = *j0p;
        int n = 1, start = 0;
        ring_end[0] = 1;
        for (int r = 1; r <= kRing && n < kLoc; ++r) {
            const int end = n;
            for (int i = start; i < end && n < kLoc; ++i)
                for (int q = 0; q < 3; ++q) {
                    const int64_t k = code[3 * ids[i] + q] >> 1;
                    if (k >= n_ei) continue;
                    const int2 e = rl[k];
                    const int64_t o = e.x == ids[i] ? e.y : e.x;
                    bool seen = false;
                    for (int s = 0; s < n && !seen; ++s) seen = ids[s] == o;
                    if (!seen && n < kLoc) ids[n++] = o;
                }
            start = end;
            ring_end[r] = n;
        }
        n_loc = n;
    }
    __syncthreads();
    const int n = n_loc;
    for (int i = tid; i < n; i += blockDim.x) {
        const int64_t j = ids[i];
        sv[i] = S[j];
        v[i] = i == 0 ? 1.0 : 0.0;
        for (int q = 0; q < 3; ++q) {
            const int64_t k = code[3 * j + q] >> 1;
            nb[i][q] = -1;
            w[i][q] = 0.0;
            if (k >= n_ei) continue;
            const int2 e = rl[k];
            const int64_t o = e.x == j ? e.y : e.x;
            for (int s = 0; s < n; ++s)
                if (ids[s] == o) nb[i][q] = s;
            w[i][q] = elen[k] / d[k];
        }
    }
    __syncthreads();
    // (K v)_i = (1/S_i) sum_q w_q (v_i - v_nb)  (a neighbour outside the set holds 0)
    for (int it = 0; it <= 5; ++it) {
        for (int i = tid; i < n; i += blockDim.x) {
            double a = 0.0;
            for (int q = 0; q < 3; ++q)
                if (w[i][q] != 0.0) a += w[i][q] * (v[i] - (nb[i][q] >= 0 ? v[nb[i][q]] : 0.0));
            kv[i] = a / sv[i];
        }
        __syncthreads();
        if (it < 5) {
            for (int i = tid; i < n; i += blockDim.x) v[i] = kv[i];
            __syncthreads();
        }
    }
    double num = 0.0, den = 0.0;
    for (int i = tid; i < n; i += blockDim.x) {
        num += sv[i] * v[i] * kv[i];
        den += sv[i] * v[i] * v[i];
    }
    red[0][tid] = num;
    red[1][tid] = den;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (tid < o) {
            red[0][tid] += red[0][tid + o];
            red[1][tid] += red[1][tid + o];
        }
        __syncthreads();
    }
    // a truncated neighbourhood (more than kLoc triangles) gives no bound
    if (tid == 0) out[0] = (ring_end[kRing] <= kLoc && n < kLoc && red[1][0] > 0) ? red[0][0] / red[1][0] : 0.0;
}

}  // namespace

int mlp_n_params() { return kNParams; }

cudaError_t launch_features(const double* xy, const int32_t* tri_nodes, const int32_t* tri_code,
                            const int2* rl, const double* elen, const double* d, const double* S,
                            int64_t n_t, int64_t n_ei, float* X, float* base, double* kdiag,
                            double* gersh, cudaStream_t s) {
    k_features<<<(unsigned)((n_t + 255) / 256), 256, 0, s>>>(xy, tri_nodes, tri_code, rl, elen, d, S,
                                                             n_t, n_ei, X, base, kdiag, gersh);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float* P, const float* X, int64_t n, int bf16, float* z,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (bf16) {
        const int64_t tiles = (n + 15) / 16;
        int blocks = (int)((tiles + 3) / 4);
        if (blocks > 152 * 16) blocks = 152 * 16;
        k_mlp_fwd_bf16<<<blocks, 128, 0, s>>>(P, X, n, z);
    } else {
        k_mlp_fwd_f32<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(P, X, n, z);
    }
    return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const float* P, const float* X, const int64_t* rows, const float* dz,
                                int64_t m, int bf16, float* work, float* grad, cudaStream_t s) {
    if (m <= 0) return cudaMemsetAsync(grad, 0, sizeof(float) * kNParams, s);
    k_mlp_bwd_rows<<<(unsigned)m, 64, 0, s>>>(P, X, rows, dz, bf16, work);
    k_colsum<<<(kNParams + 255) / 256, 256, 0, s>>>(work, m, grad);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1,
                        float b2, float eps, int t, cudaStream_t s) {
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_seg_argmax(const float* z, const float* base, const int64_t* off, int n_seg,
                              float* best, int64_t* arg, cudaStream_t s) {
    if (n_seg <= 0) return cudaSuccess;
    k_seg_argmax<<<n_seg, 256, 0, s>>>(z, base, off, n_seg, best, arg);
    return cudaGetLastError();
}

cudaError_t launch_rho_loss(const float* best, const float* target, int n_seg, float* dz,
                            float* loss, cudaStream_t s) {
    if (n_seg <= 0) return cudaSuccess;
    k_rho_loss<<<(n_seg + 255) / 256, 256, 0, s>>>(best, target, n_seg, dz, loss);
    return cudaGetLastError();
}

cudaError_t launch_max(const double* a, int64_t n, double* part, int n_part, double* out,
                       cudaStream_t s) {
    k_max_parts<<<n_part, 256, 0, s>>>(a, n, part);
    k_max_parts<<<1, 256, 0, s>>>(part, n_part, out);
    return cudaGetLastError();
}

int rho_infer_blocks() { return 152 * 4; }

cudaError_t launch_rho_infer(const float* P, const double* xy, const int32_t* tri_nodes,
                             const int32_t* tri_code, const int2* rl, const double* elen,
                             const double* d, const double* S, int64_t n_t, int64_t n_ei,
                             double* part, double* out, int64_t* arg, cudaStream_t s) {
    const int nb = rho_infer_blocks();
    k_rho_infer<<<nb, 128, 0, s>>>(P, xy, tri_nodes, tri_code, rl, elen, d, S, n_t, n_ei, part);
    k_rho_reduce<<<1, 32, 0, s>>>(part, nb, out, arg);
    return cudaGetLastError();
}

cudaError_t launch_local_rq(const int32_t* code, const int2* rl, const double* elen, const double* d,
                            const double* S, int64_t n_ei, const int64_t* j0, double* out,
                            cudaStream_t s) {
    k_local_rq<<<1, 256, 0, s>>>(code, rl, elen, d, S, n_ei, j0, out);
    return cudaGetLastError();
}

}  // namespace ue
