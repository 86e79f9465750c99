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
#include <cstddef>

#include "device.cuh"

namespace ue {

namespace {

constexpr int kH = 64, kD = 12;
constexpr int kOffW1 = 0, kOffB1 = kH * kD, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH, kNParams = kOffB3 + 1;
static_assert(kNParams == 5057, "parameter count");

// ---------------------------------------------------------------------------------------
// features (FP32, from FP64 geometry) and the per-triangle bracket terms
// ---------------------------------------------------------------------------------------
// Rounding slack of the FP32 bracket terms.  K_jj and the Gershgorin row bound are sums and
// products of positive values, formed from FP64 inputs by conversions and correctly rounded
// adds and multiplies (<= 2^-24 relative each), __frcp_rn (<= 2^-24) and the 2-ulp
// __fdividef and rsqrtf (<= 2^-22 each).  Along any path the errors add up to at most
// 20 * 2^-24 (11 for K_jj, 20 for the Gershgorin bound, first order), so the computed values lie
// within a factor 1 +- 20 * 2^-24 of the exact ones; scaling by 1 -+ 2^-16 keeps the bounds
// certified with 12x room.  Outside the normal FP32 range the terms give no bound (K_jj -> 0,
// Gershgorin -> +inf).
constexpr double kBracketSlack = 1.0 / 65536.0;

// One triangle's features, FP32.  The edge vectors are differences taken in FP64 (small
// triangles far from the origin lose nothing), then rounded; lengths and areas enter as logs
// of ratios near 1 (fast logs: every feature is rounded to BF16 before the first layer).
// The angle opposite edge q lies at vertex q+2, between E_{q+2} and -E_{q+1}; the third angle
// is pi minus the other two.  f[12] = base = log sqrt(K_jj).  kdiag = K_jj and gersh = the
// Gershgorin row bound of S^{1/2} K S^{-1/2}, both before the slack above.  The gathers are
// issued in two dependent rounds (row j's tables, then what they point to).
__device__ __forceinline__ void triangle_features(const double* __restrict__ xy,
                                                  const int32_t* __restrict__ tn,
                                                  const int32_t* __restrict__ code,
                                                  const int32_t* __restrict__ tnb,
                                                  const double* __restrict__ elen,
                                                  const double* __restrict__ d,
                                                  const double* __restrict__ S, int64_t j,
                                                  int64_t n_ei, float* f, float& kdiag,
                                                  float& gersh) {
    int vtx[3], nb[3];
    int64_t k[3];
    for (int q = 0; q < 3; ++q) {
        vtx[q] = tn[3 * j + q];
        k[q] = code[3 * j + q] >> 1;
        nb[q] = tnb[3 * j + q];
    }
    const double Sjd = S[j];
    double px[3], py[3], el[3], dd[3], sn[3];
    for (int q = 0; q < 3; ++q) {
        px[q] = xy[2 * vtx[q]];
        py[q] = xy[2 * vtx[q] + 1];
        const bool in = k[q] < n_ei;
        el[q] = in ? elen[k[q]] : 0.0;
        dd[q] = in ? d[k[q]] : 1.0;
        sn[q] = in ? S[nb[q]] : 1.0;
    }
    float ex[3], ey[3];
    for (int q = 0; q < 3; ++q) {
        const int b = q == 2 ? 0 : q + 1;
        ex[q] = (float)(px[b] - px[q]);
        ey[q] = (float)(py[b] - py[q]);
    }
    const float Sj = (float)Sjd;
    const float invS = __frcp_rn(Sj);
    const float rs = rsqrtf(Sj);
    for (int q = 0; q < 2; ++q) {
        const int u = q + 2 > 2 ? q - 1 : q + 2, v = q + 1;
        f[q] = atan2f(fabsf(ex[u] * ey[v] - ey[u] * ex[v]), -(ex[u] * ex[v] + ey[u] * ey[v]));
    }
    f[2] = 3.14159265358979f - f[0] - f[1];
    float kd = 0.f, off = 0.f;
    bool normal = Sj >= 1e-30f;
    for (int q = 0; q < 3; ++q) {
        f[3 + q] = 0.5f * __logf((ex[q] * ex[q] + ey[q] * ey[q]) * invS);
        if (k[q] < n_ei) {
            const float dk = (float)dd[q], Sn = (float)sn[q];
            const float w = __fdividef((float)el[q], dk);
            f[6 + q] = __logf(dk * rs);
            f[9 + q] = __logf(Sn * invS);
            kd = __fadd_rn(kd, w);
            off = __fadd_rn(off, __fmul_rn(__fmul_rn(w, rs), rsqrtf(Sn)));
            normal = normal && Sn >= 1e-30f && dk >= 1e-30f;
        } else {
            f[6 + q] = 4.f;    // boundary: a dual so long the edge adds nothing to K
            f[9 + q] = 0.f;
        }
    }
    kdiag = __fmul_rn(kd, invS);
    gersh = __fadd_rn(kdiag, off);
    f[12] = kd > 0.f ? 0.5f * __logf(kdiag) : -1e30f;
    if (!normal || !(kdiag <= 1e37f) || !(gersh <= 1e37f)) {
        kdiag = 0.f;
        gersh = INFINITY;
    }
}

__global__ void k_features(const double* __restrict__ xy, const int32_t* __restrict__ tn,
                           const int32_t* __restrict__ code, const int32_t* __restrict__ tnb,
                           const double* __restrict__ elen, const double* __restrict__ d,
                           const double* __restrict__ S, int64_t n_t, int64_t n_ei,
                           float* __restrict__ X, float* __restrict__ base) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_t) return;
    float f[kD + 1], kd, ge;
    triangle_features(xy, tn, code, tnb, elen, d, S, j, n_ei, f, kd, ge);
    for (int i = 0; i < kD; ++i) X[j * kD + i] = f[i];
    base[j] = f[kD];
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

// The network as the tensor-core layers read it: BF16 weights at the padded row strides (rows
// 16-byte aligned and 8 rows of an ldmatrix on distinct banks), FP32 biases.
struct PackedNet {
    __nv_bfloat16 w1[kH * kW1S];
    __nv_bfloat16 w2[kH * kW2S];
    float b1[kH], b2[kH], w3[kH];
    float b3[4];
};
static_assert(sizeof(PackedNet) % 16 == 0, "bulk copies move multiples of 16 bytes");

// N from the parameter vector: weights to BF16 (round to nearest even), zeros in the padding.
__device__ void pack_net(PackedNet& N, const float* __restrict__ P, int tid, int nth) {
    for (int i = tid; i < kH * kW1S; i += nth) {
        const int r = i / kW1S, c = i % kW1S;
        N.w1[i] = __float2bfloat16_rn(c < kD ? P[kOffW1 + r * kD + c] : 0.f);
    }
    for (int i = tid; i < kH * kW2S; i += nth) {
        const int r = i / kW2S, c = i % kW2S;
        N.w2[i] = __float2bfloat16_rn(c < kH ? P[kOffW2 + r * kH + c] : 0.f);
    }
    for (int i = tid; i < kH; i += nth) {
        N.b1[i] = P[kOffB1 + i];
        N.b2[i] = P[kOffB2 + i];
        N.w3[i] = P[kOffW3 + i];
    }
    if (tid < 4) N.b3[tid] = tid == 0 ? P[kOffB3] : 0.f;
}

// four 8x8 BF16 matrices from shared memory; lane l supplies row (l & 7) of matrix (l >> 3)
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* row) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(row)));
}

// One 16-row tile through the network on the tensor cores.  a0..a3: the A fragments of the
// BF16 inputs (rows g and g+8, k 2t.. and 2t+8..).  The accumulators start at the biases; the
// B fragments of two n-tiles come with one ldmatrix.x4.  Returns w3 . relu(h2) for rows g (s0)
// and g+8 (s1), without b3, on all four lanes of each quad.
__device__ __forceinline__ void mlp16(const PackedNet& N, uint32_t a0, uint32_t a1, uint32_t a2,
                                      uint32_t a3, float& s0, float& s1) {
    const int lane = threadIdx.x & 31, t = lane & 3, mrow = lane & 7, mi = lane >> 3;
    float h1[8][4];
#pragma unroll
    for (int np = 0; np < 4; ++np) {
        uint32_t b[4];
        ldsm_x4(b, N.w1 + ((2 * np + (mi >> 1)) * 8 + mrow) * kW1S + (mi & 1) * 8);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int nt = 2 * np + h;
            const float2 bb = *reinterpret_cast<const float2*>(N.b1 + nt * 8 + 2 * t);
            h1[nt][0] = bb.x;
            h1[nt][1] = bb.y;
            h1[nt][2] = bb.x;
            h1[nt][3] = bb.y;
            mma_bf16(h1[nt], a0, a1, a2, a3, b[2 * h], b[2 * h + 1]);
        }
    }
    // relu, then BF16: the C fragments of layer 1 (n-tiles 2kt, 2kt+1) are the A fragments of
    // layer 2's k-tile kt
    uint32_t c[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        c[kt][0] = pack_bf16(fmaxf(h1[2 * kt][0], 0.f), fmaxf(h1[2 * kt][1], 0.f));
        c[kt][1] = pack_bf16(fmaxf(h1[2 * kt][2], 0.f), fmaxf(h1[2 * kt][3], 0.f));
        c[kt][2] = pack_bf16(fmaxf(h1[2 * kt + 1][0], 0.f), fmaxf(h1[2 * kt + 1][1], 0.f));
        c[kt][3] = pack_bf16(fmaxf(h1[2 * kt + 1][2], 0.f), fmaxf(h1[2 * kt + 1][3], 0.f));
    }
    float h2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float2 bb = *reinterpret_cast<const float2*>(N.b2 + nt * 8 + 2 * t);
        h2[nt][0] = bb.x;
        h2[nt][1] = bb.y;
        h2[nt][2] = bb.x;
        h2[nt][3] = bb.y;
    }
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
#pragma unroll
        for (int np = 0; np < 4; ++np) {
            uint32_t b[4];
            ldsm_x4(b, N.w2 + ((2 * np + (mi >> 1)) * 8 + mrow) * kW2S + kt * 16 + (mi & 1) * 8);
            mma_bf16(h2[2 * np], c[kt][0], c[kt][1], c[kt][2], c[kt][3], b[0], b[1]);
            mma_bf16(h2[2 * np + 1], c[kt][0], c[kt][1], c[kt][2], c[kt][3], b[2], b[3]);
        }
    }
    float x0 = 0.f, x1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float2 w = *reinterpret_cast<const float2*>(N.w3 + nt * 8 + 2 * t);
        x0 += w.x * fmaxf(h2[nt][0], 0.f) + w.y * fmaxf(h2[nt][1], 0.f);
        x1 += w.x * fmaxf(h2[nt][2], 0.f) + w.y * fmaxf(h2[nt][3], 0.f);
    }
    x0 += __shfl_xor_sync(0xffffffffu, x0, 1);
    x0 += __shfl_xor_sync(0xffffffffu, x0, 2);
    x1 += __shfl_xor_sync(0xffffffffu, x1, 1);
    x1 += __shfl_xor_sync(0xffffffffu, x1, 2);
    s0 = x0;
    s1 = x1;
}

// Forward on BF16 tensor cores (mma.sync m16n8k16, FP32 accumulation): one warp per 16 rows.
__global__ void __launch_bounds__(128) k_mlp_fwd_bf16(const float* __restrict__ P,
                                                      const float* __restrict__ X, int64_t n,
                                                      float* __restrict__ z) {
    __shared__ __align__(16) PackedNet net;
    pack_net(net, P, threadIdx.x, blockDim.x);
    __syncthreads();
    const float b3 = net.b3[0];
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
        float s0, s1;
        mlp16(net, a0, a1, a2, a3, s0, s1);
        if (t == 0) {
            if (r0 < n) z[r0] = s0 + b3;
            if (r1 < n) z[r1] = s1 + b3;
        }
    }
}

// Fused inference for one mesh, one launch: features -> BF16 MLP -> score z_j + base_j, the
// per-block maxima of the score (with its row), of K_jj and of the Gershgorin row bound; the
// last block to finish (counter in the work space) reduces the block partials and computes the
// Rayleigh quotient lower bound near the argmax triangle.  Each warp takes 32 triangles at a
// time: every lane builds one triangle's features in shared memory, then the warp runs the
// tensor-core layers of k_mlp_fwd_bf16 on the two 16-row halves.  No feature array is written.
constexpr int kInferWarps = 4, kInferThreads = 32 * kInferWarps;
constexpr int kRing = 6, kLoc = 256;

struct InferSmem {
    PackedNet net;
    float feat[kInferWarps][32][kD + 1];
};
static_assert(offsetof(InferSmem, feat) == sizeof(PackedNet), "packed net leads the block's smem");
constexpr int kHash = 1024;      // open-addressing table of the neighbourhood, > 4 kLoc slots
struct RqSmem {
    int32_t ids[kLoc];          // triangles of rings 0..6 around the argmax, ring by ring
    int32_t hkey[kHash];        // triangle id, -1 empty
    int32_t hval[kHash];        // local index of the member holding the key
    int32_t nbq[kLoc][3];       // triangle across each edge (-1 boundary); later its local
                                // index (-1 outside the set)
    int32_t kq[kLoc][3];        // interior edge index of each edge (>= n_ei: boundary)
    float a[kLoc][3];           // |e| / (d S_i) of each interior edge (K's off-diagonal weight)
    float sv[kLoc], v[kLoc], kv[kLoc];
};
union RhoSmem {
    InferSmem a;
    RqSmem b;
};

struct RhoPart {
    float best;
    int32_t arg;
    float kmax, gmax;
};

// max of the score, ties to the smaller row (rows < 0 are empty)
__device__ __forceinline__ void better(float& b, int32_t& a, float ob, int32_t oa) {
    if (oa >= 0 && (a < 0 || ob > b || (ob == b && oa < a))) {
        b = ob;
        a = oa;
    }
}

__device__ __forceinline__ uint32_t hash_slot(int32_t key) {
    return ((uint32_t)key * 2654435761u) >> 22;   // 10 bits: kHash = 1024
}

// slot holding key (inserted if absent), -1 when the table is full
__device__ __forceinline__ int hash_insert(RqSmem& R, int32_t key) {
    uint32_t h = hash_slot(key);
    for (int p = 0; p < kHash; ++p, h = (h + 1) & (kHash - 1)) {
        const int32_t prev = atomicCAS(&R.hkey[h], -1, key);
        if (prev == -1 || prev == key) return (int)h;
    }
    return -1;
}

__device__ __forceinline__ int hash_find(const RqSmem& R, int32_t key) {
    uint32_t h = hash_slot(key);
    for (int p = 0; p < kHash; ++p, h = (h + 1) & (kHash - 1)) {
        const int32_t k = R.hkey[h];
        if (k == key) return (int)h;
        if (k == -1) return -1;
    }
    return -1;
}

// Slack of the local Rayleigh quotient.  Any vector's quotient lower-bounds lambda_max(K), so
// the rounding of the five FP32 power steps costs only accuracy; what must be bounded is the
// rounding of <v, K v>_S and <v, v>_S for the computed v.  Three FMAs per entry of K v and
// sums of at most kLoc terms in a tree of depth <= 11 give a relative error below
// 30 * 2^-24 * G / RQ, where G >= lambda_max is the Gershgorin bound.  Scaling by 1 - 2^-12
// covers that while G / RQ <= 100; beyond, the quotient is dropped.
constexpr double kRqSlack = 1.0 / 4096.0;
constexpr double kRqMaxRatio = 100.0;

// <v, K v>_S / <v, v>_S of v = K^5 delta_j0, on the rings 0..6 around j0 (exact there: K
// couples edge neighbours only, so K^5 delta_j0 lives on rings 0..5).  Returns 0 when the
// neighbourhood exceeds kLoc triangles.
// Warp 0 walks the rings breadth first, without block barriers.  The candidates of a ring are
// the table rows of its members; their own rows are loaded as soon as they are named, so the
// deduplication (__match_any_sync keeps the first lane of equal candidates, the shared hash
// drops members already in the set) runs under the load latency.  The local order (first
// naming in candidate order, hence the rounding of the sums) does not depend on timing.  Then
// all threads form K's weights and apply the scaled operator c K (c = 1/K_j0j0, so that FP32
// does not overflow over five powers) six times.  Returns the value on every thread.
__device__ float local_rayleigh(RqSmem& R, const int32_t* __restrict__ code,
                                const int32_t* __restrict__ tnb, const double* __restrict__ elen,
                                const double* __restrict__ d, const double* __restrict__ S,
                                int64_t n_ei, int32_t j0, float* red) {
    __shared__ int s_n;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31;
    for (int i = tid; i < kHash; i += nth) R.hkey[i] = -1;
    __syncthreads();
    if (tid < 32) {
        if (lane == 0) {
            R.hval[hash_insert(R, j0)] = 0;
            R.ids[0] = j0;
            for (int q = 0; q < 3; ++q) {
                R.nbq[0][q] = tnb[3 * (int64_t)j0 + q];
                R.kq[0][q] = code[3 * (int64_t)j0 + q] >> 1;
            }
            R.sv[0] = (float)S[j0];
        }
        __syncwarp();
        int n = 1, start = 0, end = 1;
        bool over = false;
        for (int r = 1; r <= kRing && !over; ++r) {
            const int cnt = 3 * (end - start);
            for (int c0 = 0; c0 < cnt; c0 += 32) {
                const int c = c0 + lane;
                const int32_t o = c < cnt ? R.nbq[start + c / 3][c % 3] : -1;
                int32_t t[3] = {-1, -1, -1}, kk[3] = {0, 0, 0};
                double so = 0.0;
                if (o >= 0) {   // the candidate's rows, in flight during the deduplication
                    for (int q = 0; q < 3; ++q) {
                        t[q] = tnb[3 * (int64_t)o + q];
                        kk[q] = code[3 * (int64_t)o + q];
                    }
                    so = S[o];
                }
                const unsigned same = __match_any_sync(0xffffffffu, o);
                const bool keep = o >= 0 && lane == __ffs(same) - 1 && hash_find(R, o) < 0;
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                const int pos = n + __popc(m & ((1u << lane) - 1u));
                if (keep) {
                    const int h = pos < kLoc ? hash_insert(R, o) : -1;
                    if (h < 0) {
                        over = true;
                    } else {
                        R.hval[h] = pos;
                        R.ids[pos] = o;
                        for (int q = 0; q < 3; ++q) {
                            R.nbq[pos][q] = t[q];
                            R.kq[pos][q] = kk[q] >> 1;
                        }
                        R.sv[pos] = (float)so;
                    }
                }
                n += __popc(m);
                over = __any_sync(0xffffffffu, over);
                __syncwarp();
            }
            if (n >= kLoc) over = true;
            start = end;
            end = n;
        }
        if (lane == 0) s_n = over ? -1 : n;
    }
    __syncthreads();
    const int n = s_n;
    if (n < 0) return 0.f;
    // local neighbour indices and weights
    for (int e = tid; e < 3 * n; e += nth) {
        const int i = e / 3, q = e % 3;
        const int64_t k = R.kq[i][q];
        int loc = -1;
        float w = 0.f;
        if (k < n_ei) {
            const int h = hash_find(R, R.nbq[i][q]);
            if (h >= 0) loc = R.hval[h];
            w = __fdividef((float)elen[k], (float)d[k] * R.sv[i]);
        }
        R.nbq[i][q] = loc;
        R.a[i][q] = w;
    }
    for (int i = tid; i < n; i += nth) R.v[i] = i == 0 ? 1.f : 0.f;
    __syncthreads();
    const float kjj = R.a[0][0] + R.a[0][1] + R.a[0][2];
    if (!(kjj > 0.f)) return 0.f;
    const float c = 1.f / kjj;
    // (c K v)_i = c sum_q a_iq (v_i - v_nbr), a neighbour outside the set holding 0; six
    // products, ping-ponging between v and kv, leave (cK)^5 delta in kv and (cK)^6 delta in v
    float* va = R.v;
    float* vb = R.kv;
    for (int it = 0; it < 6; ++it) {
        for (int i = tid; i < n; i += nth) {
            const float vi = va[i];
            float acc = 0.f;
            for (int q = 0; q < 3; ++q) {
                const int nb = R.nbq[i][q];
                acc = fmaf(R.a[i][q], vi - (nb >= 0 ? va[nb] : 0.f), acc);
            }
            vb[i] = acc * c;
        }
        __syncthreads();
        float* t = va;
        va = vb;
        vb = t;
    }
    float num = 0.f, den = 0.f;
    for (int i = tid; i < n; i += nth) {
        num += R.sv[i] * R.kv[i] * R.v[i];
        den += R.sv[i] * R.kv[i] * R.kv[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    if (lane == 0) {
        red[2 * (tid >> 5)] = num;
        red[2 * (tid >> 5) + 1] = den;
    }
    __syncthreads();
    num = den = 0.f;
    for (int w = 0; w < (nth >> 5); ++w) {
        num += red[2 * w];
        den += red[2 * w + 1];
    }
    return den > 0.f ? num / (den * c) : 0.f;
}

// Resident state of the fused inference (no allocation per call): the parameters, their packed
// form, the block partials and the completion counter (zero between launches; the last block
// resets it).
constexpr int kInferMaxBlocks = 152 * 6;
__device__ float g_rho_params[kNParams];
__device__ __align__(128) PackedNet g_rho_packed;
__device__ RhoPart g_rho_parts[kInferMaxBlocks];
__device__ unsigned int g_rho_counter;

// out = {log rho_hat, row, max K_jj (rounded down), max Gershgorin (rounded up), Rayleigh
// quotient}; host-mapped memory in the library's use, any device-visible buffer works.
__global__ void __launch_bounds__(kInferThreads, 6) k_rho_infer(
    const double* __restrict__ xy, const int32_t* __restrict__ tn,
    const int32_t* __restrict__ code, const int32_t* __restrict__ tnb, const double* __restrict__ elen,
    const double* __restrict__ d, const double* __restrict__ S, int64_t n, int64_t n_ei,
    double* __restrict__ out, unsigned long long seq) {
    __shared__ __align__(128) RhoSmem sm;
    __shared__ __align__(8) uint64_t net_bar;
    __shared__ RhoPart red[kInferWarps];
    __shared__ float dred[2 * kInferWarps];
    __shared__ int s_last;
    InferSmem& A = sm.a;
    unsigned int* counter = &g_rho_counter;
    RhoPart* part = g_rho_parts;
    // the packed network arrives by one bulk copy while the first features are gathered
    if (threadIdx.x == 0) {
        mbar_init(&net_bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) bulk_g2s(&A.net, &g_rho_packed, (uint32_t)sizeof(PackedNet), &net_bar);
    bool net_ready = false;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float (*F)[kD + 1] = A.feat[warp];
    float best = -INFINITY, kmax = 0.f, gmax = 0.f;
    int32_t arg = -1;
    const int64_t warps = (int64_t)gridDim.x * kInferWarps;
    for (int64_t tile = (int64_t)blockIdx.x * kInferWarps + warp; tile * 32 < n; tile += warps) {
        const int64_t j = tile * 32 + lane;
        if (j < n) {
            float kd, ge;
            triangle_features(xy, tn, code, tnb, elen, d, S, j, n_ei, F[lane], kd, ge);
            kmax = fmaxf(kmax, kd);
            gmax = fmaxf(gmax, ge);
        } else {
            for (int i = 0; i < kD; ++i) F[lane][i] = 0.f;
            F[lane][kD] = -1e30f;
        }
        __syncwarp();
        if (!net_ready) net_ready = mbar_wait(&net_bar, 0);
        const float b3 = A.net.b3[0];
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            const float* x0 = F[16 * half + g];
            const float* x1 = F[16 * half + g + 8];
            auto xv = [&](const float* x, int c) { return c < kD ? x[c] : 0.f; };
            const uint32_t a0 = pack_bf16(xv(x0, 2 * t), xv(x0, 2 * t + 1));
            const uint32_t a1 = pack_bf16(xv(x1, 2 * t), xv(x1, 2 * t + 1));
            const uint32_t a2 = pack_bf16(xv(x0, 2 * t + 8), xv(x0, 2 * t + 9));
            const uint32_t a3 = pack_bf16(xv(x1, 2 * t + 8), xv(x1, 2 * t + 9));
            float s0, s1;
            mlp16(A.net, a0, a1, a2, a3, s0, s1);
            if (t == 0) {
                const int64_t r0 = tile * 32 + 16 * half + g, r1 = r0 + 8;
                if (r0 < n) better(best, arg, s0 + b3 + x0[kD], (int32_t)r0);
                if (r1 < n) better(best, arg, s1 + b3 + x1[kD], (int32_t)r1);
            }
        }
        __syncwarp();
    }
    // no thread leaves (and no smem is reused) while the copy may still be writing
    if (!net_ready) net_ready = mbar_wait(&net_bar, 0);
    if (!net_ready) best = NAN;   // the wait ran out: poison the prediction (power iteration)
    for (int o = 16; o > 0; o >>= 1) {
        better(best, arg, __shfl_xor_sync(0xffffffffu, best, o), __shfl_xor_sync(0xffffffffu, arg, o));
        kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    }
    if (lane == 0) red[warp] = RhoPart{best, arg, kmax, gmax};
    __syncthreads();
    if (threadIdx.x == 0) {
        RhoPart r = red[0];
        for (int w = 1; w < kInferWarps; ++w) {
            better(r.best, r.arg, red[w].best, red[w].arg);
            r.kmax = fmaxf(r.kmax, red[w].kmax);
            r.gmax = fmaxf(r.gmax, red[w].gmax);
        }
        part[blockIdx.x] = r;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // last block: every other block's partial is visible (fence before its counter update)
    __threadfence();
    best = -INFINITY;
    arg = -1;
    kmax = gmax = 0.f;
    // all of a thread's partials in flight at once (at most kInferMaxBlocks / kInferThreads)
    constexpr int kPer = (kInferMaxBlocks + kInferThreads - 1) / kInferThreads;
    float4 q[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int i = threadIdx.x + u * kInferThreads;
        q[u] = i < (int)gridDim.x ? __ldcg(reinterpret_cast<const float4*>(part + i))
                                  : make_float4(-INFINITY, __int_as_float(-1), 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        better(best, arg, q[u].x, __float_as_int(q[u].y));
        kmax = fmaxf(kmax, q[u].z);
        gmax = fmaxf(gmax, q[u].w);
    }
    for (int o = 16; o > 0; o >>= 1) {
        better(best, arg, __shfl_xor_sync(0xffffffffu, best, o), __shfl_xor_sync(0xffffffffu, arg, o));
        kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    }
    __syncthreads();
    if (lane == 0) red[warp] = RhoPart{best, arg, kmax, gmax};
    __syncthreads();
    RhoPart r = red[0];
    for (int w = 1; w < kInferWarps; ++w) {
        better(r.best, r.arg, red[w].best, red[w].arg);
        r.kmax = fmaxf(r.kmax, red[w].kmax);
        r.gmax = fmaxf(r.gmax, red[w].gmax);
    }
    double rq = r.arg >= 0 ? (double)local_rayleigh(sm.b, code, tnb, elen, d, S, n_ei, r.arg, dred) : 0.0;
    rq = rq > 0.0 && (double)r.gmax <= kRqMaxRatio * rq ? rq * (1.0 - kRqSlack) : 0.0;
    if (threadIdx.x == 0) {
        *counter = 0u;
        out[0] = (double)r.best;
        out[1] = (double)r.arg;
        out[2] = (double)r.kmax * (1.0 - kBracketSlack);
        out[3] = (double)r.gmax * (1.0 + kBracketSlack);
        out[4] = rq;
        // completion word last: the host may read out[0..4] once it sees seq
        __threadfence_system();
        reinterpret_cast<volatile unsigned long long*>(out)[5] = seq;
    }
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

}  // namespace

int mlp_n_params() { return kNParams; }

cudaError_t launch_features(const double* xy, const int32_t* tri_nodes, const int32_t* tri_code,
                            const int32_t* tri_nb, const double* elen, const double* d, const double* S,
                            int64_t n_t, int64_t n_ei, float* X, float* base, cudaStream_t s) {
    if (n_t <= 0) return cudaSuccess;
    k_features<<<(unsigned)((n_t + 255) / 256), 256, 0, s>>>(xy, tri_nodes, tri_code, tri_nb, elen, d, S,
                                                             n_t, n_ei, X, base);
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

// g_rho_packed from g_rho_params: weights to BF16 (round to nearest even) at the padded smem
// strides, zeros in the padding.
__global__ void k_pack_net() { pack_net(g_rho_packed, g_rho_params, threadIdx.x, blockDim.x); }

// Blocks of the fused inference: enough for every warp to take one 32-triangle tile, at most
// 6 resident blocks on each of the 152 SMs.
static int rho_infer_grid(int64_t n_t) {
    const int64_t need = (n_t + kInferThreads - 1) / kInferThreads;
    return (int)(need < 1 ? 1 : need > kInferMaxBlocks ? kInferMaxBlocks : need);
}

cudaError_t rho_infer_upload(const float* P_host, cudaStream_t s) {
    cudaError_t e = cudaMemcpyToSymbolAsync(g_rho_params, P_host, sizeof(float) * kNParams, 0,
                                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    k_pack_net<<<1, 256, 0, s>>>();
    return cudaGetLastError();
}

cudaError_t launch_rho_infer(const double* xy, const int32_t* tri_nodes, const int32_t* tri_code,
                             const int32_t* tri_nb, const double* elen, const double* d, const double* S,
                             int64_t n_t, int64_t n_ei, double* out, unsigned long long seq,
                             cudaStream_t s) {
    k_rho_infer<<<rho_infer_grid(n_t), kInferThreads, 0, s>>>(xy, tri_nodes, tri_code, tri_nb, elen, d,
                                                             S, n_t, n_ei, out, seq);
    return cudaGetLastError();
}

}  // namespace ue
