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
// Rounding slack of the FP32 bracket terms.  K_jj and the Gershgorin row bound are sums,
// products, quotients and square roots of positive values, formed from FP64 inputs with at
// most 12 conversions and correctly rounded FP32 operations on any path (relative error
// <= 2^-24 each), so the computed value lies within a factor 1 +- 12 * 2^-24 of the exact
// one.  Scaling by 1 -+ 2^-16 keeps the bounds certified with 20x room.  Outside the normal
// FP32 range the terms give no bound (K_jj -> 0, Gershgorin -> +inf).
constexpr double kBracketSlack = 1.0 / 65536.0;

// One triangle's features, FP32 (coordinate differences taken in FP64 first, so that small
// triangles far from the origin lose nothing; GB300's FP64 pipes are few, and every feature
// ends in FP32 or BF16 anyway).  f[12] = base = log sqrt(K_jj).  kdiag = K_jj and gersh = the
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
    const float Sj = (float)Sjd;
    const float sq = __fsqrt_rn(Sj);
    const float rs = 1.f / sq;
    float kd = 0.f, off = 0.f;
    bool normal = Sj >= 1e-30f;
    for (int q = 0; q < 3; ++q) {
        const int a = q, b = (q + 1) % 3, o = (q + 2) % 3;
        const float ux = (float)(px[a] - px[o]), uy = (float)(py[a] - py[o]);
        const float vx = (float)(px[b] - px[o]), vy = (float)(py[b] - py[o]);
        f[q] = atan2f(fabsf(ux * vy - uy * vx), ux * vx + uy * vy);
        f[3 + q] = logf(hypotf((float)(px[b] - px[a]), (float)(py[b] - py[a])) * rs);
        if (k[q] < n_ei) {
            const float dk = (float)dd[q], Sn = (float)sn[q];
            const float w = __fdiv_rn((float)el[q], dk);
            f[6 + q] = logf(dk * rs);
            f[9 + q] = logf(Sn / Sj);
            kd = __fadd_rn(kd, w);
            off = __fadd_rn(off, __fdiv_rn(w, __fmul_rn(sq, __fsqrt_rn(Sn))));
            normal = normal && Sn >= 1e-30f && dk >= 1e-30f;
        } else {
            f[6 + q] = 4.f;    // boundary: a dual so long the edge adds nothing to K
            f[9 + q] = 0.f;
        }
    }
    kdiag = __fdiv_rn(kd, Sj);
    gersh = __fadd_rn(kdiag, off);
    f[12] = kd > 0.f ? 0.5f * logf(kdiag) : -1e30f;
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

// Fused inference for one mesh, one launch: features -> BF16 MLP -> score z_j + base_j, the
// per-block maxima of the score (with its row), of K_jj and of the Gershgorin row bound; the
// last block to finish (counter in the work space) reduces the block partials and computes the
// Rayleigh quotient lower bound near the argmax triangle.  Each warp takes 32 triangles at a
// time: every lane builds one triangle's features in shared memory, then the warp runs the
// tensor-core layers of k_mlp_fwd_bf16 on the two 16-row halves.  No feature array is written.
constexpr int kInferWarps = 4, kInferThreads = 32 * kInferWarps;
constexpr int kRing = 6, kLoc = 256;

// The network as the tensor-core layers read it (BF16 weights padded to the smem row strides,
// FP32 biases): packed once per parameter upload, brought into shared memory by one TMA bulk
// copy per block.
struct PackedNet {
    __nv_bfloat16 w1[kH * kW1S];
    __nv_bfloat16 w2[kH * kW2S];
    float b1[kH], b2[kH], w3[kH];
    float b3[4];
};
static_assert(sizeof(PackedNet) % 16 == 0, "bulk copies move multiples of 16 bytes");
struct InferSmem {
    PackedNet net;
    float feat[kInferWarps][32][kD + 1];
};
static_assert(offsetof(InferSmem, feat) == sizeof(PackedNet), "packed net leads the block's smem");
constexpr int kHash = 1024;      // open-addressing table of the neighbourhood, > 4 kLoc slots
struct RqSmem {
    int32_t ids[kLoc];          // triangles of rings 0..6 around the argmax, ring by ring
    int32_t hkey[kHash];        // triangle id, -1 empty
    int32_t hval[kHash];        // >= 0: the smallest candidate index naming the key in the
                                // current ring; < 0: in the set, at local index -1 - hval
    union {
        int32_t cslot[3 * kLoc];    // while building: hash slot of each candidate, -1 none
        int32_t nbr[kLoc][3];       // then: local index of each neighbour, -1 outside the set
    } u;
    double a[kLoc][3];          // |e| / (d S_i) of each interior edge (K's off-diagonal weight)
    double sv[kLoc], v[kLoc], kv[kLoc];
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

// Rayleigh quotient <v, K v>_S / <v, v>_S of v = K^5 delta_j0, on the rings 0..6 around j0
// (exact there: K couples edge neighbours only, so K^5 delta_j0 lives on rings 0..5).  It
// lower-bounds lambda_max(K) = rho^2.  0 when the neighbourhood exceeds kLoc triangles.
// The rings are built breadth first; a shared hash table drops triangles already in the set
// and keeps, of the repeats within a ring, the first in candidate order, so the local order
// (and the rounding of the sums) does not depend on thread timing.  Runs on all threads of
// one block; returns the value on every thread.
__device__ double local_rayleigh(RqSmem& R, const int32_t* __restrict__ code,
                                 const int32_t* __restrict__ tnb, const double* __restrict__ elen,
                                 const double* __restrict__ d, const double* __restrict__ S,
                                 int64_t n_ei, int32_t j0, double* red) {
    __shared__ int s_n, s_over;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31;
    for (int i = tid; i < kHash; i += nth) {
        R.hkey[i] = -1;
        R.hval[i] = 0x7fffffff;
    }
    __syncthreads();
    if (tid == 0) {
        R.hval[hash_insert(R, j0)] = -1;
        R.ids[0] = j0;
        s_n = 1;
        s_over = 0;
    }
    __syncthreads();
    int start = 0;
    for (int r = 1; r <= kRing; ++r) {
        const int end = s_n, cnt = 3 * (end - start);
        for (int c = tid; c < cnt; c += nth) {
            const int32_t o = tnb[3 * (int64_t)R.ids[start + c / 3] + c % 3];
            int h = -1;
            if (o >= 0) {
                h = hash_insert(R, o);
                if (h < 0) s_over = 1;
                else atomicMin(&R.hval[h], c);
            }
            R.u.cslot[c] = h;
        }
        __syncthreads();
        if (tid < 32) {   // warp 0 appends the first naming of each new triangle, in order
            int n = end;
            for (int c0 = 0; c0 < cnt; c0 += 32) {
                const int c = c0 + lane;
                const int h = c < cnt ? R.u.cslot[c] : -1;
                const bool keep = h >= 0 && R.hval[h] == c;
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                const int pos = n + __popc(m & ((1u << lane) - 1u));
                if (keep && pos < kLoc) {
                    R.ids[pos] = R.hkey[h];
                    R.hval[h] = -1 - pos;
                }
                n += __popc(m);
            }
            if (lane == 0) {
                if (n >= kLoc) s_over = 1;
                s_n = n < kLoc ? n : kLoc;
            }
        }
        __syncthreads();
        start = end;
        if (s_over) break;
    }
    if (s_over) return 0.0;
    const int n = s_n;
    __syncthreads();   // cslot is read no more; nbr takes its place
    for (int i = tid; i < n; i += nth) {
        const int32_t j = R.ids[i];
        const double Sj = S[j];
        R.sv[i] = Sj;
        R.v[i] = i == 0 ? 1.0 : 0.0;
        int64_t k[3];
        int32_t o[3];
        for (int q = 0; q < 3; ++q) {
            k[q] = code[3 * (int64_t)j + q] >> 1;
            o[q] = tnb[3 * (int64_t)j + q];
        }
        for (int q = 0; q < 3; ++q) {
            R.u.nbr[i][q] = -1;
            R.a[i][q] = 0.0;
            if (k[q] >= n_ei) continue;
            const int h = hash_find(R, o[q]);
            if (h >= 0 && R.hval[h] < 0) R.u.nbr[i][q] = -1 - R.hval[h];
            R.a[i][q] = elen[k[q]] / (d[k[q]] * Sj);
        }
    }
    __syncthreads();
    // (K v)_i = sum_q a_iq (v_i - v_nbr), a neighbour outside the set holding 0; six products,
    // ping-ponging between v and kv, leave K^5 delta in kv and K^6 delta in v
    double* va = R.v;
    double* vb = R.kv;
    for (int it = 0; it < 6; ++it) {
        for (int i = tid; i < n; i += nth) {
            const double vi = va[i];
            double acc = 0.0;
            for (int q = 0; q < 3; ++q) {
                const int nb = R.u.nbr[i][q];
                acc = fma(R.a[i][q], vi - (nb >= 0 ? va[nb] : 0.0), acc);
            }
            vb[i] = acc;
        }
        __syncthreads();
        double* t = va;
        va = vb;
        vb = t;
    }
    double num = 0.0, den = 0.0;
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
    num = den = 0.0;
    for (int w = 0; w < (nth >> 5); ++w) {
        num += red[2 * w];
        den += red[2 * w + 1];
    }
    return den > 0.0 ? num / den : 0.0;
}

// mbarrier and bulk-copy (TMA) helpers.  Waits are bounded: a wait that runs out returns
// false and the caller poisons its result instead of hanging.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// one thread: arm the barrier for `bytes` and start the copy global -> shared (16-byte aligned
// addresses, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (int i = 0; i < (1 << 22); ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Resident state of the fused inference (no allocation per call): the parameters, their packed
// form, the block partials and the completion counter (zero between launches; the last block
// resets it).
constexpr int kInferMaxBlocks = 152 * 8;
__device__ float g_rho_params[kNParams];
__device__ __align__(128) PackedNet g_rho_packed;
__device__ RhoPart g_rho_parts[kInferMaxBlocks];
__device__ unsigned int g_rho_counter;

// out = {log rho_hat, row, max K_jj (rounded down), max Gershgorin (rounded up), Rayleigh
// quotient}; host-mapped memory in the library's use, any device-visible buffer works.
__global__ void __launch_bounds__(kInferThreads, 8) k_rho_infer(
    const double* __restrict__ xy, const int32_t* __restrict__ tn,
    const int32_t* __restrict__ code, const int32_t* __restrict__ tnb, const double* __restrict__ elen,
    const double* __restrict__ d, const double* __restrict__ S, int64_t n, int64_t n_ei,
    double* __restrict__ out) {
    __shared__ __align__(128) RhoSmem sm;
    __shared__ __align__(8) uint64_t net_bar;
    __shared__ RhoPart red[kInferWarps];
    __shared__ double dred[2 * kInferWarps];
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
            float h1[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int col = nt * 8 + 2 * t;
                h1[nt][0] = h1[nt][1] = h1[nt][2] = h1[nt][3] = 0.f;
                const __nv_bfloat16* wr = A.net.w1 + (nt * 8 + g) * kW1S;
                mma_bf16(h1[nt], a0, a1, a2, a3, *reinterpret_cast<const uint32_t*>(wr + 2 * t),
                         *reinterpret_cast<const uint32_t*>(wr + 2 * t + 8));
                h1[nt][0] = fmaxf(h1[nt][0] + A.net.b1[col], 0.f);
                h1[nt][1] = fmaxf(h1[nt][1] + A.net.b1[col + 1], 0.f);
                h1[nt][2] = fmaxf(h1[nt][2] + A.net.b1[col], 0.f);
                h1[nt][3] = fmaxf(h1[nt][3] + A.net.b1[col + 1], 0.f);
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
                    const __nv_bfloat16* wr = A.net.w2 + (nt * 8 + g) * kW2S + kt * 16;
                    mma_bf16(h2[nt], c0, c1, c2, c3, *reinterpret_cast<const uint32_t*>(wr + 2 * t),
                             *reinterpret_cast<const uint32_t*>(wr + 2 * t + 8));
                }
            }
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int col = nt * 8 + 2 * t;
                s0 += A.net.w3[col] * fmaxf(h2[nt][0] + A.net.b2[col], 0.f) + A.net.w3[col + 1] * fmaxf(h2[nt][1] + A.net.b2[col + 1], 0.f);
                s1 += A.net.w3[col] * fmaxf(h2[nt][2] + A.net.b2[col], 0.f) + A.net.w3[col + 1] * fmaxf(h2[nt][3] + A.net.b2[col + 1], 0.f);
            }
            s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
            s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
            s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
            s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
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
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        const float4 q = __ldcg(reinterpret_cast<const float4*>(part + i));
        better(best, arg, q.x, __float_as_int(q.y));
        kmax = fmaxf(kmax, q.z);
        gmax = fmaxf(gmax, q.w);
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
    const double rq = r.arg >= 0 ? local_rayleigh(sm.b, code, tnb, elen, d, S, n_ei, r.arg, dred) : 0.0;
    if (threadIdx.x == 0) {
        *counter = 0u;
        out[0] = (double)r.best;
        out[1] = (double)r.arg;
        out[2] = (double)r.kmax * (1.0 - kBracketSlack);
        out[3] = (double)r.gmax * (1.0 + kBracketSlack);
        out[4] = rq;
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
__global__ void k_pack_net() {
    PackedNet& N = g_rho_packed;
    const float* P = g_rho_params;
    for (int i = threadIdx.x; i < kH * kW1S; i += blockDim.x) {
        const int r = i / kW1S, c = i % kW1S;
        N.w1[i] = __float2bfloat16_rn(c < kD ? P[kOffW1 + r * kD + c] : 0.f);
    }
    for (int i = threadIdx.x; i < kH * kW2S; i += blockDim.x) {
        const int r = i / kW2S, c = i % kW2S;
        N.w2[i] = __float2bfloat16_rn(c < kH ? P[kOffW2 + r * kH + c] : 0.f);
    }
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        N.b1[i] = P[kOffB1 + i];
        N.b2[i] = P[kOffB2 + i];
        N.w3[i] = P[kOffW3 + i];
    }
    if (threadIdx.x < 4) N.b3[threadIdx.x] = threadIdx.x == 0 ? P[kOffB3] : 0.f;
}

// Blocks of the fused inference: enough for every warp to take one 32-triangle tile, at most
// 8 resident blocks on each of the 152 SMs.
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
                             int64_t n_t, int64_t n_ei, double* out, cudaStream_t s) {
    k_rho_infer<<<rho_infer_grid(n_t), kInferThreads, 0, s>>>(xy, tri_nodes, tri_code, tri_nb, elen, d,
                                                             S, n_t, n_ei, out);
    return cudaGetLastError();
}

}  // namespace ue
