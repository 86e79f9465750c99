// Device-side definitions shared by the kernels (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/ue.h"

namespace ue {

// Shared-memory copy helpers (inline PTX): mbarriers, TMA bulk copies global -> shared, and
// 4-byte cp.async gathers.  mbarrier waits are bounded: a wait that runs out returns false and
// the caller records an error instead of hanging.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's earlier shared-memory accesses before later async-proxy (TMA) writes
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// one arrival that expects `bytes` of bulk-copy transactions on bar
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// bulk copy global -> shared completing on bar (16-byte aligned addresses, bytes % 16 == 0)
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// one thread: arm the barrier for `bytes` and start one copy
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    mbar_expect_tx(bar, bytes);
    bulk_copy_g2s(dst, src, bytes, bar);
}
// Waits for the phase of `parity` to complete, for at most about a second of SM clock cycles
// (copies complete in microseconds); returns false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    for (int i = 0; i < (1 << 26); ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 255) == 255 && clock64() - t0 > (2LL << 30)) break;
    }
    return false;
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Programmatic dependent launch: wait until the grids this one depends on have completed and
// their memory is visible (returns at once for a launch without that dependency); and let the
// next launch of the stream begin (this CTA will start no further work that it would need).
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Arithmetic with explicit rounding: every variant of the step evaluates the same sequence of
// correctly rounded operations, so their results are bit-identical (no contraction choices).
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }

// g(t) of the soft source at t = (n + 1/2) dt, in FP64: sin(w0 t) exp(-((t - t0)/tau)^2).
// One out-of-line definition with explicit rounding, shared by every variant of the step.
static __device__ __noinline__ double source_g(long long n, double dt, double w0, double t0,
                                               double tau) {
    const double t = __dmul_rn(__dadd_rn((double)n, 0.5), dt);
    const double x = __ddiv_rn(__dsub_rn(t, t0), tau);
    return __dmul_rn(sin(__dmul_rn(w0, t)), exp(-__dmul_rn(x, x)));
}

// PML frame (kernels_frame.cu): W cells of side h around the mesh's bounding box, grid of
// NX x NY cells, the mesh filling cells W..W+nx-1 x W..W+ny-1.  Frame cells are numbered in
// strip order (bottom W rows, then per middle row W left and W right cells, then the top W
// rows).  Frame sides: H(I, J) at height J between columns I and I+1 (along +x), stored at
// H[J * NX + I]; V(I, J) at column I between rows J and J+1 (along +y), at V[J * (NX + 1) + I].
// Interface edge k (the mesh's outer edges): k < nx bottom (cell (W + k, W - 1) below it),
// then nx top (cell above), ny left (cell to the left), ny right; its circulation lives in the
// mesh's U array at u_off + k, in the mesh edge's direction.
struct FrameDev {
    int W = 0, nx = 0, ny = 0, NX = 0, NY = 0;
    int64_t n_fc = 0, n_if = 0;
    int64_t u_off = 0;            // first interface slot in the mesh's edge arrays (= n_ei_pad)
    double h = 0;
    void* H = nullptr;            // T [NX * (NY + 1)] circulation h E_x
    void* V = nullptr;            // T [(NX + 1) * NY] circulation h E_y
    void* Bx = nullptr;           // T [n_fc]
    void* By = nullptr;           // T [n_fc]
    int32_t* itri = nullptr;      // [n_if] stored triangle t if it is R of the edge, else ~t
    int32_t* icell = nullptr;     // [n_if] frame cell
    void* icU = nullptr;          // T [n_if] dt |e| / d
    double* ic = nullptr;         // [n_if] |e| / d (power iteration)
    void* tab = nullptr;          // T: aH, bH [NY+1]; aV, bV [NX+1]; axc, bxc [NX]; ayc, byc [NY]
};

__host__ __device__ __forceinline__ bool frame_is_cell(const FrameDev& f, int I, int J) {
    if (I < 0 || J < 0 || I >= f.NX || J >= f.NY) return false;
    return !(I >= f.W && I < f.W + f.nx && J >= f.W && J < f.W + f.ny);
}
__host__ __device__ __forceinline__ int64_t frame_cell(const FrameDev& f, int I, int J) {
    if (J < f.W) return (int64_t)J * f.NX + I;
    if (J < f.W + f.ny)
        return (int64_t)f.W * f.NX + (int64_t)(J - f.W) * 2 * f.W + (I < f.W ? I : I - f.nx);
    return (int64_t)f.W * f.NX + (int64_t)2 * f.W * f.ny + (int64_t)(J - f.W - f.ny) * f.NX + I;
}
__host__ __device__ __forceinline__ void frame_ij(const FrameDev& f, int64_t c, int& I, int& J) {
    const int64_t bot = (int64_t)f.W * f.NX, mid = (int64_t)2 * f.W * f.ny;
    if (c < bot) {
        J = (int)(c / f.NX);
        I = (int)(c % f.NX);
    } else if (c < bot + mid) {
        const int64_t r = c - bot;
        J = f.W + (int)(r / (2 * f.W));
        const int q = (int)(r % (2 * f.W));
        I = q < f.W ? q : f.nx + q;
    } else {
        const int64_t r = c - bot - mid;
        J = f.W + f.ny + (int)(r / f.NX);
        I = (int)(r % f.NX);
    }
}

// Everything the step kernels need, in the stored numbering.// Everything the step kernels need, in the stored numbering.
struct DevMesh {
    int precision = 0;            // UE_PREC_*
    int64_t n_t = 0, n_ei = 0, n_nodes = 0;
    int64_t n_ei_pad = 0;         // round_up(n_ei + 1, 4): edge arrays, incl. the zero slot
    int64_t n_t_pad = 0;          // round_up(n_t, 4): triangle arrays
    const int2* rl = nullptr;     // [n_ei_pad] (R, L); padding (0, 0)
    int4* tri = nullptr;          // [n_t_pad] {code0, code1, code2, bits of dt/S (fp32) | 0}
    void* cU = nullptr;           // [n_ei_pad] dt*|e|/d (sign bit set on source edges); pad 0
    void* cB = nullptr;           // [n_t_pad] dt/S (fp64 check build only)
    void* U = nullptr;            // [n_ei_pad] circulation |e| E; slot n_ei stays 0
    void* B = nullptr;            // [n_t_pad]
    bool plasma = false;
    void* J = nullptr;            // [n_ei_pad] circulation |e| j
    void* pb = nullptr;           // [n_ei_pad] dt*nbar/(1 + nu dt/2)
    double pa = 1.0;              // (1 - nu dt/2)/(1 + nu dt/2)
    int64_t n_src = 0;
    int32_t* src_k = nullptr;     // [n_src] stored edge ids
    int32_t* src_grp = nullptr;   // [n_src] source group (one per mesh of a batch)
    void* src_c = nullptr;        // [n_src] dt*|e|*amp
    int2* src_hash = nullptr;     // open-addressing table {edge id, source index}
    int src_bits = 0;             // table size 2^src_bits
    int n_grp = 0;
    double* grp_par = nullptr;    // [4 * n_grp] per group: dt, omega0, t0, tau
    double* gtab = nullptr;       // [n_grp * gtab_size]: g(t) per group for the current chunk
    int gtab_size = 0;
    long long* step = nullptr;    // device step counter (source time)
    double dt = 0;
    const FrameDev* frame = nullptr;   // PML frame stepped with the plain kernels, or none
};

// Device side of the temporal-blocking tiles (kernels_tb.cu, tiles_host.cpp).
struct TBDev {
    int64_t n_tiles = 0;
    int* hdr = nullptr;           // n_tiles * 48 ints
    int4* trec = nullptr;         // local triangle records {gid, codes01, code2, bits of dt/S}
    int64_t n_trec = 0;
    int* erec = nullptr;          // local edge records, 3 ints: {gid, R | L << 16, bits of cU},
                                  // the sign bit of cU set on source edges; each tile's records
                                  // start at a multiple of 4 (16-byte aligned bulk copies)
    float* epb = nullptr;         // plasma coefficient per local edge record (plasma only)
    int64_t n_erec = 0;
    int* frec = nullptr;          // fused-kernel records (tiles_host.cpp build_fused_records)
    int64_t n_frec = 0;
    int* fedge = nullptr;
    int64_t n_fedge = 0;
    int max_src = 0;              // most source records of one tile
    int2* tsrc = nullptr;         // per-tile source records {local edge, source index}
    int max_tri_loc = 0, max_edge_loc = 0;
    int threads = 512;            // CTA size of the blocked kernel (512 or 1024)
    void* B[2] = {nullptr, nullptr};
    void* U[2] = {nullptr, nullptr};
    void* J[2] = {nullptr, nullptr};
    unsigned* done = nullptr;     // [0] CTA completion counter (step counter hand-off),
                                  // [1] error word (a bounded copy wait of k_tbp ran out)
    int sms = 0;                  // SMs of the device: CTAs of the pipelined persistent form
    int test_cta = -1;            // tests only: this CTA of the pipelined forms arms its first
                                  // record copy for bytes that never arrive
};

int tb_threads();
bool tb_fits(int max_tri_loc, int max_edge_loc, int threads);
// The fused triangle-centric kernel (kernels_tbf.cu, vacuum media): whether tiles of these
// sizes fit it, its coefficient fill, and one launch of k steps (buffer cur to cur ^ 1).
bool tbf_fits(int max_tri_loc, int max_edge_loc, int max_src);
cudaError_t launch_tbf_fill(const TBDev& t, const DevMesh& m, cudaStream_t s);
cudaError_t launch_tbf(const TBDev& t, const DevMesh& m, int ksteps, int cur, int gbase, cudaStream_t s);
// A mesh that is one tile without a halo (at most 2048 triangles): n steps in one launch of one
// CTA with the whole mesh in shared memory (buffer cur to cur ^ 1).  hdr_host: the tile's
// header on the host.
bool tbf1_fits(const TBDev& t, const int* hdr_host);
cudaError_t launch_tbf1(const TBDev& t, const DevMesh& m, long long n_steps, int cur, cudaStream_t s);
// the kernel launch_tb runs for these tiles (UE_TBK_*)
int tb_kernel_used(const TBDev& t, const DevMesh& m);
// whether launch_tb runs the pipelined persistent form k_tbp for these tiles
bool tb_pipelined(int max_tri_loc, int max_edge_loc, int threads, bool plasma);
cudaError_t launch_tb_fill(const TBDev& t, const DevMesh& m, cudaStream_t s);
// k steps of the blocked kernel reading buffer `cur`, writing buffer cur ^ 1; the source uses
// g-table entries gbase .. gbase + k - 1.
cudaError_t launch_tb(const TBDev& t, const DevMesh& m, int ksteps, int cur, int gbase,
                      cudaStream_t s);

// Persistent cooperative step (kernels_persistent.cu).
int persistent_grid(int device);
cudaError_t launch_persistent(const DevMesh& m, int n_steps, unsigned* sync, int* err,
                              long long budget, int skip_cta, int grid, cudaStream_t s);

// Launchers (kernels_step.cu).
// g(t) table for the next `count` steps (no-op without a source).
cudaError_t launch_gtab(const DevMesh& m, int count, cudaStream_t s);
// One kernel of the plain step: 0 = E half-step (with current and source), 1 = B half-step;
// s_index = this step's entry in the g table.
cudaError_t launch_step_part(const DevMesh& m, int part, int s_index, cudaStream_t s);
// g table + `count` plain steps (count <= gtab_size).
cudaError_t launch_steps_plain(const DevMesh& m, int count, cudaStream_t s);

// Geometry, coefficients, power iteration and field transfer (kernels_geom.cu).
cudaError_t launch_geom_tri(const double* xy, const int32_t* tri_nodes, double* O, double* S,
                            int64_t n_t, cudaStream_t s);
cudaError_t launch_geom_edge(const double* xy, const int32_t* edge_nodes, const int32_t* edge_opp,
                             double* elen, double* d, int64_t n_ei, cudaStream_t s);
// cU = dt|e|/d on [0, n_ei), triangle records on [0, n_t) and their padding (codes on the zero
// slot, coefficient 0).  Edge padding must be zeroed by the caller.
cudaError_t launch_coeff(const DevMesh& m, const double* elen, const double* d, const double* S,
                         const int32_t* tri_code, double dt, cudaStream_t s);
// FP64 power iteration on K = -L_E L_B in the S metric; returns rho in *rho (synchronous).
// With a frame, the iterate covers the triangles and the frame cells (start vector keyed by
// n_t + frame cell), and K is the operator of the coupled system.
cudaError_t power_iteration(const int2* rl, const int4* tri, const double* elen, const double* d,
                            const double* S, const int64_t* perm_tri, int64_t n_t, int64_t n_ei,
                            int iters, uint32_t seed, double* work, double* rho, cudaStream_t s,
                            const FrameDev* frame = nullptr);
size_t power_iteration_work_doubles(int64_t n_t, int64_t n_ei, const FrameDev* frame = nullptr);
cudaError_t launch_fields_in(const DevMesh& m, const double* E_caller, const double* B_caller,
                             const double* J_caller, const int64_t* edge_caller,
                             const int64_t* perm_tri, const double* elen, cudaStream_t s);
// relen: 1/|e| per interior edge (launch_recip), E = U * (1/|e|)
cudaError_t launch_fields_out(const DevMesh& m, double* E_caller, double* B_caller,
                              double* J_caller, const int64_t* edge_caller,
                              const int64_t* perm_tri, const double* relen, cudaStream_t s);
// The same transfers in caller order, with the caller's arrays (double, or float when f32) in
// pinned host memory at their mapped device addresses, or in device memory: k_of[n_e] = stored
// interior edge of each caller edge or -1, inv[n_t] = stored triangle of each caller triangle.
// E (and J) are written on every caller edge.
cudaError_t launch_fields_in_caller(const DevMesh& m, const void* E_caller, const void* B_caller,
                                    const void* J_caller, bool f32, const int32_t* k_of, const int32_t* inv,
                                    const double* elen, int64_t n_e, cudaStream_t s);
cudaError_t launch_fields_out_caller(const DevMesh& m, void* E_caller, void* B_caller, void* J_caller, bool f32,
                                     const int32_t* k_of, const int32_t* inv, const double* relen, int64_t n_e,
                                     cudaStream_t s);
cudaError_t launch_recip(const double* elen, double* relen, int64_t n_ei, cudaStream_t s);
// Halo exchange of a partitioned mesh: B at caller triangle ids[0..n) to buf (scatter = 0) or
// from buf (scatter = 1), in the field type; inv[n_t] = stored triangle of each caller one.
// Ids outside [0, n_t) are skipped and counted in *bad (device).
cudaError_t launch_tri_exchange(const DevMesh& m, const int32_t* inv, const int32_t* ids, int64_t n, void* buf,
                                int scatter, unsigned* bad, cudaStream_t s);
cudaError_t launch_plasma_coeff(const DevMesh& m, const double* n_nodes, const int32_t* edge_nodes,
                                double nu, double dt, cudaStream_t s);
// src_c[i] = dt_grp * |e| * amp[i], dt of the source's group.
cudaError_t launch_source_coeff(const DevMesh& m, const double* amp, const double* elen,
                                cudaStream_t s);
// Learned spectral radius (kernels_mlp.cu).
int mlp_n_params();
// tri_nb[3j+q]: the triangle across edge q of triangle j, -1 on the boundary.
cudaError_t launch_features(const double* xy, const int32_t* tri_nodes, const int32_t* tri_code,
                            const int32_t* tri_nb, const double* elen, const double* d, const double* S,
                            int64_t n_t, int64_t n_ei, float* X, float* base, cudaStream_t s);
cudaError_t launch_mlp_forward(const float* P, const float* X, int64_t n, int bf16, float* z,
                               cudaStream_t s);
cudaError_t launch_mlp_backward(const float* P, const float* X, const int64_t* rows, const float* dz,
                                int64_t m, int bf16, float* work, float* grad, cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1,
                        float b2, float eps, int t, cudaStream_t s);
cudaError_t launch_seg_argmax(const float* z, const float* base, const int64_t* off, int n_seg,
                              float* best, int64_t* arg, cudaStream_t s);
cudaError_t launch_rho_loss(const float* best, const float* target, int n_seg, float* dz,
                            float* loss, cudaStream_t s);
// Fused learned-rho inference, one launch, on device-resident parameters, partials and
// counter (one set per device: callers serialise).  rho_infer_upload copies the 5,057
// parameters in.  out[0..4] (device-visible) = {log rho_hat, argmax row, max K_jj rounded
// down, max Gershgorin bound rounded up, local Rayleigh quotient rounded down}; then the last
// CTA writes seq into the 8 bytes of out[5], after a system-scope fence.
cudaError_t rho_infer_upload(const float* P_host, cudaStream_t s);
cudaError_t launch_rho_infer(const double* xy, const int32_t* tri_nodes, const int32_t* tri_code,
                             const int32_t* tri_nb, const double* elen, const double* d, const double* S,
                             int64_t n_t, int64_t n_ei, double* out, unsigned long long seq,
                             cudaStream_t s);

// Highest eigenmodes by the complex-time method with deflation, in block form
// (kernels_modes.cu).  Block width modes_block_size(n_modes) <= 32 columns; work holds
// modes_work_doubles doubles.  omega: n_modes values, descending.  B_dev: NULL or n_modes *
// n_t doubles on the device, mode i at B_dev + i*n_t in caller triangle order, S-normalised.
// *lost_rank is set (and nothing else computed) when the block stops being of full rank.
int modes_block_size(int n_modes);
size_t modes_work_doubles(int64_t n_t, int64_t n_ei, int m);
// The lowest modes (Chebyshev-filtered subspace iteration, degree-`degree` filters, at most
// `iters` of them): omega ascending; work holds modes_low_work_doubles doubles.
size_t modes_low_work_doubles(int64_t n_t, int64_t n_ei, int m);
cudaError_t modes_low_run(const int2* rl, const int4* tri, const double* elen, const double* d,
                          const double* S, const int64_t* perm, int64_t n_t, int64_t n_ei, int n_modes,
                          int iters, int degree, uint32_t seed, double* work, double* omega,
                          double* B_dev, bool* lost_rank, cudaStream_t s);
cudaError_t modes_run(const int2* rl, const int4* tri, const double* elen, const double* d,
                      const double* S, const int64_t* perm, int64_t n_t, int64_t n_ei, int n_modes,
                      int iters, uint32_t seed, double* work, double* omega, double* B_dev,
                      bool* lost_rank, cudaStream_t s);

// Jello-model relaxation with Lawson flips (kernels_relax.cu); see ue_mesh_relax.
int mesh_relax(const double* xy, int64_t nn, const int32_t* tris, int64_t nt, const double* h_nodes,
               int32_t iters, int32_t flip_every, double tau, const int32_t* anchors, int64_t n_anchors,
               const int32_t* segs, int64_t n_segs, double* xy_out, int32_t* tris_out, int64_t* n_flips,
               cudaStream_t s, std::string& err);
// Lawson flips alone, on the host; see ue_mesh_flip.
int mesh_flip(const double* xy, int64_t nn, const int32_t* tris, int64_t nt, const int32_t* segs,
              int64_t n_segs, int32_t* tris_out, int64_t* n_flips, std::string& err);

// Energy watchdog: W of eq. 8 into wd[1], compared with the previous check (see kernels_geom.cu).
size_t energy_parts(int64_t n_ei, int64_t n_t);
cudaError_t launch_energy(const DevMesh& m, const double* elen, const double* d, const double* S,
                          double* part, double* wd, cudaStream_t s);
// Batch assembly: dst[i] = |src[i]| (coefficients without source flags), and triangle
// records re-pointed at the batch's edge numbering.
cudaError_t launch_copy_abs(void* dst, const void* src, int64_t n, bool f64, cudaStream_t s);
cudaError_t launch_tri_offset(int4* dst, const int4* src, int64_t n, int64_t ei_off, int64_t nei_m,
                              int64_t nei_all, cudaStream_t s);
// Set (on = true) or clear the source flag (sign bit of cU) of the listed stored edges.
cudaError_t launch_source_flags(const DevMesh& m, const int32_t* k, int64_t n, bool on,
                                cudaStream_t s);
cudaError_t launch_scatter_geometry(const double* O, const double* S, const double* elen,
                                    const double* d, const int64_t* perm_tri,
                                    const int64_t* edge_caller, int64_t n_t, int64_t n_ei,
                                    int64_t n_e, double* O_c, double* S_c, double* elen_c,
                                    double* d_c, cudaStream_t s);

// PML frame (kernels_frame.cu).  Interface geometry: d_k = (O_tri - C_e) . n_in + h/2 from the
// triangles' circumcentres O (stored order), icU = dt |e| / d rounded to the field type, ic =
// |e| / d (the host checks d > 0 through ic).  iface: 6 doubles per interface edge
// {x_a, y_a, x_b, y_b, n_in x, n_in y}.
cudaError_t launch_frame_geom(const FrameDev& f, const double* O, const double* iface, double dt,
                              bool f64, cudaStream_t s);
// Fields: interface E out to / in from caller edges (iedge: caller id per interface edge,
// ielen: |e|), frame B and E out (caller layout of ue_frame_fields).
cudaError_t launch_frame_iface_out(const FrameDev& f, const DevMesh& m, const int64_t* iedge,
                                   const double* ielen, double* E_caller, cudaStream_t s);
cudaError_t launch_frame_iface_in(const FrameDev& f, const DevMesh& m, const int64_t* iedge,
                                  const double* ielen, const double* E_caller, cudaStream_t s);
cudaError_t launch_frame_out(const FrameDev& f, bool f64, double* B, double* Ex, double* Ey,
                             cudaStream_t s);
// The frame's state (Bx, By, E on its sides) out of or into FP64 arrays (device pointers).
cudaError_t launch_frame_state(const FrameDev& f, bool f64, double* Bx, double* By, double* Ex, double* Ey,
                               bool write, cudaStream_t s);

// Blocked stepping of a framed mesh: the tiles whose k-ring halo stays off the mesh's outer
// edges run in the blocked kernel; the others form one region (its owned triangles plus k rings,
// see Region in ue_internal.h) that is gathered into local arrays, advanced k steps by the plain
// kernels together with the frame, and scattered back (owned values only).  Both read the fields
// of step n and write step n + k, on disjoint owned sets.
struct RegionDev {
    DevMesh dm;                   // local arrays (FP32): rl, tri, cU, U (+ interface slots), B
    FrameDev f;                   // the frame, with local triangle ids and the region's slots
    int32_t* tgid = nullptr;      // [n_t] stored triangle per local triangle
    int32_t* egid = nullptr;      // [n_ei] stored edge per local edge
    char* upd = nullptr;          // [n_t] local triangle updated (level <= k - 1)
    int64_t n_own_t = 0, n_own_e = 0;
};
// tri.w of updated local triangles and cU of local edges from the mesh's (source flags kept).
cudaError_t launch_region_coeff(const RegionDev& r, const int4* tri, const float* cU, cudaStream_t s);
// Fields of buffer n into the region / the region's owned values into buffer n + k; J (the
// plasma current) is carried when the region has plasma.
cudaError_t launch_region_gather(const RegionDev& r, const float* B, const float* U, const float* J,
                                 cudaStream_t s);
cudaError_t launch_region_scatter(const RegionDev& r, float* B, float* U, float* J, cudaStream_t s);
// pb of the local edges from the mesh's plasma coefficients.
cudaError_t launch_region_pb(const RegionDev& r, const float* pb, cudaStream_t s);

// Power iteration with a file-scope work array (noalloc.cu).
int power_iteration_static(const int32_t* edge_tri, const double* elen, const double* d,
                           const int32_t* tri_code, const double* S, const int64_t* tri_caller,
                           int64_t n_t, int64_t n_ei, int iters, uint32_t seed, cudaStream_t s,
                           double* rho, std::string& err);

}  // namespace ue
