// C ABI of the library (include/ue.h): mesh ingest, device setup, fields, time stepping.
// Host logic only; every arithmetic step of the method runs in the kernels of
// kernels_geom.cu and kernels_step.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "device.cuh"
#include "ue_internal.h"

using ue::DevMesh;
using ue::HostMesh;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

// An NVTX range for the life of a scope (a no-op unless a profiler is attached).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

// PML frame attached by ue_frame_attach (host side; the kernels are in kernels_frame.cu).
// Interface edge k: the mesh's outer edges, bottom side first (k = 0 .. nx-1 by x), then top,
// left (by y), right.
struct FrameHost {
    int W = 0, order = 3, nx = 0, ny = 0;
    double sigma_max = 0, h = 0, X0 = 0, X1 = 0, Y0 = 0, Y1 = 0;
    std::vector<int32_t> itri;    // stored triangle, or ~t when the triangle is L of the edge
    std::vector<int32_t> icell;   // frame cell across the edge (strip order)
    std::vector<int64_t> islot;   // 3 * stored triangle + q of the triangle's code for the edge
    std::vector<int32_t> ineg;    // that code's sign bit
    std::vector<int64_t> iedge;   // caller edge id
    std::vector<double> ielen;    // |e|
    std::vector<double> iface;    // 6 per edge: x_a, y_a, x_b, y_b, inward normal
};

}  // namespace

struct ue_mesh {
    HostMesh hm;
    ue_alloc_fn alloc = nullptr;
    ue_free_fn free_fn = nullptr;
    void* alloc_ctx = nullptr;
    std::vector<void*> allocs;

    bool built = false;
    int precision = UE_PREC_FP32;
    int variant = UE_VARIANT_PLAIN;
    int graph_chunk = 32;
    double dt = 0, rho = 0;
    int rho_source = UE_RHO_GIVEN;
    int64_t steps_done = 0;
    int64_t step_pending = -1;   // ue_set_step's value, put on the device by the next call that steps
    int64_t launches = 0;

    // device tables and geometry (stored numbering)
    double* d_xy = nullptr;
    int32_t* d_tri_nodes = nullptr;
    int32_t* d_edge_nodes = nullptr;
    int32_t* d_edge_opp = nullptr;
    int32_t* d_tri_code = nullptr;
    int2* d_rl = nullptr;
    int32_t* d_tri_nb = nullptr;    // 3*n_tris: triangle across each edge, -1 on the boundary
    int64_t* d_perm = nullptr;
    int64_t* d_ecaller = nullptr;
    double *d_O = nullptr, *d_S = nullptr, *d_elen = nullptr, *d_d = nullptr;
    double* d_relen = nullptr;   // 1/|e| (the readout of E)
    // transfer buffers in caller numbering
    double *d_Ec = nullptr, *d_Bc = nullptr, *d_Jc = nullptr;
    // caller -> stored maps of the direct transfers (made on first use)
    int32_t* d_kof = nullptr;       // n_edges: stored interior edge of each caller edge, or -1
    int32_t* d_inv = nullptr;       // n_tris: stored triangle of each caller triangle
    int64_t direct_fields = 0;      // field arrays moved by the direct path
    unsigned* d_xbad = nullptr;     // bad-id counter of the halo exchange
    DevMesh dm;

    // plasma and source, kept on the host so that a rebuild can re-bake them
    std::vector<double> plasma_n;
    double plasma_nu = 0;
    std::vector<int32_t> src_k;       // stored edge ids
    std::vector<double> src_amp;
    std::vector<int32_t> src_grp;     // source group of each entry (0 for a single mesh)
    std::vector<double> grp_par;      // per group: dt, omega0, t0, tau
    bool is_batch = false;

    // captured step graph (plain: one; blocked: one per starting buffer parity)
    cudaGraphExec_t gexec = nullptr;
    int64_t graph_version = -1;
    cudaGraphExec_t gexec_tb[2] = {nullptr, nullptr};
    int64_t graph_version_tb[2] = {-1, -1};
    int64_t version = 0;
    cudaStream_t capture_stream = nullptr;

    // temporally blocked variant
    ue::TileSet ts;
    ue::TBDev tb;
    int block_depth = 4;
    int tb_threads = 512;
    int tb_kernel = UE_TB_SPLIT;
    int tb_test_cta = -1;
    int cur = 0;                     // buffer holding the current fields

    // dt selection
    double dt_setup_ms = 0, rho_lo = 0, rho_hi = 0, rho_hat = 0;

    // energy watchdog
    double* wd = nullptr;            // {W previous check, W last, growth factor, flag}
    double* wd_part = nullptr;
    int watchdog_every = 0;
    double watchdog_growth = 10.0;
    int64_t since_check = 0;

    // persistent variant: {count, gen} barrier words, error word, wait budget (cycles)
    unsigned* p_sync = nullptr;
    int* p_err = nullptr;
    long long p_budget = 0;
    int p_skip = -1;
    int p_grid = 0;

    // PML frame
    FrameHost fr;
    ue::FrameDev fd;
    // blocked stepping of a framed mesh: the region of the tiles next to the frame
    bool has_reg = false;
    ue::Region reg_host;
    ue::RegionDev reg;
    cudaStream_t side = nullptr;           // the region's stream, beside the blocked kernel
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int64_t* d_iedge = nullptr;
    double* d_ielen = nullptr;
    double* d_iface = nullptr;
};

namespace {

void* dev_alloc(ue_mesh* m, size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (m->alloc) {
        p = m->alloc(bytes, (void*)s, m->alloc_ctx);
        if (p && ((uintptr_t)p & 15u) != 0) {   // TMA bulk copies need 16-byte alignment
            if (m->free_fn) m->free_fn(p, (void*)s, m->alloc_ctx);
            p = nullptr;
        }
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) m->allocs.push_back(p);
    return p;
}

void dev_free_all(ue_mesh* m, cudaStream_t s) {
    for (void* p : m->allocs) {
        if (m->free_fn) m->free_fn(p, (void*)s, m->alloc_ctx);
        else cudaFree(p);
    }
    m->allocs.clear();
}

template <typename P>
bool alloc_into(ue_mesh* m, P*& out, size_t count, size_t elem, cudaStream_t s) {
    out = (P*)dev_alloc(m, count * elem, s);
    return out != nullptr;
}

// Release one allocation made by dev_alloc (no-op for NULL).
void dev_release(ue_mesh* m, void* p, cudaStream_t s) {
    if (!p) return;
    for (size_t i = 0; i < m->allocs.size(); ++i)
        if (m->allocs[i] == p) {
            if (m->free_fn) m->free_fn(p, (void*)s, m->alloc_ctx);
            else cudaFree(p);
            m->allocs[i] = m->allocs.back();
            m->allocs.pop_back();
            return;
        }
}

#define UE_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(UE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void drop_graph(ue_mesh* m) {
    if (m->gexec) cudaGraphExecDestroy(m->gexec);
    m->gexec = nullptr;
    m->graph_version = -1;
    for (int p = 0; p < 2; ++p) {
        if (m->gexec_tb[p]) cudaGraphExecDestroy(m->gexec_tb[p]);
        m->gexec_tb[p] = nullptr;
        m->graph_version_tb[p] = -1;
    }
}

// Point the plain-kernel view of the fields at buffer c.
void set_current(ue_mesh* m, int c) {
    m->cur = c;
    if (m->variant == UE_VARIANT_BLOCKED) {
        m->dm.B = m->tb.B[c];
        m->dm.U = m->tb.U[c];
        m->dm.J = m->tb.J[c];
    }
}

cudaError_t blocked_launch(ue_mesh* m, int kk, int cur, int gbase, cudaStream_t s);
int64_t blocked_launches(const ue_mesh* m, int kk);

int tb_chunk_launches(const ue_mesh* m) {
    const int per = m->graph_chunk / (2 * m->block_depth);
    return 2 * (per < 1 ? 1 : per);
}

int ensure_graph_tb(ue_mesh* m, int parity) {
    if (m->gexec_tb[parity] && m->graph_version_tb[parity] == m->version) return UE_OK;
    if (m->gexec_tb[parity]) cudaGraphExecDestroy(m->gexec_tb[parity]);
    m->gexec_tb[parity] = nullptr;
    if (!m->capture_stream)
        UE_CUDA(cudaStreamCreateWithFlags(&m->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    UE_CUDA(cudaStreamBeginCapture(m->capture_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = ue::launch_gtab(m->dm, tb_chunk_launches(m) * m->block_depth, m->capture_stream);
    int c = parity;
    for (int i = 0; i < tb_chunk_launches(m) && le == cudaSuccess; ++i) {
        le = blocked_launch(m, m->block_depth, c, i * m->block_depth, m->capture_stream);
        c ^= 1;
    }
    cudaError_t ce = cudaStreamEndCapture(m->capture_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(UE_ERR_CUDA, std::string("blocked step capture: ") + cudaGetErrorString(le));
    }
    if (ce != cudaSuccess) return fail(UE_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(ce));
    cudaError_t ie = cudaGraphInstantiate(&m->gexec_tb[parity], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        m->gexec_tb[parity] = nullptr;
        return fail(UE_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
    }
    m->graph_version_tb[parity] = m->version;
    return UE_OK;
}

int upload_tiles(ue_mesh* m, cudaStream_t s);
int upload_tileset(ue_mesh* m, cudaStream_t s);

// The region of a framed blocked mesh on the device (local arrays, the frame re-pointed at
// them), coefficients from the mesh's.  Sources are set by region_sources.
int setup_region(ue_mesh* m, const std::vector<char>& owned, cudaStream_t s) {
    std::string err;
    ue::Region& R = m->reg_host;
    int rc = ue::build_region(m->hm, owned, m->block_depth, m->fr.islot, m->fr.ineg, R, err);
    if (rc != UE_OK) return fail(rc, err);
    ue::RegionDev& r = m->reg;
    r = ue::RegionDev();
    DevMesh& d = r.dm;
    const int64_t ntl = (int64_t)R.tgid.size(), nel = (int64_t)R.egid.size();
    const int64_t n_if = (int64_t)m->fr.itri.size();
    d.precision = UE_PREC_FP32;
    d.n_t = ntl;
    d.n_ei = nel;
    d.n_ei_pad = (nel + 4) / 4 * 4;
    d.n_t_pad = (ntl + 3) / 4 * 4;
    d.dt = m->dt;
    d.gtab_size = m->dm.gtab_size;
    int32_t* itri = nullptr;
    int2* rlw = nullptr;
    const bool ok = alloc_into(m, rlw, d.n_ei_pad, 8, s) && alloc_into(m, d.tri, d.n_t_pad, 16, s) &&
                    alloc_into(m, d.cU, d.n_ei_pad, 4, s) &&
                    alloc_into(m, d.U, d.n_ei_pad + (n_if + 3) / 4 * 4, 4, s) &&
                    alloc_into(m, d.B, d.n_t_pad, 4, s) && alloc_into(m, r.tgid, ntl, 4, s) &&
                    alloc_into(m, r.egid, nel, 4, s) && alloc_into(m, r.upd, ntl, 1, s) &&
                    alloc_into(m, itri, n_if, 4, s) &&
                    (m->tb.n_tiles == 0 || alloc_into(m, d.step, 1, 8, s));
    if (!ok) return fail(UE_ERR_ALLOC, "frame region arrays");
    // without blocked tiles the region's step counter is the mesh's (its B half-steps advance it)
    if (m->tb.n_tiles == 0) d.step = m->dm.step;
    std::vector<int32_t> rl(2 * d.n_ei_pad, 0), tri(4 * d.n_t_pad, (int32_t)(2 * nel)), tg(ntl), eg(nel), it(n_if);
    for (int64_t l = 0; l < nel; ++l) {
        rl[2 * l] = R.rl[2 * l];
        rl[2 * l + 1] = R.rl[2 * l + 1];
        eg[l] = (int32_t)R.egid[l];
    }
    for (int64_t l = 0; l < d.n_t_pad; ++l) tri[4 * l + 3] = 0;
    for (int64_t l = 0; l < ntl; ++l) {
        for (int c = 0; c < 3; ++c) tri[4 * l + c] = R.code[3 * l + c];
        tg[l] = (int32_t)R.tgid[l];
    }
    for (int64_t i = 0; i < n_if; ++i) {
        const int32_t code = m->fr.itri[i];
        const int32_t l = R.tloc[code >= 0 ? code : ~code];
        if (l < 0 || l >= R.n_own_t) return fail(UE_ERR_ARG, "internal error: an outer edge's triangle is not in the frame region");
        it[i] = code >= 0 ? l : ~l;
    }
    UE_CUDA(cudaMemcpyAsync(rlw, rl.data(), 4 * rl.size(), cudaMemcpyHostToDevice, s));
    d.rl = rlw;
    UE_CUDA(cudaMemcpyAsync(d.tri, tri.data(), 4 * tri.size(), cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemcpyAsync(r.tgid, tg.data(), 4 * ntl, cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemcpyAsync(r.egid, eg.data(), 4 * nel, cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemcpyAsync(r.upd, R.upd.data(), ntl, cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemcpyAsync(itri, it.data(), 4 * n_if, cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemsetAsync(d.cU, 0, 4 * d.n_ei_pad, s));
    UE_CUDA(cudaMemsetAsync(d.U, 0, 4 * (d.n_ei_pad + (n_if + 3) / 4 * 4), s));
    UE_CUDA(cudaMemsetAsync(d.B, 0, 4 * d.n_t_pad, s));
    if (m->tb.n_tiles > 0) UE_CUDA(cudaMemsetAsync(d.step, 0, 8, s));
    r.f = m->fd;
    r.f.itri = itri;
    r.f.u_off = d.n_ei_pad;
    d.frame = &r.f;
    r.n_own_t = R.n_own_t;
    r.n_own_e = R.n_own_e;
    UE_CUDA(ue::launch_region_coeff(r, m->dm.tri, (const float*)m->dm.cU, s));
    UE_CUDA(cudaStreamSynchronize(s));
    if (!m->side) UE_CUDA(cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking));
    if (!m->ev_fork) UE_CUDA(cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming));
    if (!m->ev_join) UE_CUDA(cudaEventCreateWithFlags(&m->ev_join, cudaEventDisableTiming));
    m->has_reg = true;
    return UE_OK;
}

// One blocked launch of k steps (buffer cur to cur ^ 1): the blocked tiles and, for a framed
// mesh, the region's gather, k plain steps and scatter.  Both read buffer cur and write
// disjoint parts of cur ^ 1, so the region runs on a side stream forked from s before the
// blocked kernel and joined after it (inside a graph capture too): its small kernels fill the
// room the one-CTA-per-SM blocked kernel leaves on each SM.
cudaError_t blocked_launch(ue_mesh* m, int kk, int cur, int gbase, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    const bool tiles = m->tb.n_tiles > 0;
    cudaStream_t rs = s;
    if (m->has_reg && tiles) {
        e = cudaEventRecord(m->ev_fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(m->side, m->ev_fork, 0);
        rs = m->side;
    }
    if (e == cudaSuccess && m->has_reg) {
        ue::RegionDev& r = m->reg;
        e = ue::launch_region_gather(r, (const float*)m->tb.B[cur], (const float*)m->tb.U[cur],
                                     (const float*)m->tb.J[cur], rs);
        for (int i = 0; i < kk && e == cudaSuccess; ++i) {
            e = ue::launch_step_part(r.dm, 0, gbase + i, rs);
            if (e == cudaSuccess) e = ue::launch_step_part(r.dm, 1, gbase + i, rs);
        }
        if (e == cudaSuccess)
            e = ue::launch_region_scatter(r, (float*)m->tb.B[cur ^ 1], (float*)m->tb.U[cur ^ 1],
                                          (float*)m->tb.J[cur ^ 1], rs);
    }
    if (e == cudaSuccess && tiles) e = ue::launch_tb(m->tb, m->dm, kk, cur, gbase, s);
    if (e == cudaSuccess && m->has_reg && tiles) {
        e = cudaEventRecord(m->ev_join, m->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, m->ev_join, 0);
    }
    return e;
}

// Kernels of one blocked launch of kk steps.
int64_t blocked_launches(const ue_mesh* m, int kk) {
    return (m->tb.n_tiles > 0 ? 1 : 0) + (m->has_reg ? 2 + 2 * (int64_t)kk : 0);
}

int ensure_graph(ue_mesh* m) {
    if (m->gexec && m->graph_version == m->version) return UE_OK;
    drop_graph(m);
    if (!m->capture_stream)
        UE_CUDA(cudaStreamCreateWithFlags(&m->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    UE_CUDA(cudaStreamBeginCapture(m->capture_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = ue::launch_steps_plain(m->dm, m->graph_chunk, m->capture_stream);
    cudaError_t ce = cudaStreamEndCapture(m->capture_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(UE_ERR_CUDA, std::string("step capture: ") + cudaGetErrorString(le));
    }
    if (ce != cudaSuccess) return fail(UE_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(ce));
    cudaError_t ie = cudaGraphInstantiate(&m->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        m->gexec = nullptr;
        return fail(UE_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
    }
    m->graph_version = m->version;
    return UE_OK;
}

// After `steps` more steps: run the energy check whenever watchdog_every steps have passed.
// Returns the number of kernels launched.
cudaError_t watchdog_tick(ue_mesh* m, int64_t steps, cudaStream_t s, int64_t* launched) {
    if (m->watchdog_every <= 0) return cudaSuccess;
    m->since_check += steps;
    if (m->since_check < m->watchdog_every) return cudaSuccess;
    m->since_check = 0;
    *launched += 2;
    return ue::launch_energy(m->dm, m->d_elen, m->d_d, m->d_S, m->wd_part, m->wd, s);
}

// kernels launched for `steps` plain steps issued in batches of `batch` (one g-table kernel
// per batch when a source is set)
int64_t plain_launches(const ue_mesh* m, int64_t steps, int64_t batch) {
    return 2 * steps + (m->dm.n_src > 0 ? (steps + batch - 1) / batch : 0);
}

int bake_plasma(ue_mesh* m, cudaStream_t s) {
    DevMesh& dm = m->dm;
    if (m->plasma_n.empty()) {
        dm.plasma = false;
        if (m->has_reg) m->reg.dm.plasma = false;
        return UE_OK;
    }
    const size_t esz = m->precision == UE_PREC_FP64 ? 8 : 4;
    if (!dm.J && !alloc_into(m, dm.J, dm.n_ei_pad, esz, s)) return fail(UE_ERR_ALLOC, "plasma current");
    if (!dm.pb && !alloc_into(m, dm.pb, dm.n_ei_pad, esz, s)) return fail(UE_ERR_ALLOC, "plasma coefficient");
    UE_CUDA(cudaMemsetAsync(dm.pb, 0, esz * dm.n_ei_pad, s));
    double* d_n = nullptr;
    if (!alloc_into(m, d_n, m->hm.n_nodes, 8, s)) return fail(UE_ERR_ALLOC, "plasma density");
    UE_CUDA(cudaMemcpyAsync(d_n, m->plasma_n.data(), 8 * m->hm.n_nodes, cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemsetAsync(dm.J, 0, esz * dm.n_ei_pad, s));
    UE_CUDA(ue::launch_plasma_coeff(dm, d_n, m->d_edge_nodes, m->plasma_nu, m->dt, s));
    dm.pa = (1.0 - 0.5 * m->plasma_nu * m->dt) / (1.0 + 0.5 * m->plasma_nu * m->dt);
    dm.plasma = true;
    if (m->variant == UE_VARIANT_BLOCKED) {
        if (!m->tb.J[0]) {
            m->tb.J[m->cur] = dm.J;
            void* other = nullptr;
            if (!alloc_into(m, other, dm.n_ei_pad, esz, s)) return fail(UE_ERR_ALLOC, "plasma current");
            m->tb.J[m->cur ^ 1] = other;
        }
        UE_CUDA(cudaMemsetAsync(m->tb.J[0], 0, esz * dm.n_ei_pad, s));
        UE_CUDA(cudaMemsetAsync(m->tb.J[1], 0, esz * dm.n_ei_pad, s));
        if (!m->tb.epb && !alloc_into(m, m->tb.epb, m->tb.n_erec + 4, 4, s))
            return fail(UE_ERR_ALLOC, "tile plasma coefficients");
        UE_CUDA(ue::launch_tb_fill(m->tb, dm, s));
    }
    if (m->has_reg) {
        // the region of a framed blocked mesh: its own current and the mesh's coefficients
        DevMesh& d = m->reg.dm;
        if (!d.J && !alloc_into(m, d.J, d.n_ei_pad, 4, s)) return fail(UE_ERR_ALLOC, "frame region current");
        if (!d.pb && !alloc_into(m, d.pb, d.n_ei_pad, 4, s)) return fail(UE_ERR_ALLOC, "frame region coefficient");
        UE_CUDA(cudaMemsetAsync(d.J, 0, 4 * d.n_ei_pad, s));
        UE_CUDA(cudaMemsetAsync(d.pb, 0, 4 * d.n_ei_pad, s));
        UE_CUDA(ue::launch_region_pb(m->reg, (const float*)dm.pb, s));
        d.pa = dm.pa;
        d.plasma = true;
    }
    UE_CUDA(cudaStreamSynchronize(s));
    return UE_OK;
}

int bake_source_mesh(ue_mesh* m, cudaStream_t s);

// The region of a framed blocked mesh: coefficients again (the mesh's cU carries the source
// flags) and its own table {local edge, source index}; the rest of the source state is the
// mesh's.
int region_sources(ue_mesh* m, cudaStream_t s) {
    ue::RegionDev& r = m->reg;
    DevMesh& d = r.dm;
    const DevMesh& g = m->dm;
    dev_release(m, d.src_hash, s);
    d.src_hash = nullptr;
    d.n_src = 0;
    d.src_bits = 0;
    d.src_c = g.src_c;
    d.src_grp = g.src_grp;
    d.gtab = g.gtab;
    d.grp_par = g.grp_par;
    d.n_grp = g.n_grp;
    d.gtab_size = g.gtab_size;
    d.dt = g.dt;
    UE_CUDA(ue::launch_region_coeff(r, g.tri, (const float*)g.cU, s));
    std::vector<int32_t> src_of(m->hm.n_ei, -1);
    for (size_t i = 0; i < m->src_k.size(); ++i) src_of[m->src_k[i]] = (int32_t)i;
    std::vector<int32_t> lk, li;
    const std::vector<int64_t>& eg = m->reg_host.egid;
    for (size_t l = 0; l < eg.size(); ++l)
        if (src_of[eg[l]] >= 0) {
            lk.push_back((int32_t)l);
            li.push_back(src_of[eg[l]]);
        }
    if (!lk.empty()) {
        int bits = 4;
        while ((int64_t(1) << bits) < 2 * (int64_t)lk.size()) ++bits;
        const uint32_t size = 1u << bits;
        std::vector<int32_t> tab(2 * (size_t)size, -1);
        for (size_t i = 0; i < lk.size(); ++i) {
            uint32_t h = ((uint32_t)lk[i] * 2654435761u) >> (32 - bits);
            while (tab[2 * h] != -1) h = (h + 1) & (size - 1);
            tab[2 * h] = lk[i];
            tab[2 * h + 1] = li[i];
        }
        int2* dh = nullptr;
        if (!alloc_into(m, dh, size, 8, s)) return fail(UE_ERR_ALLOC, "frame region source table");
        UE_CUDA(cudaMemcpyAsync(dh, tab.data(), 8 * (size_t)size, cudaMemcpyHostToDevice, s));
        d.src_hash = dh;
        d.src_bits = bits;
        d.n_src = (int64_t)lk.size();
    }
    UE_CUDA(cudaStreamSynchronize(s));
    return UE_OK;
}

int bake_source(ue_mesh* m, cudaStream_t s) {
    int rc = bake_source_mesh(m, s);
    if (rc != UE_OK) return rc;
    if (m->variant == UE_VARIANT_BLOCKED && m->tb.erec) {
        // the tile records carry the source flags of the coefficients (the pipelined kernel
        // takes a source edge's value back after the source is added)
        UE_CUDA(ue::launch_tb_fill(m->tb, m->dm, s));
        if (m->tb.frec) UE_CUDA(ue::launch_tbf_fill(m->tb, m->dm, s));
        m->tb.max_src = m->ts.max_src;
        UE_CUDA(cudaStreamSynchronize(s));
    }
    if (!m->has_reg) return rc;
    return region_sources(m, s);
}

int bake_source_mesh(ue_mesh* m, cudaStream_t s) {
    DevMesh& dm = m->dm;
    if (dm.n_src > 0 && dm.src_k) UE_CUDA(ue::launch_source_flags(dm, dm.src_k, dm.n_src, false, s));
    UE_CUDA(cudaStreamSynchronize(s));
    for (void* p : {(void*)dm.src_k, (void*)dm.src_grp, dm.src_c, (void*)dm.src_hash,
                    (void*)dm.grp_par, (void*)dm.gtab})
        dev_release(m, p, s);
    dm.src_k = dm.src_grp = nullptr;
    dm.src_c = nullptr;
    dm.src_hash = nullptr;
    dm.grp_par = dm.gtab = nullptr;
    dm.n_src = (int64_t)m->src_k.size();
    dm.n_grp = 0;
    if (dm.n_src == 0) return UE_OK;
    if (!m->is_batch) m->grp_par[0] = m->dt;   // a rebuild may have changed dt
    dm.n_grp = (int)(m->grp_par.size() / 4);
    const size_t esz = m->precision == UE_PREC_FP64 ? 8 : 4;
    int32_t *k = nullptr, *grp = nullptr;
    double *amp = nullptr, *par = nullptr, *gt = nullptr;
    void* c = nullptr;
    if (!alloc_into(m, k, dm.n_src, 4, s) || !alloc_into(m, amp, dm.n_src, 8, s) ||
        !alloc_into(m, c, dm.n_src, esz, s) || !alloc_into(m, grp, dm.n_src, 4, s) ||
        !alloc_into(m, par, m->grp_par.size(), 8, s) ||
        !alloc_into(m, gt, (size_t)dm.gtab_size * dm.n_grp, 8, s))
        return fail(UE_ERR_ALLOC, "source arrays");
    UE_CUDA(cudaMemcpyAsync(k, m->src_k.data(), 4 * dm.n_src, cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemcpyAsync(amp, m->src_amp.data(), 8 * dm.n_src, cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemcpyAsync(grp, m->src_grp.data(), 4 * dm.n_src, cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemcpyAsync(par, m->grp_par.data(), 8 * m->grp_par.size(), cudaMemcpyHostToDevice, s));
    dm.src_k = k;
    dm.src_c = c;
    dm.src_grp = grp;
    dm.grp_par = par;
    dm.gtab = gt;
    UE_CUDA(ue::launch_source_coeff(dm, amp, m->d_elen, s));
    UE_CUDA(ue::launch_source_flags(dm, k, dm.n_src, true, s));
    // open-addressing table {stored edge id, source index}, load factor <= 1/2
    int bits = 4;
    while ((int64_t(1) << bits) < 2 * dm.n_src) ++bits;
    const uint32_t size = 1u << bits;
    std::vector<int32_t> tab(2 * (size_t)size, -1);
    for (int64_t i = 0; i < dm.n_src; ++i) {
        uint32_t h = ((uint32_t)m->src_k[i] * 2654435761u) >> (32 - bits);
        while (tab[2 * h] != -1) h = (h + 1) & (size - 1);
        tab[2 * h] = m->src_k[i];
        tab[2 * h + 1] = (int32_t)i;
    }
    int2* dh = nullptr;
    if (!alloc_into(m, dh, size, 8, s)) return fail(UE_ERR_ALLOC, "source table");
    UE_CUDA(cudaMemcpyAsync(dh, tab.data(), 8 * (size_t)size, cudaMemcpyHostToDevice, s));
    dm.src_hash = dh;
    dm.src_bits = bits;
    UE_CUDA(cudaStreamSynchronize(s));
    dev_release(m, amp, s);
    if (m->variant == UE_VARIANT_BLOCKED) {
        // per-tile source records: (local edge, source index) for every local copy of a source edge
        std::vector<int32_t> src_of(m->hm.n_ei, -1);
        for (size_t i = 0; i < m->src_k.size(); ++i) src_of[m->src_k[i]] = (int32_t)i;
        std::vector<int32_t> rec;
        ue::TileSet& ts = m->ts;
        int maxn = 0;
        for (int64_t t = 0; t < ts.n_tiles; ++t) {
            int32_t* h = &ts.hdr[t * ue::TileSet::kHdr];
            h[8] = (int32_t)(rec.size() / 2);
            const int64_t off = h[7], nel = h[5];
            for (int64_t l = 0; l < nel; ++l) {
                const int32_t src = src_of[ts.erec[4 * (off + l)]];
                if (src >= 0) {
                    rec.push_back((int32_t)l);
                    rec.push_back(src);
                }
            }
            h[9] = (int32_t)(rec.size() / 2) - h[8];
            if (h[9] > maxn) maxn = h[9];
        }
        ts.max_src = maxn;
        int2* d = nullptr;
        if (!alloc_into(m, d, rec.size() / 2 + 1, 8, s)) return fail(UE_ERR_ALLOC, "tile source records");
        if (!rec.empty()) UE_CUDA(cudaMemcpyAsync(d, rec.data(), 4 * rec.size(), cudaMemcpyHostToDevice, s));
        m->tb.tsrc = d;
        UE_CUDA(cudaMemcpyAsync(m->tb.hdr, ts.hdr.data(), 4 * ts.hdr.size(), cudaMemcpyHostToDevice, s));
    }
    UE_CUDA(cudaStreamSynchronize(s));
    return UE_OK;
}

int upload_tileset(ue_mesh* m, cudaStream_t s);

// Framed blocked stepping: a tile whose rings H_0 .. H_{k-1} reach a triangle on the mesh's
// outer edges joins the region (owned[j] for its triangles); the others stay blocked tiles.
void region_plan(const ue_mesh* m, int k, std::vector<char>& interior, std::vector<char>& owned) {
    const HostMesh& h = m->hm;
    const int64_t ntiles = (int64_t)h.tile_tri_off.size() - 1;
    std::vector<int32_t> dist(h.n_tris, -1);
    std::vector<int64_t> front, next;
    for (int32_t code : m->fr.itri) {
        const int64_t t = code >= 0 ? code : ~code;
        if (dist[t] < 0) {
            dist[t] = 0;
            front.push_back(t);
        }
    }
    for (int r = 1; r <= k - 1; ++r) {
        next.clear();
        for (int64_t j : front)
            for (int q = 0; q < 3; ++q) {
                const int64_t e = h.tri_code[3 * j + q] >> 1;
                if (e >= h.n_ei) continue;
                const int64_t o = h.edge_tri[2 * e] == j ? h.edge_tri[2 * e + 1] : h.edge_tri[2 * e];
                if (dist[o] < 0) {
                    dist[o] = r;
                    next.push_back(o);
                }
            }
        front.swap(next);
    }
    interior.assign(ntiles, 1);
    owned.assign(h.n_tris, 0);
    for (int64_t t = 0; t < ntiles; ++t)
        for (int64_t j = h.tile_tri_off[t]; j < h.tile_tri_off[t + 1]; ++j)
            if (dist[j] >= 0) {
                interior[t] = 0;
                break;
            }
    for (int64_t t = 0; t < ntiles; ++t)
        if (!interior[t])
            for (int64_t j = h.tile_tri_off[t]; j < h.tile_tri_off[t + 1]; ++j) owned[j] = 1;
}

// The fused kernel's records of a built tile set: for UE_TB_FUSED, and for a mesh that is one
// tile without a halo (run in one CTA); none when the tiles do not fit them.
void fused_records(ue::TileSet& ts, const HostMesh& hm, int threads, int kernel) {
    std::string err;
    const bool whole = ts.n_tiles == 1 && ts.hdr[4] == ts.hdr[1];
    ts.frec.clear();
    ts.fedge.clear();
    if (threads == 1024 || (kernel != UE_TB_FUSED && !whole) || ue::build_fused_records(hm, ts, err) != UE_OK) {
        ts.frec.clear();
        ts.fedge.clear();
    }
}

int upload_tiles(ue_mesh* m, cudaStream_t s) {
    std::string err;
    if (m->fr.W == 0) {
        int rc = ue::build_tiles(m->hm, m->block_depth, m->ts, err);
        if (rc != UE_OK) return fail(rc, err);
        fused_records(m->ts, m->hm, m->tb_threads, m->tb_kernel);
        return upload_tileset(m, s);
    }
    std::vector<char> interior, owned;
    region_plan(m, m->block_depth, interior, owned);
    const HostMesh& h = m->hm;
    const int k = m->block_depth;
    int rc = ue::build_tiles(h, k, m->ts, err, &interior);
    if (rc != UE_OK) return fail(rc, err);
    fused_records(m->ts, h, m->tb_threads, m->tb_kernel);
    if ((rc = upload_tileset(m, s)) != UE_OK) return rc;
    return setup_region(m, owned, s);
}

// Device copy of m->ts, second field buffers, and the coefficient slots of the records.
// Every index the blocked kernels follow, checked on the host before the records reach the
// device: headers (counts ordered by ring level and inside the record arrays), global ids of
// the records inside the field arrays, local triangle slots of the edge records and local edge
// codes of the triangle records inside the tile (the zero slot nel included), and for the fused
// records their neighbour offsets and edge ids.  A violation is an internal error of the tile
// builder, reported instead of launched.
bool tiles_in_range(const ue::TileSet& ts, int64_t n_t, int64_t n_ei, std::string& why) {
    const int64_t n_trec = (int64_t)ts.trec.size() / 4, n_erec = (int64_t)ts.erec.size() / 4;
    const int64_t n_frec = (int64_t)ts.frec.size() / 5, n_fedge = (int64_t)ts.fedge.size() / 2;
    for (int64_t t = 0; t < ts.n_tiles; ++t) {
        const int32_t* h = &ts.hdr[t * ue::TileSet::kHdr];
        const int ntl = h[4], nel = h[5], k = h[10];
        auto bad = [&](const char* what) {
            why = "tile " + std::to_string(t) + ": " + what;
            return false;
        };
        if (ntl < 0 || nel < 0 || h[1] < 0 || h[1] > ntl || h[3] < 0 || h[3] > nel || k < 1 || k > 15)
            return bad("counts");
        if (h[0] < 0 || (int64_t)h[0] + h[1] > n_t || h[2] < 0 || (int64_t)h[2] + h[3] > n_ei)
            return bad("owned ranges");
        if (h[6] < 0 || (int64_t)h[6] + ntl > n_trec || h[7] < 0 || (int64_t)h[7] + nel > n_erec)
            return bad("record offsets");
        for (int r = 0; r < 16; ++r) {
            if (h[16 + r] < (r ? h[15 + r] : 0) || h[16 + r] > ntl) return bad("triangle levels");
            if (h[32 + r] < (r ? h[31 + r] : 0) || h[32 + r] > nel) return bad("edge levels");
        }
        const int32_t* tr = &ts.trec[4 * (size_t)h[6]];
        const int nupd = h[16 + k - 1];
        for (int l = 0; l < ntl; ++l) {
            if (tr[4 * l] < 0 || tr[4 * l] >= n_t) return bad("triangle id");
            if (l >= nupd) continue;
            const uint32_t c[3] = {(uint32_t)tr[4 * l + 1] & 0xFFFFu, (uint32_t)tr[4 * l + 1] >> 16,
                                   (uint32_t)tr[4 * l + 2]};
            for (int q = 0; q < 3; ++q)
                if ((int64_t)(c[q] >> 1) > nel) return bad("triangle edge code");
        }
        const int32_t* er = &ts.erec[4 * (size_t)h[7]];
        for (int l = 0; l < nel; ++l) {
            const uint32_t w = (uint32_t)er[4 * l + 1];
            if (er[4 * l] < 0 || er[4 * l] >= n_ei) return bad("edge id");
            if ((int)(w & 0xFFFFu) >= ntl || (int)(w >> 16) >= ntl) return bad("edge triangle slot");
        }
        if (!ts.frec.empty()) {
            if (h[11] < 0 || (int64_t)h[11] + ntl > n_frec || h[12] < 0 || (int64_t)h[12] + nel + 1 > n_fedge)
                return bad("fused record offsets");
            const int32_t* fr = &ts.frec[5 * (size_t)h[11]];
            for (int l = 0; l < nupd; ++l) {
                const uint32_t r1 = (uint32_t)fr[5 * l + 1], r2 = (uint32_t)fr[5 * l + 2], r3 = (uint32_t)fr[5 * l + 3];
                const uint32_t nb[3] = {(r1 & 0xFFFFu) / 4, (r1 >> 16) / 4, (r2 & 0x3FFFu) / 4};
                const uint32_t e[3] = {(r2 >> 14) & 0x1FFFu, r3 & 0x1FFFu, (r3 >> 16) & 0x1FFFu};
                for (int q = 0; q < 3; ++q)
                    if ((int)nb[q] >= ntl || (int)e[q] > nel) return bad("fused record");
            }
        }
    }
    return true;
}

int upload_tileset(ue_mesh* m, cudaStream_t s) {
    ue::TileSet& ts = m->ts;
    {
        std::string why;
        if (!tiles_in_range(ts, m->hm.n_tris, m->hm.n_ei, why))
            return fail(UE_ERR_ARG, "internal error: a tile record is out of range (" + why + ")");
    }
    if (!ue::tb_fits(ts.max_tri_loc, ts.max_edge_loc, m->tb_threads))
        return fail(UE_ERR_ARG, "tiles with halo too large for the blocked kernel (" +
                                    std::to_string(ts.max_tri_loc) + " triangles, " +
                                    std::to_string(ts.max_edge_loc) + " edges): lower tile_tris or block_depth");
    ue::TBDev& tb = m->tb;
    tb = ue::TBDev();
    tb.n_tiles = ts.n_tiles;
    tb.n_trec = (int64_t)ts.trec.size() / 4;
    tb.n_erec = (int64_t)ts.erec.size() / 4;
    tb.max_tri_loc = ts.max_tri_loc;
    tb.max_edge_loc = ts.max_edge_loc;
    tb.threads = m->tb_threads;
    // edge records go to the device as 3 ints {gid, R | L << 16, cU}: the coefficient is filled
    // by launch_tb_fill, the plasma coefficient kept apart (tb.epb)
    std::vector<int32_t> e3(3 * (size_t)tb.n_erec);
    for (int64_t i = 0; i < tb.n_erec; ++i) {
        e3[3 * i] = ts.erec[4 * i];
        e3[3 * i + 1] = ts.erec[4 * i + 1];
        e3[3 * i + 2] = 0;
    }
    bool ok = alloc_into(m, tb.hdr, ts.hdr.size(), 4, s) && alloc_into(m, tb.trec, tb.n_trec + 1, 16, s) &&
              alloc_into(m, tb.erec, 3 * (tb.n_erec + 4), 4, s) && alloc_into(m, tb.done, 2, 4, s) &&
              alloc_into(m, tb.B[1], m->dm.n_t_pad, 4, s) && alloc_into(m, tb.U[1], m->dm.n_ei_pad, 4, s);
    if (!ok) return fail(UE_ERR_ALLOC, "tile arrays");
    tb.B[0] = m->dm.B;
    tb.U[0] = m->dm.U;
    UE_CUDA(cudaMemcpyAsync(tb.hdr, ts.hdr.data(), 4 * ts.hdr.size(), cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemcpyAsync(tb.trec, ts.trec.data(), 4 * ts.trec.size(), cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemcpyAsync(tb.erec, e3.data(), 4 * e3.size(), cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaStreamSynchronize(s));   // e3 is a host temporary
    UE_CUDA(cudaMemsetAsync(tb.done, 0, 8, s));
    {
        int dev = 0;
        UE_CUDA(cudaGetDevice(&dev));
        UE_CUDA(cudaDeviceGetAttribute(&tb.sms, cudaDevAttrMultiProcessorCount, dev));
    }
    UE_CUDA(cudaMemsetAsync(tb.B[1], 0, 4 * m->dm.n_t_pad, s));
    UE_CUDA(cudaMemsetAsync(tb.U[1], 0, 4 * m->dm.n_ei_pad, s));
    UE_CUDA(ue::launch_tb_fill(tb, m->dm, s));
    // records of the fused kernel (vacuum media, 512 threads), when the tiles fit it
    if (m->tb_threads != 1024 && !ts.frec.empty()) {
        tb.n_frec = (int64_t)ts.frec.size() / 5;
        tb.n_fedge = (int64_t)ts.fedge.size() / 2;
        if (!alloc_into(m, tb.frec, ts.frec.size(), 4, s) || !alloc_into(m, tb.fedge, ts.fedge.size(), 4, s))
            return fail(UE_ERR_ALLOC, "fused tile records");
        UE_CUDA(cudaMemcpyAsync(tb.frec, ts.frec.data(), 4 * ts.frec.size(), cudaMemcpyHostToDevice, s));
        UE_CUDA(cudaMemcpyAsync(tb.fedge, ts.fedge.data(), 4 * ts.fedge.size(), cudaMemcpyHostToDevice, s));
        UE_CUDA(ue::launch_tbf_fill(tb, m->dm, s));
        UE_CUDA(cudaStreamSynchronize(s));
    }
    tb.max_src = ts.max_src;
    tb.test_cta = m->tb_test_cta;
    return UE_OK;
}

// The triangle-neighbour table (from the R/L table) on the device, made on first use: the
// learned-rho kernels walk triangle neighbourhoods with it.
int ensure_tri_nb(ue_mesh* m, cudaStream_t s) {
    if (m->d_tri_nb) return UE_OK;
    const HostMesh& h = m->hm;
    std::vector<int32_t> nb(3 * (size_t)h.n_tris);
    for (int64_t j = 0; j < h.n_tris; ++j)
        for (int q = 0; q < 3; ++q) {
            const int64_t k = h.tri_code[3 * j + q] >> 1;
            nb[3 * j + q] = k < h.n_ei ? (h.edge_tri[2 * k] == j ? h.edge_tri[2 * k + 1] : h.edge_tri[2 * k]) : -1;
        }
    if (!alloc_into(m, m->d_tri_nb, 3 * h.n_tris, 4, s)) return fail(UE_ERR_ALLOC, "triangle neighbour table");
    UE_CUDA(cudaMemcpyAsync(m->d_tri_nb, nb.data(), 12 * h.n_tris, cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaStreamSynchronize(s));
    return UE_OK;
}

// Learned-rho resources of one device: a host-mapped pinned result buffer (the kernel writes
// its five results straight into host memory) and a host mirror of the parameters resident on
// the device, so that a call with unchanged parameters uploads nothing.  Created once per
// process and device, on first use, before dt_setup_ms starts; calls serialise on the mutex
// (the device-side partials and counter are shared).
struct LearnedRes {
    double* h_out = nullptr;
    double* d_out = nullptr;
    unsigned long long seq = 0;
    std::vector<float> params;
};
constexpr int kMaxDevices = 64;
std::mutex g_learned_mu;
LearnedRes g_learned[kMaxDevices];

LearnedRes* learned_res() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    LearnedRes& r = g_learned[dev];
    if (!r.h_out) {
        void* h = nullptr;
        if (cudaHostAlloc(&h, 8 * sizeof(double), cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        void* dp = nullptr;
        if (cudaHostGetDevicePointer(&dp, h, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeHost(h);
            return nullptr;
        }
        std::memset(h, 0, 8 * sizeof(double));
        r.h_out = (double*)h;
        r.d_out = (double*)dp;
    }
    return &r;
}

// Learned rho: one fused launch (features -> BF16 MLP -> max of z + base, max K_jj, max
// Gershgorin bound, then the local Rayleigh quotient near the argmax triangle), synchronous.
// Sets m->rho_hat, m->rho_lo, m->rho_hi.  Caller holds g_learned_mu.
int learned_rho(ue_mesh* m, const ue_options& o, LearnedRes* r, cudaStream_t s) {
    const size_t np = (size_t)ue::mlp_n_params();
    if (r->params.size() != np || std::memcmp(r->params.data(), o.mlp_params, sizeof(float) * np) != 0) {
        UE_CUDA(ue::rho_infer_upload(o.mlp_params, s));
        r->params.assign(o.mlp_params, o.mlp_params + np);
    }
    const unsigned long long seq = ++r->seq;
    UE_CUDA(ue::launch_rho_infer(m->d_xy, m->d_tri_nodes, m->d_tri_code, m->d_tri_nb, m->d_elen,
                                 m->d_d, m->d_S, m->hm.n_tris, m->hm.n_ei, r->d_out, seq, s));
    // The kernel's last write is seq into the mapped buffer: spin on it (up to 2 s, then let
    // the stream report), which returns sooner than a stream synchronisation.
    const volatile unsigned long long* flag = reinterpret_cast<const volatile unsigned long long*>(r->h_out + 5);
    const auto t_spin = std::chrono::steady_clock::now();
    bool seen = false;
    for (unsigned it = 1;; ++it) {
        if (*flag == seq) {
            seen = true;
            break;
        }
        if ((it & 1023u) == 0 && std::chrono::steady_clock::now() - t_spin > std::chrono::seconds(2)) break;
    }
    if (!seen) {
        UE_CUDA(cudaStreamSynchronize(s));
        if (*flag != seq) return fail(UE_ERR_CUDA, "learned dt: inference finished without its result");
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    const volatile double* rh = r->h_out;
    m->rho_hat = std::exp(rh[0]);
    m->rho_lo = std::sqrt(std::max(rh[2], rh[4]));
    m->rho_hi = std::sqrt(rh[3]);
    return UE_OK;
}

// Allocate the device arrays of a mesh (variant, precision, graph_chunk and block_depth set)
// and upload its connectivity tables.  Coefficients are zeroed.
int alloc_and_upload(ue_mesh* m, cudaStream_t s) {
    const HostMesh& h = m->hm;
    const size_t esz = m->precision == UE_PREC_FP64 ? 8 : 4;
    const int64_t nt = h.n_tris, nei = h.n_ei, nn = h.n_nodes, ne = h.n_edges;
    bool ok = alloc_into(m, m->d_xy, 2 * nn, 8, s) && alloc_into(m, m->d_tri_nodes, 3 * nt, 4, s) &&
              alloc_into(m, m->d_edge_nodes, 2 * nei + 2, 4, s) &&
              alloc_into(m, m->d_edge_opp, 2 * nei + 2, 4, s) &&
              alloc_into(m, m->d_tri_code, 3 * nt, 4, s) &&
              alloc_into(m, m->d_rl, (nei + 4) / 4 * 4, 8, s) &&
              alloc_into(m, m->d_perm, nt, 8, s) && alloc_into(m, m->d_ecaller, nei + 1, 8, s) &&
              alloc_into(m, m->d_O, 2 * nt, 8, s) && alloc_into(m, m->d_S, nt, 8, s) &&
              alloc_into(m, m->d_elen, nei + 1, 8, s) && alloc_into(m, m->d_d, nei + 1, 8, s) &&
              alloc_into(m, m->d_relen, nei + 1, 8, s) &&
              alloc_into(m, m->d_Ec, ne, 8, s) && alloc_into(m, m->d_Bc, nt, 8, s) &&
              alloc_into(m, m->d_Jc, ne, 8, s);
    DevMesh& dm = m->dm;
    dm.precision = m->precision;
    dm.n_t = nt;
    dm.n_ei = nei;
    dm.n_nodes = nn;
    dm.n_ei_pad = (nei + 4) / 4 * 4;
    dm.n_t_pad = (nt + 3) / 4 * 4;
    // a frame's interface edges keep their circulation after the zero slot
    const int64_t n_if = m->fr.W > 0 ? (int64_t)m->fr.itri.size() : 0;
    ok = ok && alloc_into(m, dm.tri, dm.n_t_pad, 16, s) && alloc_into(m, dm.cU, dm.n_ei_pad, esz, s) &&
         alloc_into(m, dm.U, dm.n_ei_pad + (n_if + 3) / 4 * 4, esz, s) &&
         alloc_into(m, dm.B, dm.n_t_pad, esz, s) && alloc_into(m, dm.step, 1, 8, s);
    if (ok && m->precision == UE_PREC_FP64) ok = alloc_into(m, dm.cB, dm.n_t_pad, 8, s);
    {
        int g = 64;
        if (m->graph_chunk > g) g = m->graph_chunk;
        if (m->variant == UE_VARIANT_BLOCKED && tb_chunk_launches(m) * m->block_depth > g)
            g = tb_chunk_launches(m) * m->block_depth;
        dm.gtab_size = g;
    }
    ok = ok && alloc_into(m, m->wd, 4, 8, s) &&
         alloc_into(m, m->wd_part, ue::energy_parts(nei, nt), 8, s);
    if (!ok) {
        dev_free_all(m, s);
        m->d_tri_nb = nullptr;
        m->d_kof = m->d_inv = nullptr;
        return fail(UE_ERR_ALLOC, "device allocation failed");
    }
    {
        const double w0[4] = {0.0, 0.0, m->watchdog_growth, 0.0};
        UE_CUDA(cudaMemcpyAsync(m->wd, w0, sizeof(w0), cudaMemcpyHostToDevice, s));
        UE_CUDA(cudaStreamSynchronize(s));
        m->since_check = 0;
    }
    dm.rl = m->d_rl;
    UE_CUDA(cudaMemsetAsync(m->d_rl, 0, 8 * dm.n_ei_pad, s));
    UE_CUDA(cudaMemsetAsync(dm.cU, 0, esz * dm.n_ei_pad, s));
    UE_CUDA(cudaMemcpyAsync(m->d_xy, h.xy.data(), 16 * nn, cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemcpyAsync(m->d_tri_nodes, h.tri_nodes.data(), 12 * nt, cudaMemcpyHostToDevice, s));
    if (n_if > 0) {
        // the triangles' codes of the outer edges point at the interface slots
        std::vector<int32_t> code(h.tri_code);
        for (int64_t k = 0; k < n_if; ++k)
            code[m->fr.islot[k]] = (int32_t)(2 * (dm.n_ei_pad + k) + m->fr.ineg[k]);
        UE_CUDA(cudaMemcpyAsync(m->d_tri_code, code.data(), 12 * nt, cudaMemcpyHostToDevice, s));
        UE_CUDA(cudaStreamSynchronize(s));
    } else {
        UE_CUDA(cudaMemcpyAsync(m->d_tri_code, h.tri_code.data(), 12 * nt, cudaMemcpyHostToDevice, s));
    }
    UE_CUDA(cudaMemcpyAsync(m->d_perm, h.perm_tri.data(), 8 * nt, cudaMemcpyHostToDevice, s));
    if (nei > 0) {
        UE_CUDA(cudaMemcpyAsync(m->d_edge_nodes, h.edge_nodes.data(), 8 * nei, cudaMemcpyHostToDevice, s));
        UE_CUDA(cudaMemcpyAsync(m->d_edge_opp, h.edge_opp.data(), 8 * nei, cudaMemcpyHostToDevice, s));
        UE_CUDA(cudaMemcpyAsync(m->d_rl, h.edge_tri.data(), 8 * nei, cudaMemcpyHostToDevice, s));
        UE_CUDA(cudaMemcpyAsync(m->d_ecaller, h.edge_caller.data(), 8 * nei, cudaMemcpyHostToDevice, s));
    }
    return UE_OK;
}


// The caller's array as a device address when it lies in pinned (page-locked, mapped) host
// memory and is 8-byte aligned; NULL otherwise (the transfer is then staged through a copy).
// The caller's array as a device address when it lies in pinned (page-locked, mapped) host
// memory and is aligned to its element size; NULL otherwise (the transfer is then staged).
const void* mapped_view(const void* p, size_t elem) {
    if (!p || (reinterpret_cast<uintptr_t>(p) & (elem - 1))) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // not a CUDA-known pointer: clear the error
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return a.devicePointer;
}

// Caller -> stored maps of the direct transfers (made by ue_geometry_build).
int ensure_caller_maps(ue_mesh* m, cudaStream_t s) {
    if (m->d_kof) return UE_OK;
    const HostMesh& h = m->hm;
    std::vector<int32_t> kof(h.n_edges), inv(h.n_tris);
    for (int64_t c = 0; c < h.n_edges; ++c) kof[c] = (int32_t)h.k_of_edge[c];
    for (int64_t j = 0; j < h.n_tris; ++j) inv[h.perm_tri[j]] = (int32_t)j;
    int32_t *a = nullptr, *b = nullptr;
    if (!alloc_into(m, a, h.n_edges, 4, s) || !alloc_into(m, b, h.n_tris, 4, s))
        return fail(UE_ERR_ALLOC, "caller maps of the direct field transfer");
    UE_CUDA(cudaMemcpyAsync(a, kof.data(), 4 * kof.size(), cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemcpyAsync(b, inv.data(), 4 * inv.size(), cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaStreamSynchronize(s));
    m->d_kof = a;
    m->d_inv = b;
    return UE_OK;
}

// Which of the given arrays go the direct way: all of them when each is pinned host memory and
// the mesh has no PML frame (whose interface edges travel through the staging buffer).
bool direct_transfer(const ue_mesh* m, const void* E, const void* B, const void* j, size_t elem,
                     const void*& dE, const void*& dB, const void*& dj) {
    dE = mapped_view(E, elem);
    dB = mapped_view(B, elem);
    dj = mapped_view(j, elem);
    if (m->dm.frame || m->fr.W > 0) return false;
    return (!E || dE) && (!B || dB) && (!j || dj) && (E || B || j);
}

// The watchdog words (energy, reference, growth limit, flag) and the error words reset in one
// launch: values travel as kernel arguments, so no host buffer outlives the call.
__global__ void k_rearm(double* wd, double growth, int* p_err, unsigned* tb_err) {
    if (threadIdx.x != 0) return;
    wd[0] = 0.0;
    wd[1] = 0.0;
    wd[2] = growth;
    wd[3] = 0.0;
    if (p_err) *p_err = 0;
    if (tb_err) *tb_err = 0u;
}

__global__ void k_put_step(long long* step, long long v) {
    if (threadIdx.x == 0) *step = v;
}

// Re-arm the watchdog and the error words after new fields are written.
int rearm(ue_mesh* m, cudaStream_t s) {
    m->since_check = 0;
    unsigned* tb_err = (m->variant == UE_VARIANT_BLOCKED && m->tb.done) ? m->tb.done + 1 : nullptr;
    k_rearm<<<1, 32, 0, s>>>(m->wd, m->watchdog_growth, m->p_err, tb_err);
    UE_CUDA(cudaGetLastError());
    return UE_OK;
}

// A step counter set by ue_set_step reaches the device in the stream of the next call that
// steps, ordered before its kernels.
int flush_step(ue_mesh* m, cudaStream_t s) {
    if (m->step_pending < 0) return UE_OK;
    k_put_step<<<1, 32, 0, s>>>(m->dm.step, (long long)m->step_pending);
    UE_CUDA(cudaGetLastError());
    m->step_pending = -1;
    return UE_OK;
}

// Fields in the caller's numbering as float (the product's precision), for meshes without a
// PML frame: in place when the arrays are pinned host memory, else through a device copy.
// wd: where a read also copies the watchdog words, in the same stream before its one wait
int fields_f32(ue_mesh* m, float* E, float* B, float* j, bool write, cudaStream_t s, double* wd = nullptr) {
    if (!m || !m->built) return fail(UE_ERR_ARG, "geometry not built");
    if (m->dm.frame || m->fr.W > 0)
        return fail(UE_ERR_ARG, "a mesh with a PML frame exchanges its fields through ue_write_fields / ue_read_fields");
    const HostMesh& h = m->hm;
    if (!m->dm.J && j) {
        if (!write) std::memset(j, 0, 4 * (size_t)h.n_edges);   // no current in this medium
        j = nullptr;
    }
    const void *dE = nullptr, *dB = nullptr, *dj = nullptr;
    const bool direct = direct_transfer(m, E, B, j, 4, dE, dB, dj);
    if (!direct) {
        // device copies in the staging buffers (float views of the double ones)
        dE = E ? m->d_Ec : nullptr;
        dB = B ? m->d_Bc : nullptr;
        dj = j ? m->d_Jc : nullptr;
        if (write) {
            if (E) UE_CUDA(cudaMemcpyAsync(m->d_Ec, E, 4 * h.n_edges, cudaMemcpyHostToDevice, s));
            if (B) UE_CUDA(cudaMemcpyAsync(m->d_Bc, B, 4 * h.n_tris, cudaMemcpyHostToDevice, s));
            if (j) UE_CUDA(cudaMemcpyAsync(m->d_Jc, j, 4 * h.n_edges, cudaMemcpyHostToDevice, s));
        }
    } else {
        m->direct_fields += (E ? 1 : 0) + (B ? 1 : 0) + (j ? 1 : 0);
    }
    if (write) {
        UE_CUDA(ue::launch_fields_in_caller(m->dm, dE, dB, dj, true, m->d_kof, m->d_inv, m->d_elen, h.n_edges, s));
        const int rc = rearm(m, s);
        if (rc != UE_OK) return rc;
    } else {
        UE_CUDA(ue::launch_fields_out_caller(m->dm, const_cast<void*>(dE), const_cast<void*>(dB),
                                             const_cast<void*>(dj), true, m->d_kof, m->d_inv, m->d_relen,
                                             h.n_edges, s));
        if (!direct) {
            if (E) UE_CUDA(cudaMemcpyAsync(E, m->d_Ec, 4 * h.n_edges, cudaMemcpyDeviceToHost, s));
            if (B) UE_CUDA(cudaMemcpyAsync(B, m->d_Bc, 4 * h.n_tris, cudaMemcpyDeviceToHost, s));
            if (j) UE_CUDA(cudaMemcpyAsync(j, m->d_Jc, 4 * h.n_edges, cudaMemcpyDeviceToHost, s));
        }
        if (wd) UE_CUDA(cudaMemcpyAsync(wd, m->wd, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    UE_CUDA(cudaStreamSynchronize(s));
    return UE_OK;
}

}  // namespace

extern "C" {

void ue_options_default(ue_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->reorder = UE_REORDER_RCM;
    o->precision = UE_PREC_FP32;
    o->dt_mode = UE_DT_POWER;
    o->power_iters = 200;
    o->power_seed = 0;
    o->variant = UE_VARIANT_PLAIN;
    o->graph_chunk = 32;
    o->tile_tris = 2048;
    o->block_depth = 4;
    o->dt = 0.0;
    o->safety = 0.5;
    o->watchdog_growth = 10.0;
    o->watchdog_every = 0;
    o->mlp_params = nullptr;
    o->learned_margin = 1.05;
    o->timeout_ms = 2000;
    o->test_skip_cta = -1;
}

const char* ue_last_error(void) { return g_err.c_str(); }

int ue_mesh_load(const double* xy, int64_t n_nodes, const int32_t* tris, int64_t n_tris,
                 const ue_options* opt, ue_alloc_fn alloc, ue_free_fn free_fn, void* alloc_ctx,
                 ue_mesh** out) {
    Range nvtx_range("ue_mesh_load: ingest");
    if (!out) return fail(UE_ERR_ARG, "out is NULL");
    *out = nullptr;
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(UE_ERR_ARG, "alloc and free callbacks must both be set or both be NULL");
    ue_options d;
    ue_options_default(&d);
    const ue_options& o = opt ? *opt : d;
    if (o.reorder != UE_REORDER_NONE && o.reorder != UE_REORDER_RCM && o.reorder != UE_REORDER_KD &&
        o.reorder != UE_REORDER_GREEDY && o.reorder != UE_REORDER_GREEDY_RINGS)
        return fail(UE_ERR_ARG, "unknown reorder option");
    ue_mesh* m = new (std::nothrow) ue_mesh();
    if (!m) return fail(UE_ERR_ARG, "out of host memory");
    std::string err;
    int rc;
    try {
        rc = ue::build_host_mesh(xy, n_nodes, tris, n_tris, o.reorder, o.tile_tris, m->hm, err);
    } catch (const std::bad_alloc&) {
        rc = UE_ERR_ARG;
        err = "out of host memory";
    }
    if (rc != UE_OK) {
        delete m;
        return fail(rc, err);
    }
    m->alloc = alloc;
    m->free_fn = free_fn;
    m->alloc_ctx = alloc_ctx;
    *out = m;
    return UE_OK;
}

// Frame device arrays: layout, interface tables, zeroed fields (after alloc_and_upload).
int setup_frame(ue_mesh* m, cudaStream_t s) {
    const FrameHost& fr = m->fr;
    ue::FrameDev& f = m->fd;
    f = ue::FrameDev();
    const size_t esz = m->precision == UE_PREC_FP64 ? 8 : 4;
    f.W = fr.W;
    f.nx = fr.nx;
    f.ny = fr.ny;
    f.NX = fr.nx + 2 * fr.W;
    f.NY = fr.ny + 2 * fr.W;
    f.n_fc = 2 * (int64_t)fr.W * f.NX + 2 * (int64_t)fr.W * fr.ny;
    f.n_if = (int64_t)fr.itri.size();
    f.u_off = m->dm.n_ei_pad;
    f.h = fr.h;
    const int64_t nh = (int64_t)f.NX * (f.NY + 1), nv = (int64_t)(f.NX + 1) * f.NY;
    const int64_t ntab = 2 * (f.NY + 1) + 2 * (f.NX + 1) + 2 * f.NX + 2 * f.NY;
    const bool ok = alloc_into(m, f.H, nh, esz, s) && alloc_into(m, f.V, nv, esz, s) &&
                    alloc_into(m, f.Bx, f.n_fc, esz, s) && alloc_into(m, f.By, f.n_fc, esz, s) &&
                    alloc_into(m, f.itri, f.n_if, 4, s) && alloc_into(m, f.icell, f.n_if, 4, s) &&
                    alloc_into(m, f.icU, f.n_if, esz, s) && alloc_into(m, f.ic, f.n_if, 8, s) &&
                    alloc_into(m, f.tab, ntab, esz, s) && alloc_into(m, m->d_iedge, f.n_if, 8, s) &&
                    alloc_into(m, m->d_ielen, f.n_if, 8, s) && alloc_into(m, m->d_iface, 6 * f.n_if, 8, s);
    if (!ok) return fail(UE_ERR_ALLOC, "frame arrays");
    UE_CUDA(cudaMemcpyAsync(f.itri, fr.itri.data(), 4 * f.n_if, cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemcpyAsync(f.icell, fr.icell.data(), 4 * f.n_if, cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemcpyAsync(m->d_iedge, fr.iedge.data(), 8 * f.n_if, cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemcpyAsync(m->d_ielen, fr.ielen.data(), 8 * f.n_if, cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemcpyAsync(m->d_iface, fr.iface.data(), 48 * f.n_if, cudaMemcpyHostToDevice, s));
    UE_CUDA(cudaMemsetAsync(f.H, 0, esz * nh, s));
    UE_CUDA(cudaMemsetAsync(f.V, 0, esz * nv, s));
    UE_CUDA(cudaMemsetAsync(f.Bx, 0, esz * f.n_fc, s));
    UE_CUDA(cudaMemsetAsync(f.By, 0, esz * f.n_fc, s));
    UE_CUDA(cudaStreamSynchronize(s));
    m->dm.frame = &m->fd;
    return UE_OK;
}

// Decay tables of the frame for time step dt (FP64, rounded once to the field type):
// a = (1 - sigma dt/2)/(1 + sigma dt/2); b = dt/(1 + sigma dt/2) on sides, (dt/h^2)/(...) on
// cells; sigma(delta) = sigma_max (delta / (W h))^order at each field's position.
int frame_tables(ue_mesh* m, double dt, cudaStream_t s) {
    const FrameHost& fr = m->fr;
    const ue::FrameDev& f = m->fd;
    const double h = fr.h;
    auto sig = [&](double delta) { return fr.sigma_max * std::pow(delta / (fr.W * h), fr.order); };
    auto dx = [&](double x) { return std::max(0.0, std::max(fr.X0 - x, x - fr.X1)); };
    auto dy = [&](double y) { return std::max(0.0, std::max(fr.Y0 - y, y - fr.Y1)); };
    std::vector<double> t;
    std::vector<double> aH(f.NY + 1), bH(f.NY + 1), aV(f.NX + 1), bV(f.NX + 1), axc(f.NX), bxc(f.NX),
        ayc(f.NY), byc(f.NY);
    auto ab = [&](double sg, double b0, double& a, double& b) {
        a = (1.0 - 0.5 * sg * dt) / (1.0 + 0.5 * sg * dt);
        b = b0 / (1.0 + 0.5 * sg * dt);
    };
    for (int J = 0; J <= f.NY; ++J) ab(sig(dy(fr.Y0 + (J - fr.W) * h)), dt, aH[J], bH[J]);
    for (int I = 0; I <= f.NX; ++I) ab(sig(dx(fr.X0 + (I - fr.W) * h)), dt, aV[I], bV[I]);
    for (int I = 0; I < f.NX; ++I) ab(sig(dx(fr.X0 + (I - fr.W + 0.5) * h)), dt / (h * h), axc[I], bxc[I]);
    for (int J = 0; J < f.NY; ++J) ab(sig(dy(fr.Y0 + (J - fr.W + 0.5) * h)), dt / (h * h), ayc[J], byc[J]);
    for (auto* v : {&aH, &bH, &aV, &bV, &axc, &bxc, &ayc, &byc}) t.insert(t.end(), v->begin(), v->end());
    if (m->precision == UE_PREC_FP64) {
        UE_CUDA(cudaMemcpyAsync(f.tab, t.data(), 8 * t.size(), cudaMemcpyHostToDevice, s));
        UE_CUDA(cudaStreamSynchronize(s));
    } else {
        std::vector<float> tf(t.begin(), t.end());
        UE_CUDA(cudaMemcpyAsync(f.tab, tf.data(), 4 * tf.size(), cudaMemcpyHostToDevice, s));
        UE_CUDA(cudaStreamSynchronize(s));
    }
    UE_CUDA(ue::launch_frame_geom(f, m->d_O, m->d_iface, dt, m->precision == UE_PREC_FP64, s));
    return UE_OK;
}

int ue_geometry_build(ue_mesh* m, const ue_options* opt, void* stream) {
    Range nvtx_range("ue_geometry_build");
    if (!m) return fail(UE_ERR_ARG, "mesh is NULL");
    ue_options d;
    ue_options_default(&d);
    const ue_options& o = opt ? *opt : d;
    if (o.precision != UE_PREC_FP32 && o.precision != UE_PREC_FP64)
        return fail(UE_ERR_ARG, "unknown precision");
    if (o.dt_mode == UE_DT_GIVEN && !(o.dt > 0)) return fail(UE_ERR_ARG, "dt must be > 0");
    if (o.dt_mode != UE_DT_GIVEN && o.dt_mode != UE_DT_POWER && o.dt_mode != UE_DT_LEARNED)
        return fail(UE_ERR_ARG, "unknown dt mode");
    if (o.dt_mode != UE_DT_GIVEN && (o.power_iters < 1 || !(o.safety > 0)))
        return fail(UE_ERR_ARG, "power iteration needs iters >= 1 and safety > 0");
    if (o.dt_mode == UE_DT_LEARNED && (!o.mlp_params || !(o.learned_margin >= 1.0)))
        return fail(UE_ERR_ARG, "learned dt needs mlp_params and learned_margin >= 1");
    if (o.variant != 0 && o.variant != UE_VARIANT_PLAIN && o.variant != UE_VARIANT_BLOCKED &&
        o.variant != UE_VARIANT_PERSISTENT)
        return fail(UE_ERR_ARG, "unknown variant");
    if (o.variant == UE_VARIANT_PERSISTENT && (o.precision != UE_PREC_FP32 || o.timeout_ms < 1))
        return fail(UE_ERR_ARG, "the persistent variant is FP32 only and needs timeout_ms >= 1");
    if (o.variant == UE_VARIANT_BLOCKED) {
        if (o.precision != UE_PREC_FP32) return fail(UE_ERR_ARG, "the blocked variant is FP32 only");
        if (m->hm.tile_tri_off.size() < 2) return fail(UE_ERR_ARG, "the blocked variant needs tiles (UE_REORDER_KD, UE_REORDER_GREEDY or UE_REORDER_GREEDY_RINGS)");
        if (o.block_depth < 1 || o.block_depth > 15) return fail(UE_ERR_ARG, "block_depth must be in 1..15");
        if (o.tb_threads != 0 && o.tb_threads != 512 && o.tb_threads != 1024)
            return fail(UE_ERR_ARG, "tb_threads must be 0, 512 or 1024");
    }
    const bool framed = m->fr.W > 0;
    if (framed) {
        if (o.variant == UE_VARIANT_PERSISTENT)
            return fail(UE_ERR_ARG, "a framed mesh steps with the plain or the blocked variant");
        if (o.dt_mode == UE_DT_LEARNED)
            return fail(UE_ERR_ARG, "a framed mesh takes its dt from UE_DT_GIVEN or UE_DT_POWER");

    }
    cudaStream_t s = (cudaStream_t)stream;
    const HostMesh& h = m->hm;
    // a rebuild starts from scratch
    drop_graph(m);
    UE_CUDA(cudaStreamSynchronize(s));
    dev_free_all(m, s);
    m->d_tri_nb = nullptr;
    m->d_kof = m->d_inv = nullptr;
    m->d_xbad = nullptr;
    m->built = false;
    m->dm = DevMesh();
    m->tb = ue::TBDev();
    m->fd = ue::FrameDev();
    m->has_reg = false;
    m->reg = ue::RegionDev();
    m->reg_host = ue::Region();
    m->cur = 0;
    m->variant = o.variant == 0 ? UE_VARIANT_PLAIN : o.variant;
    m->block_depth = o.block_depth;
    m->tb_threads = o.tb_threads == 1024 ? 1024 : 512;
    if (o.tb_kernel != UE_TB_SPLIT && o.tb_kernel != UE_TB_FUSED) return fail(UE_ERR_ARG, "tb_kernel must be UE_TB_SPLIT or UE_TB_FUSED");
    m->tb_kernel = o.tb_kernel;
    m->tb_test_cta = m->variant == UE_VARIANT_BLOCKED ? o.test_skip_cta : -1;
    m->precision = o.precision;
    m->graph_chunk = o.graph_chunk == 0 ? 32 : o.graph_chunk;
    if (o.watchdog_every < 0 || !(o.watchdog_growth > 1.0))
        return fail(UE_ERR_ARG, "watchdog_every must be >= 0 and watchdog_growth > 1");
    m->watchdog_every = o.watchdog_every;
    m->watchdog_growth = o.watchdog_growth;
    int arc = alloc_and_upload(m, s);
    if (arc != UE_OK) return arc;
    if (framed && (arc = setup_frame(m, s)) != UE_OK) return arc;
    DevMesh& dm = m->dm;
    const size_t esz = m->precision == UE_PREC_FP64 ? 8 : 4;
    const int64_t nt = h.n_tris, nei = h.n_ei;
    UE_CUDA(ue::launch_geom_tri(m->d_xy, m->d_tri_nodes, m->d_O, m->d_S, nt, s));
    UE_CUDA(ue::launch_geom_edge(m->d_xy, m->d_edge_nodes, m->d_edge_opp, m->d_elen, m->d_d, nei, s));
    UE_CUDA(ue::launch_recip(m->d_elen, m->d_relen, nei, s));
    // dual lengths must be positive (eq. 3 divides by |O_R O_L|)
    {
        std::vector<double> dd(nei), ll(nei);
        if (nei > 0) {
            UE_CUDA(cudaMemcpyAsync(dd.data(), m->d_d, 8 * nei, cudaMemcpyDeviceToHost, s));
            UE_CUDA(cudaMemcpyAsync(ll.data(), m->d_elen, 8 * nei, cudaMemcpyDeviceToHost, s));
        }
        UE_CUDA(cudaStreamSynchronize(s));
        for (int64_t k = 0; k < nei; ++k)
            if (!(dd[k] > 1e-12 * ll[k])) {
                const int64_t e = h.edge_caller[k];
                return fail(UE_ERR_DUAL, "interior edge " + std::to_string(e) + " (nodes " +
                                             std::to_string(h.edges[2 * e]) + "," +
                                             std::to_string(h.edges[2 * e + 1]) +
                                             ") has dual length |O_R O_L| <= 0: mesh is not Delaunay");
            }
    }
    if (framed) {
        // the mesh's outer edges face the frame cells: their dual lengths must be positive too
        const int64_t n_if = m->fd.n_if;
        UE_CUDA(ue::launch_frame_geom(m->fd, m->d_O, m->d_iface, 0.0, m->precision == UE_PREC_FP64, s));
        std::vector<double> ic(n_if);
        UE_CUDA(cudaMemcpyAsync(ic.data(), m->fd.ic, 8 * n_if, cudaMemcpyDeviceToHost, s));
        UE_CUDA(cudaStreamSynchronize(s));
        for (int64_t k = 0; k < n_if; ++k)
            if (!(ic[k] > 0.0 && ic[k] < 1e12))
                return fail(UE_ERR_DUAL, "outer edge " + std::to_string(m->fr.iedge[k]) +
                                             " has dual length <= 0 to its frame cell");
    }
    // triangle records first with dt = 0: the power iteration reads only their edge codes
    UE_CUDA(ue::launch_coeff(dm, m->d_elen, m->d_d, m->d_S, m->d_tri_code, 0.0, s));
    // work space of the chosen dt method, allocated before dt_setup_ms starts (the power
    // iteration's again inside it when a learned prediction falls back)
    double* pwork = nullptr;
    LearnedRes* lres = nullptr;
    std::unique_lock<std::mutex> llock(g_learned_mu, std::defer_lock);
    if (o.dt_mode == UE_DT_LEARNED) {
        const int nrc = ensure_tri_nb(m, s);
        if (nrc != UE_OK) return nrc;
        llock.lock();
        if (!(lres = learned_res())) return fail(UE_ERR_ALLOC, "learned dt result buffer");
    } else if (o.dt_mode == UE_DT_POWER) {
        if (!alloc_into(m, pwork, ue::power_iteration_work_doubles(nt, nei, framed ? &m->fd : nullptr), 8, s))
            return fail(UE_ERR_ALLOC, "power iteration work space");
    }
    UE_CUDA(cudaStreamSynchronize(s));
    Range nvtx_dt("ue_geometry_build: dt, coefficients, tiles");
    const auto t_dt0 = std::chrono::steady_clock::now();
    m->rho_lo = m->rho_hi = m->rho_hat = 0;
    bool need_power = o.dt_mode == UE_DT_POWER;
    if (o.dt_mode == UE_DT_LEARNED) {
        int lrc = learned_rho(m, o, lres, s);
        llock.unlock();
        if (lrc != UE_OK) return lrc;
        // the prediction, raised to the certified lower bound, must keep the chosen dt at least
        // learned_margin below the stability limit of eq. 20 even for rho = rho_hi
        const double rt = std::max(m->rho_hat, m->rho_lo);
        const bool ok = std::isfinite(rt) && rt <= m->rho_hi &&
                        rt >= o.learned_margin * o.safety * m->rho_hi;
        if (ok) {
            m->rho = rt;
            m->rho_source = UE_RHO_LEARNED;
            m->dt = o.safety * 2.0 / m->rho;
        } else {
            need_power = true;
        }
    }
    if (need_power) {
        if (!pwork && !alloc_into(m, pwork, ue::power_iteration_work_doubles(nt, nei, framed ? &m->fd : nullptr), 8, s))
            return fail(UE_ERR_ALLOC, "power iteration work space");
        double rho = 0;
        UE_CUDA(ue::power_iteration(m->d_rl, dm.tri, m->d_elen, m->d_d, m->d_S, m->d_perm, nt, nei,
                                    o.power_iters, o.power_seed, pwork, &rho, s,
                                    framed ? &m->fd : nullptr));
        if (!(rho > 0) || !std::isfinite(rho)) return fail(UE_ERR_DUAL, "power iteration gave rho <= 0");
        m->rho = rho;
        m->rho_source = o.dt_mode == UE_DT_LEARNED ? UE_RHO_POWER_FALLBACK : UE_RHO_POWER;
        m->dt = o.safety * 2.0 / rho;
    }
    if (o.dt_mode != UE_DT_GIVEN) {
        m->dt_setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_dt0).count();
    } else {
        m->rho = 0;
        m->rho_source = UE_RHO_GIVEN;
        m->dt = o.dt;
    }
    if (pwork) dev_release(m, pwork, s);
    dm.dt = m->dt;
    UE_CUDA(ue::launch_coeff(dm, m->d_elen, m->d_d, m->d_S, m->d_tri_code, m->dt, s));
    if (framed) {
        const int frc = frame_tables(m, m->dt, s);
        if (frc != UE_OK) return frc;
    }
    UE_CUDA(cudaMemsetAsync(dm.U, 0, esz * (dm.n_ei_pad + (framed ? (m->fd.n_if + 3) / 4 * 4 : 0)), s));
    UE_CUDA(cudaMemsetAsync(dm.B, 0, esz * dm.n_t_pad, s));
    UE_CUDA(cudaMemsetAsync(dm.step, 0, 8, s));
    m->step_pending = -1;
    if (m->variant == UE_VARIANT_BLOCKED) {
        int trc = upload_tiles(m, s);
        if (trc != UE_OK) return trc;
    }
    if (m->variant == UE_VARIANT_PERSISTENT) {
        if (!alloc_into(m, m->p_sync, 2, 4, s) || !alloc_into(m, m->p_err, 1, 4, s))
            return fail(UE_ERR_ALLOC, "persistent barrier words");
        UE_CUDA(cudaMemsetAsync(m->p_sync, 0, 8, s));
        UE_CUDA(cudaMemsetAsync(m->p_err, 0, 4, s));
        int dev = 0, khz = 0;
        UE_CUDA(cudaGetDevice(&dev));
        UE_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
        m->p_budget = (long long)o.timeout_ms * (long long)khz;   // kHz * ms = cycles
        m->p_skip = o.test_skip_cta;
        m->p_grid = ue::persistent_grid(dev);
    }
    UE_CUDA(cudaStreamSynchronize(s));
    if (m->fr.W == 0) {
        // the caller -> stored maps of field transfers in place (pinned host arrays), made here
        // so that the first such transfer does not build them
        const int mrc = ensure_caller_maps(m, s);
        if (mrc != UE_OK) return mrc;
    }
    m->steps_done = 0;
    m->built = true;
    m->version++;
    int rc = bake_plasma(m, s);
    if (rc != UE_OK) return rc;
    return bake_source(m, s);
}

int ue_batch_create(ue_mesh* const* meshes, int32_t n, void* stream, ue_mesh** out) {
    if (!out || !meshes || n < 1) return fail(UE_ERR_ARG, "need at least one mesh and an output");
    *out = nullptr;
    const ue_mesh* m0 = meshes[0];
    for (int32_t i = 0; i < n; ++i) {
        const ue_mesh* m = meshes[i];
        if (!m || !m->built) return fail(UE_ERR_ARG, "mesh " + std::to_string(i) + " is not built");
        if (m->is_batch) return fail(UE_ERR_ARG, "a batch cannot contain a batch");
        if (m->precision != m0->precision || m->variant != m0->variant)
            return fail(UE_ERR_ARG, "all meshes of a batch need the same precision and variant");
        if (m->variant == UE_VARIANT_BLOCKED &&
            (m->block_depth != m0->block_depth || m->tb_threads != m0->tb_threads))
            return fail(UE_ERR_ARG, "all blocked meshes of a batch need the same block_depth and tb_threads");
        if (m->dm.plasma) return fail(UE_ERR_ARG, "batches of plasma media are not supported");
        if (m->dm.frame) return fail(UE_ERR_ARG, "batches of framed meshes are not supported");
    }
    cudaStream_t s = (cudaStream_t)stream;
    ue_mesh* B = new (std::nothrow) ue_mesh();
    if (!B) return fail(UE_ERR_ARG, "out of host memory");
    B->alloc = m0->alloc;
    B->free_fn = m0->free_fn;
    B->alloc_ctx = m0->alloc_ctx;
    B->is_batch = true;
    B->precision = m0->precision;
    B->variant = m0->variant;
    B->block_depth = m0->block_depth;
    B->tb_threads = m0->tb_threads;
    B->graph_chunk = m0->graph_chunk;
    B->watchdog_every = m0->watchdog_every;
    B->watchdog_growth = m0->watchdog_growth;
    B->dt = m0->dt;
    B->rho = 0;
    B->rho_source = m0->rho_source;
    // host tables: mesh-major concatenation
    HostMesh& H = B->hm;
    std::vector<int64_t> t_off(n + 1, 0), e_off(n + 1, 0), k_off(n + 1, 0), v_off(n + 1, 0);
    for (int32_t i = 0; i < n; ++i) {
        const HostMesh& h = meshes[i]->hm;
        t_off[i + 1] = t_off[i] + h.n_tris;
        e_off[i + 1] = e_off[i] + h.n_edges;
        k_off[i + 1] = k_off[i] + h.n_ei;
        v_off[i + 1] = v_off[i] + h.n_nodes;
    }
    H.n_tris = t_off[n];
    H.n_edges = e_off[n];
    H.n_ei = k_off[n];
    H.n_nodes = v_off[n];
    if (H.n_tris > (INT32_MAX / 4) || H.n_nodes > INT32_MAX) {
        delete B;
        return fail(UE_ERR_ARG, "batch too large for 32-bit indices");
    }
    const int64_t NEI = H.n_ei;
    for (int32_t i = 0; i < n; ++i) {
        const HostMesh& h = meshes[i]->hm;
        H.xy.insert(H.xy.end(), h.xy.begin(), h.xy.end());
        for (int64_t x : h.edges) H.edges.push_back(x + v_off[i]);
        for (int64_t x : h.perm_tri) H.perm_tri.push_back(x + t_off[i]);
        for (int64_t x : h.edge_caller) H.edge_caller.push_back(x + e_off[i]);
        for (int64_t x : h.k_of_edge) H.k_of_edge.push_back(x < 0 ? -1 : x + k_off[i]);
        for (int32_t x : h.edge_tri) H.edge_tri.push_back((int32_t)(x + t_off[i]));
        for (int32_t c : h.tri_code)
            H.tri_code.push_back((c >> 1) == h.n_ei ? (int32_t)(2 * NEI) : (int32_t)(c + 2 * k_off[i]));
        for (int32_t x : h.tri_nodes) H.tri_nodes.push_back((int32_t)(x + v_off[i]));
        for (int32_t x : h.edge_nodes) H.edge_nodes.push_back((int32_t)(x + v_off[i]));
        for (int32_t x : h.edge_opp) H.edge_opp.push_back((int32_t)(x + v_off[i]));
        if (B->variant == UE_VARIANT_BLOCKED) {
            if (H.tile_tri_off.empty()) H.tile_tri_off.push_back(0);
            for (size_t t = 1; t < h.tile_tri_off.size(); ++t)
                H.tile_tri_off.push_back(h.tile_tri_off[t] + t_off[i]);
        }
    }
    int rc = alloc_and_upload(B, s);
    if (rc != UE_OK) {
        ue_mesh_free(B);
        return rc;
    }
    DevMesh& dm = B->dm;
    const bool f64 = B->precision == UE_PREC_FP64;
    const size_t esz = f64 ? 8 : 4;
#define UE_BATCH_CUDA(call)                                                                       \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            ue_mesh_free(B);                                                                      \
            return fail(UE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
        }                                                                                         \
    } while (0)
    for (int32_t i = 0; i < n; ++i) {
        const ue_mesh* m = meshes[i];
        const int64_t nt = m->hm.n_tris, nei = m->hm.n_ei, to = t_off[i], ko = k_off[i];
        UE_BATCH_CUDA(cudaMemcpyAsync(B->d_O + 2 * to, m->d_O, 16 * nt, cudaMemcpyDeviceToDevice, s));
        UE_BATCH_CUDA(cudaMemcpyAsync(B->d_S + to, m->d_S, 8 * nt, cudaMemcpyDeviceToDevice, s));
        UE_BATCH_CUDA(cudaMemcpyAsync((char*)dm.B + esz * to, m->dm.B, esz * nt, cudaMemcpyDeviceToDevice, s));
        UE_BATCH_CUDA(ue::launch_tri_offset(dm.tri + to, m->dm.tri, nt, ko, nei, NEI, s));
        if (f64)
            UE_BATCH_CUDA(cudaMemcpyAsync((double*)dm.cB + to, m->dm.cB, 8 * nt, cudaMemcpyDeviceToDevice, s));
        if (nei > 0) {
            UE_BATCH_CUDA(cudaMemcpyAsync(B->d_elen + ko, m->d_elen, 8 * nei, cudaMemcpyDeviceToDevice, s));
            UE_BATCH_CUDA(cudaMemcpyAsync(B->d_d + ko, m->d_d, 8 * nei, cudaMemcpyDeviceToDevice, s));
            UE_BATCH_CUDA(ue::launch_copy_abs((char*)dm.cU + esz * ko, m->dm.cU, nei, f64, s));
            UE_BATCH_CUDA(cudaMemcpyAsync((char*)dm.U + esz * ko, m->dm.U, esz * nei, cudaMemcpyDeviceToDevice, s));
        }
    }
    UE_BATCH_CUDA(ue::launch_recip(B->d_elen, B->d_relen, NEI, s));   // the readout's 1/|e|
    {
        // padding records of the batch point at its zero slot with coefficient 0
        std::vector<int4> pad(dm.n_t_pad - H.n_tris);
        for (auto& r : pad) r = make_int4((int)(2 * NEI), (int)(2 * NEI), (int)(2 * NEI), 0);
        if (!pad.empty())
            UE_BATCH_CUDA(cudaMemcpyAsync(dm.tri + H.n_tris, pad.data(), 16 * pad.size(), cudaMemcpyHostToDevice, s));
        UE_BATCH_CUDA(cudaMemsetAsync((char*)dm.U + esz * NEI, 0, esz * (dm.n_ei_pad - NEI), s));
        UE_BATCH_CUDA(cudaMemsetAsync((char*)dm.B + esz * H.n_tris, 0, esz * (dm.n_t_pad - H.n_tris), s));
        UE_BATCH_CUDA(cudaMemsetAsync(dm.step, 0, 8, s));
        UE_BATCH_CUDA(cudaStreamSynchronize(s));
    }
#undef UE_BATCH_CUDA
    dm.dt = B->dt;
    if (B->variant == UE_VARIANT_BLOCKED) {
        ue::TileSet& T = B->ts;
        T = ue::TileSet();
        T.k_max = m0->ts.k_max;
        bool all_fused = true;
        for (int32_t i = 0; i < n; ++i) {
            const ue::TileSet& ts = meshes[i]->ts;
            const int64_t tr0 = (int64_t)T.trec.size() / 4, er0 = (int64_t)T.erec.size() / 4;
            for (int64_t t = 0; t < ts.n_tiles; ++t) {
                const int32_t* h = &ts.hdr[t * ue::TileSet::kHdr];
                std::vector<int32_t> hh(h, h + ue::TileSet::kHdr);
                hh[0] += (int32_t)t_off[i];
                hh[2] += (int32_t)k_off[i];
                hh[6] += (int32_t)tr0;
                hh[7] += (int32_t)er0;
                hh[8] = hh[9] = 0;
                T.hdr.insert(T.hdr.end(), hh.begin(), hh.end());
            }
            for (size_t r = 0; r < ts.trec.size(); r += 4) {
                T.trec.push_back(ts.trec[r] + (int32_t)t_off[i]);
                T.trec.push_back(ts.trec[r + 1]);
                T.trec.push_back(ts.trec[r + 2]);
                T.trec.push_back(0);
            }
            for (size_t r = 0; r < ts.erec.size(); r += 4) {
                T.erec.push_back(ts.erec[r] + (int32_t)k_off[i]);
                T.erec.push_back(ts.erec[r + 1]);
                T.erec.push_back(0);
                T.erec.push_back(0);
            }
            for (int64_t x : ts.erec_tile) T.erec_tile.push_back(x + T.n_tiles);
            if (!ts.frec.empty()) {
                const int64_t f0 = (int64_t)T.frec.size() / 5, e0 = (int64_t)T.fedge.size() / 2;
                for (int64_t t = 0; t < ts.n_tiles; ++t) {
                    int32_t* hh = &T.hdr[(T.n_tiles + t) * ue::TileSet::kHdr];
                    hh[11] += (int32_t)f0;
                    hh[12] += (int32_t)e0;
                }
                for (size_t r = 0; r < ts.frec.size(); r += 5) {
                    T.frec.push_back(ts.frec[r] + (int32_t)t_off[i]);
                    T.frec.insert(T.frec.end(), ts.frec.begin() + r + 1, ts.frec.begin() + r + 5);
                }
                for (size_t r = 0; r < ts.fedge.size(); r += 2) {
                    T.fedge.push_back(ts.fedge[r] >= 0 ? ts.fedge[r] + (int32_t)k_off[i] : -1);
                    T.fedge.push_back(0);
                }
            } else {
                all_fused = false;
            }
            T.n_tiles += ts.n_tiles;
            T.max_tri_loc = std::max(T.max_tri_loc, ts.max_tri_loc);
            T.max_edge_loc = std::max(T.max_edge_loc, ts.max_edge_loc);
        }
        if (!all_fused) {
            T.frec.clear();
            T.fedge.clear();
        }
        rc = upload_tileset(B, s);
        if (rc != UE_OK) {
            ue_mesh_free(B);
            return rc;
        }
        UE_CUDA(cudaStreamSynchronize(s));
    }
    // sources: one group per mesh that has a source
    for (int32_t i = 0; i < n; ++i) {
        const ue_mesh* m = meshes[i];
        if (m->src_k.empty()) continue;
        const int32_t g = (int32_t)(B->grp_par.size() / 4);
        B->grp_par.insert(B->grp_par.end(), {m->dt, m->grp_par[1], m->grp_par[2], m->grp_par[3]});
        for (size_t q = 0; q < m->src_k.size(); ++q) {
            B->src_k.push_back((int32_t)(m->src_k[q] + k_off[i]));
            B->src_amp.push_back(m->src_amp[q]);
            B->src_grp.push_back(g);
        }
    }
    if (B->variant == UE_VARIANT_PERSISTENT) {
        // the batch's own grid-barrier words; wait budget and grid from its first mesh
        if (!alloc_into(B, B->p_sync, 2, 4, s) || !alloc_into(B, B->p_err, 1, 4, s)) {
            ue_mesh_free(B);
            return fail(UE_ERR_ALLOC, "persistent barrier words");
        }
        if (cudaMemsetAsync(B->p_sync, 0, 8, s) != cudaSuccess || cudaMemsetAsync(B->p_err, 0, 4, s) != cudaSuccess) {
            ue_mesh_free(B);
            return fail(UE_ERR_CUDA, "persistent barrier words");
        }
        B->p_budget = m0->p_budget;
        B->p_skip = -1;
        B->p_grid = m0->p_grid;
    }
    B->built = true;
    B->steps_done = 0;
    B->version++;
    rc = bake_source(B, s);
    if (rc != UE_OK) {
        ue_mesh_free(B);
        return rc;
    }
    *out = B;
    return UE_OK;
}

int ue_get_dt(const ue_mesh* m, double* dt, double* rho, int32_t* src) {
    if (!m || !m->built) return fail(UE_ERR_ARG, "geometry not built");
    if (dt) *dt = m->dt;
    if (rho) *rho = m->rho;
    if (src) *src = m->rho_source;
    return UE_OK;
}

int ue_set_plasma(ue_mesh* m, const double* n, double nu) {
    if (!m || !m->built) return fail(UE_ERR_ARG, "geometry not built");
    if (m->is_batch) return fail(UE_ERR_ARG, "batches of plasma media are not supported");
    if (n && !(nu >= 0)) return fail(UE_ERR_ARG, "collision rate must be >= 0");
    if (n) {
        for (int64_t v = 0; v < m->hm.n_nodes; ++v)
            if (!std::isfinite(n[v]) || n[v] < 0) return fail(UE_ERR_ARG, "density must be finite and >= 0");
        m->plasma_n.assign(n, n + m->hm.n_nodes);
        m->plasma_nu = nu;
    } else {
        m->plasma_n.clear();
    }
    m->version++;
    return bake_plasma(m, nullptr);
}

int ue_set_source(ue_mesh* m, const int32_t* ids, const double* amp, int64_t n, double w0,
                  double t0, double tau) {
    if (!m || !m->built) return fail(UE_ERR_ARG, "geometry not built");
    if (m->is_batch) return fail(UE_ERR_ARG, "a batch takes its sources from its meshes");
    if (n < 0 || (n > 0 && (!ids || !amp))) return fail(UE_ERR_ARG, "bad source arrays");
    if (n > 0 && !(tau > 0)) return fail(UE_ERR_ARG, "tau must be > 0");
    std::vector<int32_t> ks(n);
    std::vector<char> used(m->hm.n_ei, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (ids[i] < 0 || ids[i] >= m->hm.n_edges) return fail(UE_ERR_ARG, "source edge id out of range");
        const int64_t k = m->hm.k_of_edge[ids[i]];
        if (k < 0) return fail(UE_ERR_ARG, "source on a boundary edge (E = 0 there)");
        if (used[k]) return fail(UE_ERR_ARG, "repeated source edge");
        if (!std::isfinite(amp[i])) return fail(UE_ERR_ARG, "non-finite source amplitude");
        used[k] = 1;
        ks[i] = (int32_t)k;
    }
    m->src_k = ks;
    m->src_amp.assign(amp, amp + n);
    m->src_grp.assign(n, 0);
    m->grp_par = {m->dt, w0, t0, tau};
    m->version++;
    return bake_source(m, nullptr);
}


int ue_write_fields(ue_mesh* m, const double* E, const double* B, const double* j, void* stream) {
    Range nvtx_range("ue_write_fields");
    if (!m || !m->built) return fail(UE_ERR_ARG, "geometry not built");
    cudaStream_t s = (cudaStream_t)stream;
    const HostMesh& h = m->hm;
    const void *dE = nullptr, *dB = nullptr, *dj = nullptr;
    if (!m->dm.J) j = nullptr;
    if (direct_transfer(m, E, B, j, 8, dE, dB, dj)) {
        // pinned host arrays: the kernels read them in place
        const int rc = ensure_caller_maps(m, s);
        if (rc != UE_OK) return rc;
        UE_CUDA(ue::launch_fields_in_caller(m->dm, dE, dB, dj, false, m->d_kof, m->d_inv, m->d_elen, h.n_edges, s));
        m->direct_fields += (E ? 1 : 0) + (B ? 1 : 0) + (j ? 1 : 0);
    } else {
        if (E) UE_CUDA(cudaMemcpyAsync(m->d_Ec, E, 8 * h.n_edges, cudaMemcpyHostToDevice, s));
        if (B) UE_CUDA(cudaMemcpyAsync(m->d_Bc, B, 8 * h.n_tris, cudaMemcpyHostToDevice, s));
        if (j) UE_CUDA(cudaMemcpyAsync(m->d_Jc, j, 8 * h.n_edges, cudaMemcpyHostToDevice, s));
        UE_CUDA(ue::launch_fields_in(m->dm, E ? m->d_Ec : nullptr, B ? m->d_Bc : nullptr,
                                     j ? m->d_Jc : nullptr, m->d_ecaller, m->d_perm, m->d_elen, s));
    }
    if (m->dm.frame) {
        const ue::FrameDev& f = m->fd;
        const size_t esz = m->precision == UE_PREC_FP64 ? 8 : 4;
        if (E && m->has_reg)
            UE_CUDA(ue::launch_frame_iface_in(m->reg.f, m->reg.dm, m->d_iedge, m->d_ielen, m->d_Ec, s));
        else if (E)
            UE_CUDA(ue::launch_frame_iface_in(f, m->dm, m->d_iedge, m->d_ielen, m->d_Ec, s));
        UE_CUDA(cudaMemsetAsync(f.H, 0, esz * f.NX * (f.NY + 1), s));
        UE_CUDA(cudaMemsetAsync(f.V, 0, esz * (f.NX + 1) * f.NY, s));
        UE_CUDA(cudaMemsetAsync(f.Bx, 0, esz * f.n_fc, s));
        UE_CUDA(cudaMemsetAsync(f.By, 0, esz * f.n_fc, s));
    }
    {
        const int rc = rearm(m, s);
        if (rc != UE_OK) return rc;
    }
    UE_CUDA(cudaStreamSynchronize(s));
    return UE_OK;
}

int ue_write_fields_f32(ue_mesh* m, const float* E, const float* B, const float* j, void* stream) {
    Range nvtx_range("ue_write_fields_f32");
    return fields_f32(m, const_cast<float*>(E), const_cast<float*>(B), const_cast<float*>(j), true,
                      (cudaStream_t)stream);
}

int ue_read_fields_f32(ue_mesh* m, float* E, float* B, float* j, void* stream) {
    Range nvtx_range("ue_read_fields_f32");
    double wd[4];
    int rc = fields_f32(m, E, B, j, false, (cudaStream_t)stream, wd);
    if (rc != UE_OK) return rc;
    if (wd[3] != 0.0)
        return fail(UE_ERR_UNSTABLE, std::string("energy watchdog: ") +
                                         (wd[3] == 1.0 ? "non-finite energy" : "energy growth beyond the limit"));
    return UE_OK;
}

int ue_exchange_tris(ue_mesh* m, const int32_t* ids, int64_t n, void* buf, int32_t scatter, void* stream) {
    if (!m || !m->built) return fail(UE_ERR_ARG, "geometry not built");
    if (n < 0 || (n > 0 && (!ids || !buf))) return fail(UE_ERR_ARG, "NULL ids or buffer, or n < 0");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_caller_maps(m, s);
    if (rc != UE_OK) return rc;
    if (!m->d_xbad && !alloc_into(m, m->d_xbad, 1, 4, s)) return fail(UE_ERR_ALLOC, "exchange counter");
    UE_CUDA(cudaMemsetAsync(m->d_xbad, 0, 4, s));
    UE_CUDA(ue::launch_tri_exchange(m->dm, m->d_inv, ids, n, buf, scatter ? 1 : 0, m->d_xbad, s));
    unsigned bad = 0;
    UE_CUDA(cudaMemcpyAsync(&bad, m->d_xbad, 4, cudaMemcpyDeviceToHost, s));
    UE_CUDA(cudaStreamSynchronize(s));
    if (bad) return fail(UE_ERR_ARG, "ue_exchange_tris: " + std::to_string(bad) + " ids outside [0, n_tris)");
    return UE_OK;
}

int ue_step_n(ue_mesh* m, int64_t n, void* stream) {
    Range nvtx_range("ue_step_n");
    if (!m || !m->built) return fail(UE_ERR_ARG, "geometry not built");
    if (n < 0) return fail(UE_ERR_ARG, "n_steps < 0");
    cudaStream_t s = (cudaStream_t)stream;
    {
        const int rc = flush_step(m, s);
        if (rc != UE_OK) return rc;
    }
    int64_t left = n;
    if (m->variant == UE_VARIANT_PERSISTENT) {
        int64_t launched = 0;
        while (left > 0) {
            const int batch = (int)(left < m->dm.gtab_size ? left : m->dm.gtab_size);
            UE_CUDA(ue::launch_gtab(m->dm, batch, s));
            UE_CUDA(cudaMemsetAsync(m->p_sync, 0, 8, s));
            UE_CUDA(ue::launch_persistent(m->dm, batch, m->p_sync, m->p_err, m->p_budget, m->p_skip,
                                          m->p_grid, s));
            launched += 1 + (m->dm.n_src > 0 ? 1 : 0);
            left -= batch;
            UE_CUDA(watchdog_tick(m, batch, s, &launched));
        }
        m->steps_done += n;
        m->launches += launched;
        return UE_OK;
    }
    if (m->variant == UE_VARIANT_BLOCKED && n > 0 && !m->dm.plasma && !m->has_reg && !m->ts.hdr.empty() &&
        ue::tbf1_fits(m->tb, m->ts.hdr.data())) {
        // the whole mesh is one tile without a halo: all n steps in one launch of one CTA
        UE_CUDA(ue::launch_tbf1(m->tb, m->dm, n, m->cur, s));
        set_current(m, m->cur ^ 1);
        int64_t launched = 1;
        UE_CUDA(watchdog_tick(m, n, s, &launched));
        m->steps_done += n;
        m->launches += launched;
        return UE_OK;
    }
    if (m->variant == UE_VARIANT_BLOCKED) {
        const int64_t k = m->block_depth;
        const int64_t chunk = (int64_t)tb_chunk_launches(m) * k;
        int64_t launched = 0;
        if (m->graph_chunk > 0 && left >= chunk) {
            int rc = ensure_graph_tb(m, m->cur);
            if (rc != UE_OK) return rc;
            while (left >= chunk) {
                UE_CUDA(cudaGraphLaunch(m->gexec_tb[m->cur], s));
                left -= chunk;
                launched += tb_chunk_launches(m) * blocked_launches(m, (int)k) + (m->dm.n_src > 0 ? 1 : 0);
                UE_CUDA(watchdog_tick(m, chunk, s, &launched));
            }
        }
        while (left > 0) {
            // a batch of launches sharing one g table
            const int64_t batch = left < chunk ? left : chunk;
            UE_CUDA(ue::launch_gtab(m->dm, (int)batch, s));
            if (m->dm.n_src > 0) ++launched;
            // ceil(batch / k) launches with step counts as even as possible (20 steps at k = 8:
            // 7 + 7 + 6, not 8 + 8 + 4): each launch pays for its halo rings only up to its own
            // depth, so even shares recompute fewer rings in total
            const int64_t nl = (batch + k - 1) / k;
            int64_t done = 0;
            for (int64_t i = 0; i < nl; ++i) {
                const int kk = (int)(batch / nl + (i < batch % nl ? 1 : 0));
                UE_CUDA(blocked_launch(m, kk, m->cur, (int)done, s));
                set_current(m, m->cur ^ 1);
                done += kk;
                launched += blocked_launches(m, kk);
            }
            left -= batch;
            UE_CUDA(watchdog_tick(m, batch, s, &launched));
        }
        m->steps_done += n;
        m->launches += launched;
        return UE_OK;
    }
    int64_t glaunched = 0;
    if (m->graph_chunk > 0 && n >= m->graph_chunk) {
        int rc = ensure_graph(m);
        if (rc != UE_OK) return rc;
        while (left >= m->graph_chunk) {
            UE_CUDA(cudaGraphLaunch(m->gexec, s));
            left -= m->graph_chunk;
            glaunched += plain_launches(m, m->graph_chunk, m->graph_chunk);
            UE_CUDA(watchdog_tick(m, m->graph_chunk, s, &glaunched));
        }
    }
    int64_t launched = 0;
    while (left > 0) {
        const int batch = (int)(left < m->dm.gtab_size ? left : m->dm.gtab_size);
        UE_CUDA(ue::launch_steps_plain(m->dm, batch, s));
        launched += plain_launches(m, batch, batch);
        left -= batch;
        UE_CUDA(watchdog_tick(m, batch, s, &launched));
    }
    m->steps_done += n;
    m->launches += launched + glaunched;
    return UE_OK;
}

int ue_step_prepare(ue_mesh* m, void* stream) {
    Range nvtx_range("ue_step_prepare");
    if (!m || !m->built) return fail(UE_ERR_ARG, "geometry not built");
    cudaStream_t s = (cudaStream_t)stream;
    if (m->graph_chunk <= 0 || m->variant == UE_VARIANT_PERSISTENT) return UE_OK;
    if (m->variant == UE_VARIANT_BLOCKED) {
        if (!m->dm.plasma && !m->has_reg && !m->ts.hdr.empty() && ue::tbf1_fits(m->tb, m->ts.hdr.data()))
            return UE_OK;   // one launch per call, no graph
        for (int p = 0; p < 2; ++p) {
            const int rc = ensure_graph_tb(m, p);
            if (rc != UE_OK) return rc;
            UE_CUDA(cudaGraphUpload(m->gexec_tb[p], s));
        }
        return UE_OK;
    }
    const int rc = ensure_graph(m);
    if (rc != UE_OK) return rc;
    UE_CUDA(cudaGraphUpload(m->gexec, s));
    return UE_OK;
}

int ue_read_fields(ue_mesh* m, double* E, double* B, double* j, void* stream) {
    Range nvtx_range("ue_read_fields");
    if (!m || !m->built) return fail(UE_ERR_ARG, "geometry not built");
    cudaStream_t s = (cudaStream_t)stream;
    const HostMesh& h = m->hm;
    const void *dE = nullptr, *dB = nullptr, *dj = nullptr;
    if (j && !m->dm.J) {
        // no current in this medium: j reads as zero
        UE_CUDA(cudaMemsetAsync(m->d_Jc, 0, 8 * h.n_edges, s));
        UE_CUDA(cudaMemcpyAsync(j, m->d_Jc, 8 * h.n_edges, cudaMemcpyDeviceToHost, s));
        j = nullptr;
    }
    if (direct_transfer(m, E, B, j, 8, dE, dB, dj)) {
        // pinned host arrays: the kernels write them in place
        const int rc = ensure_caller_maps(m, s);
        if (rc != UE_OK) return rc;
        UE_CUDA(ue::launch_fields_out_caller(m->dm, const_cast<void*>(dE), const_cast<void*>(dB),
                                             const_cast<void*>(dj), false, m->d_kof, m->d_inv, m->d_relen,
                                             h.n_edges, s));
        m->direct_fields += (E ? 1 : 0) + (B ? 1 : 0) + (j ? 1 : 0);
    } else {
        if (E) UE_CUDA(cudaMemsetAsync(m->d_Ec, 0, 8 * h.n_edges, s));
        if (j) UE_CUDA(cudaMemsetAsync(m->d_Jc, 0, 8 * h.n_edges, s));
        UE_CUDA(ue::launch_fields_out(m->dm, E ? m->d_Ec : nullptr, B ? m->d_Bc : nullptr,
                                      j ? m->d_Jc : nullptr, m->d_ecaller, m->d_perm, m->d_relen, s));
        if (E && m->has_reg)
            UE_CUDA(ue::launch_frame_iface_out(m->reg.f, m->reg.dm, m->d_iedge, m->d_ielen, m->d_Ec, s));
        else if (E && m->dm.frame)
            UE_CUDA(ue::launch_frame_iface_out(m->fd, m->dm, m->d_iedge, m->d_ielen, m->d_Ec, s));
        if (E) UE_CUDA(cudaMemcpyAsync(E, m->d_Ec, 8 * h.n_edges, cudaMemcpyDeviceToHost, s));
        if (B) UE_CUDA(cudaMemcpyAsync(B, m->d_Bc, 8 * h.n_tris, cudaMemcpyDeviceToHost, s));
        if (j) UE_CUDA(cudaMemcpyAsync(j, m->d_Jc, 8 * h.n_edges, cudaMemcpyDeviceToHost, s));
    }
    double wd[4];
    UE_CUDA(cudaMemcpyAsync(wd, m->wd, sizeof(wd), cudaMemcpyDeviceToHost, s));
    UE_CUDA(cudaStreamSynchronize(s));
    if (wd[3] != 0.0)
        return fail(UE_ERR_UNSTABLE, std::string("energy watchdog: ") +
                                         (wd[3] == 1.0 ? "non-finite energy" : "energy growth beyond the limit") +
                                         " (W = " + std::to_string(wd[1]) + ")");
    return UE_OK;
}

int ue_energy(ue_mesh* m, double* W, void* stream) {
    if (!m || !m->built || !W) return fail(UE_ERR_ARG, "geometry not built or NULL output");
    cudaStream_t s = (cudaStream_t)stream;
    UE_CUDA(ue::launch_energy(m->dm, m->d_elen, m->d_d, m->d_S, m->wd_part, m->wd, s));
    double wd[4];
    UE_CUDA(cudaMemcpyAsync(wd, m->wd, sizeof(wd), cudaMemcpyDeviceToHost, s));
    UE_CUDA(cudaStreamSynchronize(s));
    *W = wd[1];
    return UE_OK;
}

int ue_check(ue_mesh* m, double* W, int32_t* flag) {
    if (!m || !m->built) return fail(UE_ERR_ARG, "geometry not built");
    double wd[4];
    UE_CUDA(cudaMemcpy(wd, m->wd, sizeof(wd), cudaMemcpyDeviceToHost));
    if (W) *W = wd[1];
    if (flag) *flag = (int32_t)wd[3];
    if (m->p_err) {
        int e = 0;
        UE_CUDA(cudaMemcpy(&e, m->p_err, 4, cudaMemcpyDeviceToHost));
        if (e) {
            if (flag) *flag = 3;
            return fail(UE_ERR_TIMEOUT, "a grid barrier of the persistent kernel ran out of time");
        }
    }
    if (m->variant == UE_VARIANT_BLOCKED && m->tb.done) {
        unsigned e = 0;
        UE_CUDA(cudaMemcpy(&e, m->tb.done + 1, 4, cudaMemcpyDeviceToHost));
        if (e) {
            if (flag) *flag = 3;
            return fail(UE_ERR_TIMEOUT, "a copy wait of the pipelined blocked kernel ran out of time");
        }
    }
    if (wd[3] != 0.0)
        return fail(UE_ERR_UNSTABLE, std::string("energy watchdog: ") +
                                         (wd[3] == 1.0 ? "non-finite energy" : "energy growth beyond the limit"));
    return UE_OK;
}

int ue_get_step(const ue_mesh* m, int64_t* step) {
    if (!m || !m->built || !step) return fail(UE_ERR_ARG, "geometry not built or NULL output");
    if (m->step_pending >= 0) {   // set and not stepped since
        *step = m->step_pending;
        return UE_OK;
    }
    long long v = 0;
    UE_CUDA(cudaMemcpy(&v, m->dm.step, 8, cudaMemcpyDeviceToHost));
    *step = v;
    return UE_OK;
}

int ue_set_step(ue_mesh* m, int64_t step) {
    if (!m || !m->built || step < 0) return fail(UE_ERR_ARG, "geometry not built or step < 0");
    m->step_pending = step;
    m->steps_done = 0;
    return UE_OK;
}

int ue_get_sizes(const ue_mesh* m, int64_t* nn, int64_t* nt, int64_t* ne, int64_t* nei) {
    if (!m) return fail(UE_ERR_ARG, "mesh is NULL");
    if (nn) *nn = m->hm.n_nodes;
    if (nt) *nt = m->hm.n_tris;
    if (ne) *ne = m->hm.n_edges;
    if (nei) *nei = m->hm.n_ei;
    return UE_OK;
}

int ue_get_tables(const ue_mesh* m, int64_t* perm_tri, int64_t* edge_caller, int32_t* edge_tri,
                  int32_t* tri_code) {
    if (!m) return fail(UE_ERR_ARG, "mesh is NULL");
    const HostMesh& h = m->hm;
    if (perm_tri) std::memcpy(perm_tri, h.perm_tri.data(), 8 * h.n_tris);
    if (edge_caller) std::memcpy(edge_caller, h.edge_caller.data(), 8 * h.n_ei);
    if (edge_tri) std::memcpy(edge_tri, h.edge_tri.data(), 8 * h.n_ei);
    if (tri_code) std::memcpy(tri_code, h.tri_code.data(), 12 * h.n_tris);
    return UE_OK;
}

int ue_get_tiles(const ue_mesh* m, int64_t* n_tiles, int64_t* tile_off) {
    if (!m || !n_tiles) return fail(UE_ERR_ARG, "mesh or n_tiles is NULL");
    const std::vector<int64_t>& o = m->hm.tile_tri_off;
    *n_tiles = o.size() < 2 ? 0 : (int64_t)o.size() - 1;
    if (tile_off && *n_tiles > 0) std::memcpy(tile_off, o.data(), 8 * o.size());
    return UE_OK;
}

int ue_frame_attach(ue_mesh* m, int32_t width, double sigma_max, int32_t order) {
    if (!m) return fail(UE_ERR_ARG, "mesh is NULL");
    if (m->is_batch) return fail(UE_ERR_ARG, "a batch cannot take a frame");
    if (width == 0) {
        m->fr = FrameHost();
        return UE_OK;
    }
    if (width < 1 || width > 256 || order < 1 || order > 8 || !std::isfinite(sigma_max))
        return fail(UE_ERR_ARG, "frame: width in [1, 256], order in [1, 8], finite sigma_max");
    const HostMesh& h = m->hm;
    if (h.n_nodes < 3 || h.n_tris < 1) return fail(UE_ERR_ARG, "frame: empty mesh");
    FrameHost fr;
    fr.W = width;
    fr.order = order;
    fr.X0 = fr.X1 = h.xy[0];
    fr.Y0 = fr.Y1 = h.xy[1];
    for (int64_t v = 0; v < h.n_nodes; ++v) {
        fr.X0 = std::min(fr.X0, h.xy[2 * v]);
        fr.X1 = std::max(fr.X1, h.xy[2 * v]);
        fr.Y0 = std::min(fr.Y0, h.xy[2 * v + 1]);
        fr.Y1 = std::max(fr.Y1, h.xy[2 * v + 1]);
    }
    const double tol = 1e-9 * std::max(fr.X1 - fr.X0, fr.Y1 - fr.Y0);
    // the mesh's boundary edges that lie on a side of the bounding box
    struct BE {
        int64_t slot;
        int32_t a, b;
        double lo;
    };
    std::vector<BE> side[4];   // bottom, top, left, right
    for (int64_t t = 0; t < h.n_tris; ++t)
        for (int q = 0; q < 3; ++q) {
            if ((h.tri_code[3 * t + q] >> 1) != h.n_ei) continue;
            const int32_t a = h.tri_nodes[3 * t + q], b = h.tri_nodes[3 * t + (q + 1) % 3];
            const double xa = h.xy[2 * a], ya = h.xy[2 * a + 1], xb = h.xy[2 * b], yb = h.xy[2 * b + 1];
            int sd = -1;
            if (std::fabs(ya - fr.Y0) <= tol && std::fabs(yb - fr.Y0) <= tol) sd = 0;
            else if (std::fabs(ya - fr.Y1) <= tol && std::fabs(yb - fr.Y1) <= tol) sd = 1;
            else if (std::fabs(xa - fr.X0) <= tol && std::fabs(xb - fr.X0) <= tol) sd = 2;
            else if (std::fabs(xa - fr.X1) <= tol && std::fabs(xb - fr.X1) <= tol) sd = 3;
            if (sd < 0) continue;
            side[sd].push_back({3 * t + q, a, b, sd < 2 ? std::min(xa, xb) : std::min(ya, yb)});
        }
    fr.nx = (int)side[0].size();
    fr.ny = (int)side[2].size();
    if (fr.nx < 1 || fr.ny < 1 || (int)side[1].size() != fr.nx || (int)side[3].size() != fr.ny)
        return fail(UE_ERR_ARG, "frame: the outer boundary is not an axis-aligned rectangle");
    fr.h = (fr.X1 - fr.X0) / fr.nx;
    if (std::fabs((fr.Y1 - fr.Y0) - fr.ny * fr.h) > 1e-6 * fr.h)
        return fail(UE_ERR_ARG, "frame: the boundary spacing differs between the x and y sides");
    ue::FrameDev lay;
    lay.W = fr.W;
    lay.nx = fr.nx;
    lay.ny = fr.ny;
    lay.NX = fr.nx + 2 * fr.W;
    lay.NY = fr.ny + 2 * fr.W;
    const double nin[4][2] = {{0, 1}, {0, -1}, {1, 0}, {-1, 0}};
    for (int sd = 0; sd < 4; ++sd) {
        std::vector<BE>& v = side[sd];
        std::sort(v.begin(), v.end(), [](const BE& p, const BE& q) { return p.lo < q.lo; });
        const double start = sd < 2 ? fr.X0 : fr.Y0;
        for (size_t i = 0; i < v.size(); ++i) {
            const BE& e = v[i];
            const double lo = start + (double)i * fr.h;
            const double p0 = sd < 2 ? std::min(h.xy[2 * e.a], h.xy[2 * e.b]) : std::min(h.xy[2 * e.a + 1], h.xy[2 * e.b + 1]);
            const double p1 = sd < 2 ? std::max(h.xy[2 * e.a], h.xy[2 * e.b]) : std::max(h.xy[2 * e.a + 1], h.xy[2 * e.b + 1]);
            if (std::fabs(p0 - lo) > 1e-6 * fr.h || std::fabs(p1 - (lo + fr.h)) > 1e-6 * fr.h)
                return fail(UE_ERR_ARG, "frame: the outer boundary nodes are not uniformly spaced");
            const int t = (int)(e.slot / 3);
            const bool triR = e.a < e.b;   // the triangle runs the edge low -> high: it is R
            int I = 0, J = 0;
            if (sd == 0) { I = fr.W + (int)i; J = fr.W - 1; }
            else if (sd == 1) { I = fr.W + (int)i; J = fr.W + fr.ny; }
            else if (sd == 2) { I = fr.W - 1; J = fr.W + (int)i; }
            else { I = fr.W + fr.nx; J = fr.W + (int)i; }
            fr.itri.push_back(triR ? t : ~t);
            fr.icell.push_back((int32_t)ue::frame_cell(lay, I, J));
            fr.islot.push_back(e.slot);
            fr.ineg.push_back(triR ? 0 : 1);
            const int64_t lo_n = std::min(e.a, e.b), hi_n = std::max(e.a, e.b);
            int64_t lo_i = 0, hi_i = h.n_edges;   // caller edges are sorted (low, high) pairs
            while (lo_i < hi_i) {
                const int64_t mid = (lo_i + hi_i) / 2;
                const int64_t ma = h.edges[2 * mid], mb = h.edges[2 * mid + 1];
                if (ma < lo_n || (ma == lo_n && mb < hi_n)) lo_i = mid + 1;
                else hi_i = mid;
            }
            fr.iedge.push_back(lo_i);
            const double ex = h.xy[2 * e.b] - h.xy[2 * e.a], ey = h.xy[2 * e.b + 1] - h.xy[2 * e.a + 1];
            fr.ielen.push_back(std::sqrt(ex * ex + ey * ey));
            const double g[6] = {h.xy[2 * e.a], h.xy[2 * e.a + 1], h.xy[2 * e.b], h.xy[2 * e.b + 1],
                                 nin[sd][0], nin[sd][1]};
            fr.iface.insert(fr.iface.end(), g, g + 6);
        }
    }
    fr.sigma_max = sigma_max >= 0 ? sigma_max
                                  : (order + 1) * std::log(1e6) / (2.0 * width * fr.h);
    m->fr = std::move(fr);
    return UE_OK;
}

int ue_frame_get(const ue_mesh* m, int64_t* dims, double* geom) {
    if (!m || m->fr.W == 0) return fail(UE_ERR_ARG, "no frame");
    const FrameHost& fr = m->fr;
    const int64_t NX = fr.nx + 2 * fr.W, NY = fr.ny + 2 * fr.W;
    if (dims) {
        const int64_t d[7] = {fr.W, fr.nx, fr.ny, NX, NY, 2 * fr.W * NX + 2 * (int64_t)fr.W * fr.ny,
                              (int64_t)fr.itri.size()};
        std::memcpy(dims, d, sizeof(d));
    }
    if (geom) {
        const double g[4] = {fr.h, fr.X0, fr.Y0, fr.sigma_max};
        std::memcpy(geom, g, sizeof(g));
    }
    return UE_OK;
}

int ue_frame_interface(const ue_mesh* m, int64_t* edge, int64_t* cell) {
    if (!m || m->fr.W == 0) return fail(UE_ERR_ARG, "no frame");
    const FrameHost& fr = m->fr;
    for (size_t k = 0; k < fr.itri.size(); ++k) {
        if (edge) edge[k] = fr.iedge[k];
        if (cell) cell[k] = fr.icell[k];
    }
    return UE_OK;
}

int ue_frame_region(const ue_mesh* m, int32_t block_depth, int64_t* counts) {
    if (!m || m->fr.W == 0 || !counts) return fail(UE_ERR_ARG, "no frame or NULL counts");
    if (m->hm.tile_tri_off.size() < 2) return fail(UE_ERR_ARG, "the mesh has no tiles");
    if (block_depth < 1 || block_depth > 15) return fail(UE_ERR_ARG, "block_depth must be in 1..15");
    std::vector<char> interior, owned;
    region_plan(m, block_depth, interior, owned);
    ue::Region R;
    std::string err;
    const int rc = ue::build_region(m->hm, owned, block_depth, m->fr.islot, m->fr.ineg, R, err);
    if (rc != UE_OK) return fail(rc, err);
    int64_t n_int = 0;
    for (char c : interior) n_int += c;
    counts[0] = (int64_t)interior.size();
    counts[1] = n_int;
    counts[2] = R.n_own_t;
    counts[3] = (int64_t)R.tgid.size();
    counts[4] = (int64_t)R.egid.size();
    counts[5] = R.n_own_e;
    return UE_OK;
}

int ue_frame_state(ue_mesh* m, double* Bx, double* By, double* Ex, double* Ey, int32_t write, void* stream) {
    if (!m || !m->built || !m->dm.frame) return fail(UE_ERR_ARG, "no frame built");
    if (!Bx || !By || !Ex || !Ey) return fail(UE_ERR_ARG, "ue_frame_state needs all four arrays");
    cudaStream_t s = (cudaStream_t)stream;
    const ue::FrameDev& f = m->fd;
    const int64_t nh = (int64_t)f.NX * (f.NY + 1), nv = (int64_t)(f.NX + 1) * f.NY;
    double *tx = nullptr, *ty = nullptr, *th = nullptr, *tv = nullptr;
    if (!alloc_into(m, tx, f.n_fc, 8, s) || !alloc_into(m, ty, f.n_fc, 8, s) || !alloc_into(m, th, nh, 8, s) ||
        !alloc_into(m, tv, nv, 8, s))
        return fail(UE_ERR_ALLOC, "frame state buffers");
    const bool f64 = m->precision == UE_PREC_FP64;
    if (write) {
        UE_CUDA(cudaMemcpyAsync(tx, Bx, 8 * f.n_fc, cudaMemcpyHostToDevice, s));
        UE_CUDA(cudaMemcpyAsync(ty, By, 8 * f.n_fc, cudaMemcpyHostToDevice, s));
        UE_CUDA(cudaMemcpyAsync(th, Ex, 8 * nh, cudaMemcpyHostToDevice, s));
        UE_CUDA(cudaMemcpyAsync(tv, Ey, 8 * nv, cudaMemcpyHostToDevice, s));
        UE_CUDA(ue::launch_frame_state(f, f64, tx, ty, th, tv, true, s));
    } else {
        UE_CUDA(ue::launch_frame_state(f, f64, tx, ty, th, tv, false, s));
        UE_CUDA(cudaMemcpyAsync(Bx, tx, 8 * f.n_fc, cudaMemcpyDeviceToHost, s));
        UE_CUDA(cudaMemcpyAsync(By, ty, 8 * f.n_fc, cudaMemcpyDeviceToHost, s));
        UE_CUDA(cudaMemcpyAsync(Ex, th, 8 * nh, cudaMemcpyDeviceToHost, s));
        UE_CUDA(cudaMemcpyAsync(Ey, tv, 8 * nv, cudaMemcpyDeviceToHost, s));
    }
    UE_CUDA(cudaStreamSynchronize(s));
    for (double* p : {tx, ty, th, tv}) dev_release(m, p, s);
    return UE_OK;
}

int ue_frame_fields(ue_mesh* m, double* B, double* Ex, double* Ey, void* stream) {
    if (!m || !m->built || !m->dm.frame) return fail(UE_ERR_ARG, "no frame built");
    cudaStream_t s = (cudaStream_t)stream;
    const ue::FrameDev& f = m->fd;
    const int64_t nh = (int64_t)f.NX * (f.NY + 1), nv = (int64_t)(f.NX + 1) * f.NY;
    double *tB = nullptr, *tx = nullptr, *ty = nullptr;
    if ((B && !alloc_into(m, tB, f.n_fc, 8, s)) || (Ex && !alloc_into(m, tx, nh, 8, s)) ||
        (Ey && !alloc_into(m, ty, nv, 8, s)))
        return fail(UE_ERR_ALLOC, "frame export buffers");
    UE_CUDA(ue::launch_frame_out(f, m->precision == UE_PREC_FP64, tB, tx, ty, s));
    if (B) UE_CUDA(cudaMemcpyAsync(B, tB, 8 * f.n_fc, cudaMemcpyDeviceToHost, s));
    if (Ex) UE_CUDA(cudaMemcpyAsync(Ex, tx, 8 * nh, cudaMemcpyDeviceToHost, s));
    if (Ey) UE_CUDA(cudaMemcpyAsync(Ey, ty, 8 * nv, cudaMemcpyDeviceToHost, s));
    UE_CUDA(cudaStreamSynchronize(s));
    dev_release(m, tB, s);
    dev_release(m, tx, s);
    dev_release(m, ty, s);
    return UE_OK;
}

int ue_get_geometry(ue_mesh* m, double* O, double* S, double* elen, double* d) {
    if (!m || !m->built) return fail(UE_ERR_ARG, "geometry not built");
    const HostMesh& h = m->hm;
    cudaStream_t s = nullptr;
    double *tO = nullptr, *tS = nullptr, *tl = nullptr, *td = nullptr;
    if ((O && !alloc_into(m, tO, 2 * h.n_tris, 8, s)) || (S && !alloc_into(m, tS, h.n_tris, 8, s)) ||
        (elen && !alloc_into(m, tl, h.n_edges, 8, s)) || (d && !alloc_into(m, td, h.n_edges, 8, s)))
        return fail(UE_ERR_ALLOC, "geometry export buffers");
    UE_CUDA(ue::launch_scatter_geometry(m->d_O, m->d_S, m->d_elen, m->d_d, m->d_perm, m->d_ecaller,
                                        h.n_tris, h.n_ei, h.n_edges, tO, tS, tl, td, s));
    if (O) UE_CUDA(cudaMemcpy(O, tO, 16 * h.n_tris, cudaMemcpyDeviceToHost));
    if (S) UE_CUDA(cudaMemcpy(S, tS, 8 * h.n_tris, cudaMemcpyDeviceToHost));
    if (elen) UE_CUDA(cudaMemcpy(elen, tl, 8 * h.n_edges, cudaMemcpyDeviceToHost));
    if (d) UE_CUDA(cudaMemcpy(d, td, 8 * h.n_edges, cudaMemcpyDeviceToHost));
    return UE_OK;
}

int ue_rho_features(ue_mesh* m, float* X, float* base, void* stream) {
    if (!m || !m->built || !X || !base) return fail(UE_ERR_ARG, "geometry not built or NULL output");
    // the outer edges of a framed mesh are unknowns the features do not describe
    if (m->dm.frame) return fail(UE_ERR_ARG, "ue_rho_features: not on a framed mesh");
    cudaStream_t s = (cudaStream_t)stream;
    const int nrc = ensure_tri_nb(m, s);
    if (nrc != UE_OK) return nrc;
    UE_CUDA(ue::launch_features(m->d_xy, m->d_tri_nodes, m->d_tri_code, m->d_tri_nb, m->d_elen, m->d_d,
                                m->d_S, m->hm.n_tris, m->hm.n_ei, X, base, s));
    UE_CUDA(cudaStreamSynchronize(s));
    return UE_OK;
}

int ue_mlp_forward(const float* params, const float* X, int64_t n, int32_t bf16, float* z, void* stream) {
    if (!params || !X || !z || n < 0) return fail(UE_ERR_ARG, "bad arguments");
    UE_CUDA(ue::launch_mlp_forward(params, X, n, bf16 ? 1 : 0, z, (cudaStream_t)stream));
    return UE_OK;
}

int ue_mlp_backward(const float* params, const float* X, const int64_t* rows, const float* dz,
                    int64_t m, int32_t bf16, float* work, float* grad, void* stream) {
    if (!params || !X || !grad || m < 0 || (m > 0 && (!rows || !dz || !work))) return fail(UE_ERR_ARG, "bad arguments");
    UE_CUDA(ue::launch_mlp_backward(params, X, rows, dz, m, bf16 ? 1 : 0, work, grad, (cudaStream_t)stream));
    return UE_OK;
}

int ue_adam(float* params, const float* grad, float* m1, float* m2, int32_t n, float lr, float beta1,
            float beta2, float eps, int32_t t, void* stream) {
    if (!params || !grad || !m1 || !m2 || n < 1 || t < 1) return fail(UE_ERR_ARG, "bad arguments");
    UE_CUDA(ue::launch_adam(params, grad, m1, m2, n, lr, beta1, beta2, eps, t, (cudaStream_t)stream));
    return UE_OK;
}

int ue_seg_argmax(const float* z, const float* base, const int64_t* off, int32_t n_seg, float* best,
                  int64_t* arg, void* stream) {
    if (!z || !base || !off || !best || !arg || n_seg < 0) return fail(UE_ERR_ARG, "bad arguments");
    UE_CUDA(ue::launch_seg_argmax(z, base, off, n_seg, best, arg, (cudaStream_t)stream));
    return UE_OK;
}

int ue_rho_loss(const float* best, const float* target, int32_t n_seg, float* dz, float* loss, void* stream) {
    if (!best || !target || !dz || !loss || n_seg < 0) return fail(UE_ERR_ARG, "bad arguments");
    UE_CUDA(ue::launch_rho_loss(best, target, n_seg, dz, loss, (cudaStream_t)stream));
    return UE_OK;
}

int ue_profile_steps(ue_mesh* m, int64_t n, void* stream, double* ms, double* bytes) {
    if (!m || !m->built) return fail(UE_ERR_ARG, "geometry not built");
    if (n < 1 || n > 4096 || !ms) return fail(UE_ERR_ARG, "n_steps must be in 1..4096 and ms non-NULL");
    cudaStream_t s = (cudaStream_t)stream;
    {
        const int frc = flush_step(m, s);
        if (frc != UE_OK) return frc;
    }
    const bool blocked = m->variant == UE_VARIANT_BLOCKED;
    // events: plain step i = [gtab | E half-step | B half-step] at 4i..4i+3;
    // blocked launch i = [g table (untimed) ... | k_tb] at 4i+1..4i+2
    std::vector<cudaEvent_t> ev(4 * n, nullptr);
    int rc = UE_OK;
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            rc = fail(UE_ERR_CUDA, "cudaEventCreate");
            break;
        }
    for (int64_t i = 0; i < n && rc == UE_OK; ++i) {
        cudaError_t e = cudaEventRecord(ev[4 * i], s);
        if (e == cudaSuccess) e = ue::launch_gtab(m->dm, blocked ? m->block_depth : 1, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[4 * i + 1], s);
        if (blocked) {
            // the blocked tiles, then (framed) the region: timed apart
            if (e == cudaSuccess && m->tb.n_tiles > 0) e = ue::launch_tb(m->tb, m->dm, m->block_depth, m->cur, 0, s);
            if (e == cudaSuccess) e = cudaEventRecord(ev[4 * i + 2], s);
            if (e == cudaSuccess && m->has_reg) {
                const bool tiles = m->tb.n_tiles > 0;
                m->tb.n_tiles = 0;   // region part only
                e = blocked_launch(m, m->block_depth, m->cur, 0, s);
                m->tb.n_tiles = tiles ? m->ts.n_tiles : 0;
            }
            if (e == cudaSuccess) set_current(m, m->cur ^ 1);
            if (e == cudaSuccess) e = cudaEventRecord(ev[4 * i + 3], s);
        } else {
            if (e == cudaSuccess) e = ue::launch_step_part(m->dm, 0, 0, s);
            if (e == cudaSuccess) e = cudaEventRecord(ev[4 * i + 2], s);
            if (e == cudaSuccess) e = ue::launch_step_part(m->dm, 1, 0, s);
            if (e == cudaSuccess) e = cudaEventRecord(ev[4 * i + 3], s);
        }
        if (e != cudaSuccess) rc = fail(UE_ERR_CUDA, std::string("profile launch: ") + cudaGetErrorString(e));
    }
    double acc[3] = {0, 0, 0};
    if (rc == UE_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = fail(UE_ERR_CUDA, std::string("profile sync: ") + cudaGetErrorString(e));
        for (int64_t i = 0; i < n && rc == UE_OK; ++i) {
            float t[3] = {0, 0, 0};
            for (int p = 0; p < 3; ++p) cudaEventElapsedTime(&t[p], ev[4 * i + p], ev[4 * i + p + 1]);
            acc[0] += t[1];   // E half-step, or the blocked kernel
            acc[1] += t[0];   // g table
            acc[2] += t[2];   // B half-step
        }
    }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (rc != UE_OK) return rc;
    for (int p = 0; p < 3; ++p) ms[p] = acc[p] / (double)n;
    const int64_t per = blocked ? m->block_depth : 1;
    m->steps_done += n * per;
    m->launches += blocked ? n * (blocked_launches(m, m->block_depth) + (m->dm.n_src > 0 ? 1 : 0))
                           : plain_launches(m, n, 1);
    if (bytes) {
        const double f = m->precision == UE_PREC_FP64 ? 2.0 : 1.0;
        const HostMesh& h = m->hm;
        const double pl = m->dm.plasma ? 1.0 : 0.0;
        if (blocked) {
            // the blocked kernel owns what the region (if any) does not
            const double ot = (double)(h.n_tris - (m->has_reg ? m->reg.n_own_t : 0));
            const double oe = (double)(h.n_ei - (m->has_reg ? m->reg.n_own_e : 0));
            bytes[0] = (double)per * ((20.0 + 12.0 * pl) * oe + 24.0 * ot);
            bytes[1] = 20.0 * (double)m->tb.n_trec + (16.0 + 8.0 * pl) * (double)m->tb.n_erec + 4.0 * ot +
                       (4.0 + 4.0 * pl) * oe;
            bytes[2] = m->has_reg ? (double)per * (20.0 * (double)m->reg.dm.n_ei + 24.0 * (double)m->reg.dm.n_t) : 0.0;
            if (!m->has_reg) ms[2] = 0;
        } else {
            bytes[0] = (8.0 + f * 12.0 + pl * f * 12.0) * (double)h.n_ei;
            bytes[1] = 8.0 * (m->dm.n_src > 0 ? 1.0 : 0.0);
            bytes[2] = (16.0 + f * 8.0 + (m->precision == UE_PREC_FP64 ? 8.0 : 0.0)) * (double)h.n_tris;
        }
    }
    return UE_OK;
}

int ue_mesh_flip(const double* xy, int64_t n_nodes, const int32_t* tris, int64_t n_tris, const int32_t* segs,
                 int64_t n_segs, int32_t* tris_out, int64_t* n_flips) {
    Range nvtx_range("ue_mesh_flip");
    if (!xy || !tris || !tris_out || n_nodes < 3 || n_tris < 1 || n_segs < 0 || (n_segs > 0 && !segs))
        return fail(UE_ERR_ARG, "ue_mesh_flip: bad arguments");
    if (n_nodes >= (int64_t)1 << 31 || 3 * n_tris >= (int64_t)1 << 31)
        return fail(UE_ERR_ARG, "ue_mesh_flip: mesh too large for 32-bit indices");
    std::string err;
    const int rc = ue::mesh_flip(xy, n_nodes, tris, n_tris, segs, n_segs, tris_out, n_flips, err);
    if (rc != UE_OK) return fail(rc, "ue_mesh_flip: " + err);
    return UE_OK;
}

int ue_mesh_relax(const double* xy, int64_t n_nodes, const int32_t* tris, int64_t n_tris,
                  const double* h_nodes, int32_t iters, int32_t flip_every, double tau,
                  const int32_t* anchors, int64_t n_anchors, const int32_t* segs, int64_t n_segs,
                  double* xy_out, int32_t* tris_out, int64_t* n_flips, void* stream) {
    Range nvtx_range("ue_mesh_relax");
    if (!xy || !tris || !xy_out || !tris_out || n_nodes < 3 || n_tris < 1 || iters < 0 || flip_every < 0 ||
        n_anchors < 0 || n_segs < 0 || (n_anchors > 0 && !anchors) || (n_segs > 0 && !segs))
        return fail(UE_ERR_ARG, "ue_mesh_relax: bad arguments");
    if (n_nodes >= (int64_t)1 << 31 || 3 * n_tris >= (int64_t)1 << 31)
        return fail(UE_ERR_ARG, "ue_mesh_relax: mesh too large for 32-bit indices");
    if (!(tau > 0.0 && tau <= 0.1)) return fail(UE_ERR_ARG, "ue_mesh_relax: tau must be in (0, 0.1]");
    std::string err;
    const int rc = ue::mesh_relax(xy, n_nodes, tris, n_tris, h_nodes, iters, flip_every, tau, anchors,
                                  n_anchors, segs, n_segs, xy_out, tris_out, n_flips, (cudaStream_t)stream, err);
    if (rc != UE_OK) return fail(rc, err);
    return UE_OK;
}

int ue_triangulate(const double* xy, int64_t n_nodes, const int32_t* segs, int64_t n_segs,
                   const double* holes, int64_t n_holes, int32_t flags, int32_t* tris, int64_t cap_tris,
                   int64_t* n_tris, int64_t* n_flips) {
    Range nvtx_range("ue_triangulate");
    if (!tris || !n_tris || cap_tris < 0 || (flags & ~UE_TRI_DROP_EXTERIOR))
        return fail(UE_ERR_ARG, "ue_triangulate: bad arguments");
    std::vector<int32_t> out;
    std::string err;
    int rc;
    try {
        rc = ue::triangulate(xy, n_nodes, segs, n_segs, holes, n_holes, flags, out, n_flips, err);
    } catch (const std::bad_alloc&) {
        rc = UE_ERR_ARG;
        err = "ue_triangulate: out of host memory";
    }
    if (rc != UE_OK) return fail(rc, err);
    *n_tris = (int64_t)out.size() / 3;
    if (*n_tris > cap_tris) return fail(UE_ERR_ARG, "ue_triangulate: cap_tris too small");
    std::memcpy(tris, out.data(), sizeof(int32_t) * out.size());
    return UE_OK;
}

int ue_modes_low(ue_mesh* m, int32_t n_modes, int32_t iters, int32_t degree, uint32_t seed, double* omega,
                 double* B, void* stream) {
    Range nvtx_range("ue_modes_low");
    if (!m || !m->built || !omega) return fail(UE_ERR_ARG, "geometry not built or NULL omega");
    if (n_modes < 1 || n_modes > 16 || iters < 1 || degree < 2 || degree > 200)
        return fail(UE_ERR_ARG, "ue_modes_low: n_modes in [1, 16], iters >= 1, degree in [2, 200]");
    if (m->dm.frame) return fail(UE_ERR_ARG, "ue_modes_low: not on a framed mesh");
    cudaStream_t s = (cudaStream_t)stream;
    const HostMesh& h = m->hm;
    const int64_t nt = h.n_tris, nei = h.n_ei;
    const int bw = ue::modes_block_size(n_modes);
    if (nt < bw) return fail(UE_ERR_ARG, "ue_modes_low: the mesh has fewer triangles than the block of vectors");
    double* work = nullptr;
    double* Bd = nullptr;
    if (!alloc_into(m, work, ue::modes_low_work_doubles(nt, nei, bw), 8, s) ||
        (B && !alloc_into(m, Bd, (size_t)n_modes * nt, 8, s)))
        return fail(UE_ERR_ALLOC, "ue_modes_low work space");
    bool lost = false;
    UE_CUDA(ue::modes_low_run(m->d_rl, m->dm.tri, m->d_elen, m->d_d, m->d_S, m->d_perm, nt, nei, n_modes,
                              iters, degree, seed, work, omega, Bd, &lost, s));
    if (lost) {
        dev_release(m, work, s);
        if (Bd) dev_release(m, Bd, s);
        return fail(UE_ERR_DUAL, "ue_modes_low: the block of vectors lost rank");
    }
    if (B) UE_CUDA(cudaMemcpy(B, Bd, sizeof(double) * n_modes * nt, cudaMemcpyDeviceToHost));
    dev_release(m, work, s);
    if (Bd) dev_release(m, Bd, s);
    return UE_OK;
}

int ue_modes(ue_mesh* m, int32_t n_modes, int32_t iters, uint32_t seed, double* omega, double* B,
             void* stream) {
    Range nvtx_range("ue_modes");
    if (!m || !m->built || !omega) return fail(UE_ERR_ARG, "geometry not built or NULL omega");
    if (n_modes < 1 || n_modes > 24 || iters < 1)
        return fail(UE_ERR_ARG, "ue_modes: n_modes must be in [1, 24] and iters >= 1");
    // the modes of the closed cavity; a PML frame makes the operator lossy
    if (m->dm.frame) return fail(UE_ERR_ARG, "ue_modes: not on a framed mesh");
    cudaStream_t s = (cudaStream_t)stream;
    const HostMesh& h = m->hm;
    const int64_t nt = h.n_tris, nei = h.n_ei;
    if (nt < ue::modes_block_size(n_modes))
        return fail(UE_ERR_ARG, "ue_modes: the mesh has fewer triangles than the block of vectors");
    double* work = nullptr;
    double* Bd = nullptr;
    if (!alloc_into(m, work, ue::modes_work_doubles(nt, nei, ue::modes_block_size(n_modes)), 8, s) ||
        (B && !alloc_into(m, Bd, (size_t)n_modes * nt, 8, s)))
        return fail(UE_ERR_ALLOC, "ue_modes work space");
    bool lost = false;
    UE_CUDA(ue::modes_run(m->d_rl, m->dm.tri, m->d_elen, m->d_d, m->d_S, m->d_perm, nt, nei, n_modes,
                          iters, seed, work, omega, Bd, &lost, s));
    if (lost) {
        dev_release(m, work, s);
        if (Bd) dev_release(m, Bd, s);
        return fail(UE_ERR_DUAL, "ue_modes: the block of vectors lost rank (fewer independent modes than asked)");
    }
    if (B) UE_CUDA(cudaMemcpy(B, Bd, sizeof(double) * n_modes * nt, cudaMemcpyDeviceToHost));
    dev_release(m, work, s);
    if (Bd) dev_release(m, Bd, s);
    return UE_OK;
}

int ue_power_iteration_static(const int32_t* edge_tri, const double* elen, const double* d,
                              const int32_t* tri_code, const double* S,
                              const int64_t* tri_caller, int64_t n_tris, int64_t n_ei,
                              int32_t iters, uint32_t seed, void* stream, double* rho) {
    std::string err;
    const int rc = ue::power_iteration_static(edge_tri, elen, d, tri_code, S, tri_caller, n_tris,
                                              n_ei, iters, seed, (cudaStream_t)stream, rho, err);
    if (rc != UE_OK) return fail(rc, err);
    return UE_OK;
}

int ue_stats(const ue_mesh* m, ue_stats_t* out) {
    if (!m || !out) return fail(UE_ERR_ARG, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    const HostMesh& h = m->hm;
    out->n_nodes = h.n_nodes;
    out->n_tris = h.n_tris;
    out->n_edges = h.n_edges;
    out->n_interior_edges = h.n_ei;
    out->steps_done = m->steps_done;
    out->dt = m->dt;
    out->rho = m->rho;
    out->rho_source = m->rho_source;
    out->precision = m->precision;
    const double f = m->precision == UE_PREC_FP64 ? 2.0 : 1.0;
    // per edge: (R,L) 8 B, coefficient, U read + write; per triangle: 3 codes + dt/S record
    // (16 B; fp64 adds an 8 B dt/S), B read + write; plasma: J read + write and its coefficient
    double per_edge = 8.0 + f * 12.0 + (m->dm.plasma ? f * 12.0 : 0.0);
    double per_tri = 16.0 + f * 8.0 + (m->precision == UE_PREC_FP64 ? 8.0 : 0.0);
    out->bytes_per_step = per_edge * (double)h.n_ei + per_tri * (double)h.n_tris;
    out->kernel_launches = m->launches;
    out->dt_setup_ms = m->dt_setup_ms;
    out->rho_lo = m->rho_lo;
    out->rho_hi = m->rho_hi;
    out->rho_hat = m->rho_hat;
    out->direct_fields = m->direct_fields;
    if (m->variant == UE_VARIANT_BLOCKED && m->built) {
        const bool whole = !m->dm.plasma && !m->has_reg && !m->ts.hdr.empty() && ue::tbf1_fits(m->tb, m->ts.hdr.data());
        out->tb_kernel_used = whole ? UE_TBK_WHOLE_MESH : ue::tb_kernel_used(m->tb, m->dm);
    }
    return UE_OK;
}

void ue_mesh_free(ue_mesh* m) {
    if (!m) return;
    drop_graph(m);
    cudaDeviceSynchronize();
    dev_free_all(m, nullptr);
    if (m->capture_stream) cudaStreamDestroy(m->capture_stream);
    if (m->side) cudaStreamDestroy(m->side);
    if (m->ev_fork) cudaEventDestroy(m->ev_fork);
    if (m->ev_join) cudaEventDestroy(m->ev_join);
    delete m;
}

}  // extern "C"
