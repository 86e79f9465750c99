/*
 * ue.h - C ABI of the leap-frog Maxwell solver on unstructured triangle meshes.
 *
 * Method: D.A. Fadeev, "Numerical simulation of 2D electrodynamic problems with unstructured
 * triangular meshes".  E (and the plasma current j) live on edges, B (out of plane) at the
 * triangles' circumcentres, the plasma density n on nodes (Section 1, Fig. 1).  One time step
 * is the leap-frog pair of eq. 14 (E from t to t+dt, with eq. 3 or, in plasma, eqs. 5-6) and
 * eq. 15 (B from t+dt/2 to t+3dt/2 with eq. 4).
 *
 * Conventions shared by every call:
 *  - All arrays passed in or out are HOST arrays in the CALLER's numbering, owned by the caller;
 *    the library copies what it needs before returning.  Device memory is the library's.
 *  - Nodes: xy[2*v + 0/1].  Triangles: tris[3*j + 0..2] (any orientation; the library makes
 *    them counter-clockwise using the sign of the FP64 orientation determinant).
 *  - Edges are the unique unordered node pairs, numbered by sorting (low id, high id)
 *    lexicographically.  E_i is the projection of E on the edge directed low -> high node id
 *    (the paper leaves the direction free, Fig. 2).  Boundary edges (one triangle) are perfect
 *    conductors: E = 0 there (ideal resonator, eq. 10); they are not unknowns.
 *  - R(i) is the triangle around which edge i runs counter-clockwise, L(i) the other (the
 *    choice that makes eq. 10 vanish).  B is the +z component for right-handed (x, y).
 *  - Time levels: after k steps E is at k*dt, B and j at (k + 1/2)*dt.
 *  - stream arguments are cudaStream_t values passed as void* (NULL = legacy default stream).
 *  - Return codes: UE_OK or a negative UE_ERR_*; ue_last_error() gives the text (per thread).
 *    No C++ exception crosses this boundary.
 */
#ifndef UE_H
#define UE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define UE_OK 0
#define UE_ERR_ARG (-1)          /* bad argument, size or state                               */
#define UE_ERR_NONMANIFOLD (-2)  /* an edge with >2 triangles, or two on the same side        */
#define UE_ERR_DEGENERATE (-3)   /* zero orientation determinant or repeated vertex           */
#define UE_ERR_DUAL (-4)         /* |O_R O_L| <= 0 on an interior edge (mesh not Delaunay)    */
#define UE_ERR_CUDA (-5)         /* a CUDA runtime call failed                                */
#define UE_ERR_ALLOC (-6)        /* device allocation failed (callback returned NULL)         */
#define UE_ERR_UNSTABLE (-7)     /* energy watchdog: growth or non-finite field               */
#define UE_ERR_TIMEOUT (-8)      /* a bounded device wait ran out (persistent kernels)        */

#define UE_REORDER_NONE 0        /* triangles in caller order                                 */
#define UE_REORDER_RCM 1         /* reverse Cuthill-McKee on the dual graph (default)         */
#define UE_REORDER_KD 2          /* KD tiles of <= tile_tris triangles, RCM order inside      */
#define UE_REORDER_GREEDY 3      /* greedy tiles of <= tile_tris triangles, grown breadth     */
                                 /* first from the sharpest boundary triangle, small parts    */
                                 /* and hanging triangles joined; RCM order inside            */
#define UE_REORDER_GREEDY_RINGS 4 /* the same tiles; inside each, the triangles within 15     */
                                 /* rings of its boundary first, ring by ring, each ring by   */
                                 /* angle around the tile's centroid (then RCM order), so a   */
                                 /* neighbour's halo is a few runs of stored ids: the blocked */
                                 /* kernel's layout (tiles as in the greedy method)           */

#define UE_PREC_FP32 0           /* FP32 fields and coefficients (product)                    */
#define UE_PREC_FP64 1           /* FP64 fields and coefficients (check build)                */

#define UE_DT_GIVEN 0            /* use ue_options.dt                                         */
#define UE_DT_POWER 1            /* dt = safety * 2 / rho(M), rho by FP64 power iteration     */
#define UE_DT_LEARNED 2          /* rho from the learned predictor if certified, else power:  */
                                 /* rho~ = max(rho_hat, rho_lo) is used when rho~ <= rho_hi   */
                                 /* and safety * rho_hi * learned_margin <= rho~, i.e. the    */
                                 /* dt it gives stays a margin below 2/rho_hi (eq. 20)        */

#define UE_VARIANT_PLAIN 1       /* two kernels per step (edge half-step, triangle half-step) */
#define UE_VARIANT_BLOCKED 2     /* one kernel per block_depth steps on the tiles, halo       */
                                 /* recomputed in shared memory; FP32; needs KD or greedy     */
                                 /* tiles (UE_REORDER_KD, _GREEDY or _GREEDY_RINGS)           */
#define UE_VARIANT_PERSISTENT 3  /* one cooperative launch per chunk of steps, timed grid     */
                                 /* barriers between half-steps; FP32                         */

#define UE_RHO_GIVEN 0
#define UE_RHO_POWER 1
#define UE_RHO_LEARNED 2         /* learned prediction accepted                               */
#define UE_RHO_POWER_FALLBACK 3  /* learned prediction outside the bracket: power iteration   */

#define UE_MLP_PARAMS 5057       /* W1[64x12], b1[64], W2[64x64], b2[64], w3[64], b3          */

typedef struct ue_mesh ue_mesh;  /* opaque, owned by the library until ue_mesh_free        */

/* Device allocator hooks: alloc(bytes, stream, ctx) returns a device pointer or NULL;
 * free(ptr, stream, ctx) releases it.  Both NULL = cudaMalloc / cudaFree.  Pointers must be
 * 16-byte aligned (the blocked kernels move records and fields with TMA bulk copies): one that
 * is not is handed back to free and the call fails with UE_ERR_ALLOC. */
typedef void* (*ue_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*ue_free_fn)(void* ptr, void* stream, void* ctx);

/* Kernel of the blocked variant (ue_options.tb_kernel).  Both give the plain step's results bit
 * for bit.  SPLIT advances each tile's edges, then its triangles (two barriers per step); FUSED
 * gives each triangle's thread its three edges as well (one barrier per step, half the
 * shared-memory traffic, more instructions), for vacuum media with tiles of at most 4096
 * triangles and halo; others run SPLIT.  A mesh that is a single tile without a halo (at most
 * 2048 triangles) runs all the steps of a call in one launch of one CTA either way. */
#define UE_TB_SPLIT 0
#define UE_TB_FUSED 1

typedef struct ue_options {
    int32_t reorder;       /* UE_REORDER_*, used by ue_mesh_load                              */
    int32_t precision;     /* UE_PREC_*                                                      */
    int32_t dt_mode;       /* UE_DT_*                                                        */
    int32_t power_iters;   /* power-iteration steps (default 200)                            */
    uint32_t power_seed;   /* start vector: SplitMix64(seed * 2^32 + caller triangle id)     */
    int32_t variant;       /* UE_VARIANT_* (0 = default: plain)                              */
    int32_t graph_chunk;   /* steps per captured CUDA graph launch; 0 = default, <0 = none   */
    int32_t tile_tris;     /* UE_REORDER_KD / _GREEDY / _GREEDY_RINGS: maximum triangles per tile (ue_mesh_load) */
    int32_t block_depth;   /* UE_VARIANT_BLOCKED: steps per launch, 1..15                    */
    int32_t tb_threads;    /* UE_VARIANT_BLOCKED: CTA size, 0 = 512 (default) or 1024        */
    double dt;             /* UE_DT_GIVEN: the time step                                     */
    double safety;         /* UE_DT_POWER: dt = safety * 2 / rho (default 0.5)               */
    double watchdog_growth;/* energy watchdog: flag growth by more than this factor between  */
                           /* two checks (default 10)                                        */
    int32_t watchdog_every;/* steps between energy checks inside ue_step_n (0 = off)         */
    int32_t tb_kernel;     /* UE_VARIANT_BLOCKED, vacuum media: UE_TB_SPLIT (default) or     */
                           /* UE_TB_FUSED (see below)                                        */
    const float* mlp_params;/* UE_DT_LEARNED: host array of UE_MLP_PARAMS floats             */
    double learned_margin; /* UE_DT_LEARNED: certified stability margin (default 1.05)       */
    int32_t timeout_ms;    /* UE_VARIANT_PERSISTENT: grid-barrier wait limit (default 2000)  */
    int32_t test_skip_cta; /* tests only (-1 otherwise): UE_VARIANT_PERSISTENT: this CTA     */
                           /* never arrives at the grid barrier; UE_VARIANT_BLOCKED: this CTA */
                           /* of the pipelined forms waits for record bytes that never come.  */
                           /* Either way the bounded wait runs out: UE_ERR_TIMEOUT            */
} ue_options;

typedef struct ue_stats_t {
    int64_t n_nodes, n_tris, n_edges, n_interior_edges;
    int64_t steps_done;          /* leap-frog steps taken since the last ue_set_step          */
    double dt, rho;
    int32_t rho_source;          /* UE_RHO_*                                                  */
    int32_t precision;
    double bytes_per_step;       /* algorithmic HBM bytes of one plain step                   */
    int64_t kernel_launches;     /* kernels the library launched so far                       */
    double dt_setup_ms;          /* wall time of the dt selection in ue_geometry_build (work  */
                                 /* space allocated before it starts)                          */
    double rho_lo, rho_hi;       /* certified bracket (UE_DT_LEARNED), 0 otherwise            */
    double rho_hat;              /* learned prediction (UE_DT_LEARNED), 0 otherwise           */
    int64_t direct_fields;       /* field arrays that ue_write_fields / ue_read_fields moved  */
                                 /* in place in pinned host memory (no staging copy)          */
    int32_t tb_kernel_used;      /* UE_VARIANT_BLOCKED: the kernel its launches run (UE_TBK_*) */
    int32_t reserved2;
} ue_stats_t;

/* Kernels of the blocked variant (ue_stats_t.tb_kernel_used). */
#define UE_TBK_NONE 0              /* not blocked                                              */
#define UE_TBK_SPLIT 1             /* one CTA per tile, edges then triangles                    */
#define UE_TBK_SHARED_RECORDS 2    /* the same with 1024 threads and records in shared memory   */
#define UE_TBK_SPLIT_PIPELINED 3   /* one CTA per SM walking its tiles, next tile's loads ahead */
#define UE_TBK_FUSED 4             /* the same, one thread per triangle with its three edges    */
#define UE_TBK_WHOLE_MESH 5        /* one tile, no halo: every step of a call in one CTA        */

/* Fill *opt with defaults (RCM, FP32, power-iteration dt, safety 0.5, 200 iterations). */
void ue_options_default(ue_options* opt);

/* Mesh ingest (host only; Fig. 2 symbols).  xy: n_nodes*2 doubles, tris: n_tris*3 int32.
 * Orients triangles, builds edges, R/L and the sign table, drops boundary edges from the
 * unknowns and reorders triangles (opt->reorder; opt may be NULL).  alloc/free may be NULL.
 * Errors: UE_ERR_ARG (sizes, indices), UE_ERR_NONMANIFOLD, UE_ERR_DEGENERATE. */
int ue_mesh_load(const double* xy, int64_t n_nodes, const int32_t* tris, int64_t n_tris,
                 const ue_options* opt, ue_alloc_fn alloc, ue_free_fn free_fn, void* alloc_ctx,
                 ue_mesh** out);

/* Device setup: FP64 geometry on the GPU (circumcentres O_j, |e_i|, S_j, and the dual length
 * |O_R O_L| of eq. 3 in the cotangent form), the time step (eq. 20 with rho(M) from FP64 power
 * iteration, Section 2, or the given dt), the update coefficients dt*|e|/d (eq. 3) and dt/S
 * (eq. 4) rounded to the field precision, and zeroed fields.  Synchronous.
 * UE_DT_LEARNED: one fused launch on parameters kept resident on the device (uploaded again
 * only when opt->mlp_params holds other values than the last call on this device); such
 * calls serialise on a library mutex.  The first one per device pins a 64-byte host buffer.
 * Errors: UE_ERR_DUAL if some interior edge has d <= 1e-12*|e|; UE_ERR_CUDA; UE_ERR_ALLOC. */
int ue_geometry_build(ue_mesh* m, const ue_options* opt, void* stream);

/* Batch of independent meshes advanced together: one E and one B half-step launch per step for
 * all of them (or one blocked launch per block_depth steps over all their tiles), inside the
 * same CUDA graphs.  meshes[0..n): built meshes (ue_geometry_build done) with the same
 * precision and variant (blocked: same block_depth and tb_threads) and no plasma medium.  The
 * batch copies their device tables, coefficients, current fields and sources; the meshes stay
 * valid and independent.  Each mesh keeps its own dt and source (its coefficients and source
 * group); the batch's step counter starts at 0.  Caller numbering of the batch is the
 * mesh-major concatenation of the meshes' nodes, triangles and edges.  After k batched steps
 * the fields of every mesh are bit-identical to k steps of that mesh alone.  Free the batch
 * with ue_mesh_free.  ue_set_source and ue_set_plasma are rejected on a batch. */
int ue_batch_create(ue_mesh* const* meshes, int32_t n, void* stream, ue_mesh** out_batch);

/* dt, rho(M) and how rho was obtained (UE_RHO_*). */
int ue_get_dt(const ue_mesh* m, double* dt, double* rho, int32_t* rho_source);

/* Plasma-like medium (eqs. 5-6): n_nodes_density[v] is n at caller node v (n = omega_p^2 in
 * the paper's dimensionless units), nu the collision rate.  The edge density is the mean of
 * its two end nodes.  Requires ue_geometry_build; switches the step to the plasma update.
 * Passing NULL removes the medium. */
int ue_set_plasma(ue_mesh* m, const double* n_nodes_density, double nu);

/* Soft source: at the E update that ends at step n+1, E_i += dt * amp[k] * g(t) with
 * t = (n + 1/2) dt and g(t) = sin(omega0 t) exp(-((t - t0)/tau)^2), for edge_ids[k] (caller
 * numbering, interior edges only, no repeats).  n = 0 removes the source. */
int ue_set_source(ue_mesh* m, const int32_t* edge_ids, const double* amp, int64_t n,
                  double omega0, double t0, double tau);

/* Set E^0 (n_edges values; boundary entries ignored, except the outer edges of a framed mesh),
 * B^{1/2} (n_tris values) and, in plasma, j^{-1/2} (n_edges values, may be NULL = 0).  Any
 * pointer may be NULL to leave that field.  A PML frame's own fields are zeroed.
 * When every given array is 8-byte aligned pinned host memory (cudaHostAlloc, or registered
 * with cudaHostRegister) and the mesh has no PML frame, the kernels read the arrays in place
 * through their mapped device addresses; otherwise they are first copied to the device.  The
 * results are the same either way. */
int ue_write_fields(ue_mesh* m, const double* E, const double* B, const double* j, void* stream);

/* Halo exchange of a mesh partitioned across ranks ("Divide and conqueror": parts exchange the
 * values on their shared boundary every step): B of the triangles with caller ids ids[0..n)
 * is written to buf (scatter = 0) or set from buf (scatter = 1), packed in the field type
 * (float, or double for UE_PREC_FP64).  ids and buf are DEVICE pointers owned by the caller.
 * Synchronous on `stream`.  Ids outside [0, n_tris) are not followed: UE_ERR_ARG. */
int ue_exchange_tris(ue_mesh* m, const int32_t* ids, int64_t n, void* buf, int32_t scatter, void* stream);

/* The same transfers with float arrays (the FP32 product's precision, half the bytes):
 * ue_write_fields_f32 sets U = |e| E and B from them (in FP64, rounded once to the field type),
 * ue_read_fields_f32 returns E = U * (1/|e|) and B rounded to float.  Pinned host arrays are read and
 * written in place; others go through a device copy.  Synchronous.  UE_ERR_ARG for a mesh with
 * a PML frame (use the double calls); ue_read_fields_f32 returns UE_ERR_UNSTABLE (after
 * copying) if the watchdog has flagged the run. */
int ue_write_fields_f32(ue_mesh* m, const float* E, const float* B, const float* j, void* stream);
int ue_read_fields_f32(ue_mesh* m, float* E, float* B, float* j, void* stream);

/* Advance n_steps leap-frog steps, asynchronously on `stream`.  Errors of the launches are
 * reported here; device-side conditions surface at the next synchronous call. */
int ue_step_n(ue_mesh* m, int64_t n_steps, void* stream);

/* Capture and instantiate now the CUDA graphs that ue_step_n replays (a blocked mesh: one per
 * field buffer parity; the plain variant: one), and upload them on `stream`, so that the first
 * ue_step_n call long enough to use them pays no capture.  Steps nothing and leaves the fields
 * and the step counter as they are.  A later call that changes what the steps read
 * (ue_set_source, ue_set_plasma, ue_geometry_build) makes ue_step_n capture again.  No-op for the persistent variant, a mesh stepped
 * as one tile, or graph_chunk 0.  UE_ERR_ARG before geometry_build; UE_ERR_CUDA if a capture
 * fails. */
int ue_step_prepare(ue_mesh* m, void* stream);

/* Copy the fields back in the caller's numbering (synchronous).  E, j: n_edges values (0 on
 * boundary edges, except the outer edges of a framed mesh); B: n_tris values.  Any pointer may
 * be NULL.  Pinned host arrays are written in place by the kernels, as in ue_write_fields.
 * Returns UE_ERR_UNSTABLE (after copying) if the energy watchdog has flagged the run. */
int ue_read_fields(ue_mesh* m, double* E, double* B, double* j, void* stream);

/* Energy W = sum d_i |e_i| E_i^2 + sum S_j B_j^2 of eq. 8 (eq. 7 metric) of the current fields,
 * reduced on the device in FP64 (synchronous).  Also a watchdog check (see ue_check). */
int ue_energy(ue_mesh* m, double* W, void* stream);

/* Watchdog state (synchronous): *W = energy at the last check, *flag = 0 ok, 1 non-finite
 * energy, 2 energy grew by more than watchdog_growth between two checks.  Returns
 * UE_ERR_UNSTABLE when the flag is set, UE_ERR_TIMEOUT (flag 3) when a grid barrier of the
 * persistent variant ran out of time.  ue_write_fields re-arms both. */
int ue_check(ue_mesh* m, double* W, int32_t* flag);

/* Step counter used by the source time t = (n + 1/2) dt (checkpoint / resume).  ue_set_step
 * returns at once: the value reaches the device in the stream of the next ue_step_n (or
 * ue_profile_steps), ordered before its kernels; ue_get_step returns it until then.
 * ue_get_step otherwise reads the device counter (synchronous). */
int ue_get_step(const ue_mesh* m, int64_t* step);
int ue_set_step(ue_mesh* m, int64_t step);

/* Sizes: nodes, triangles, edges, interior edges (unknowns). */
int ue_get_sizes(const ue_mesh* m, int64_t* n_nodes, int64_t* n_tris, int64_t* n_edges,
                 int64_t* n_interior_edges);

/* Connectivity tables as stored on the device (bit-exact checks):
 * perm_tri[n_tris]: caller id of stored triangle j; edge_caller[n_ei]: caller id of stored
 * interior edge k; edge_tri[2*n_ei]: (R, L) in stored triangle ids; tri_code[3*n_tris]:
 * 2*k + (s(j,q) < 0) for the stored edge k = A(j,q), 2*n_ei for a boundary edge, q taken from
 * the vertex triple rotated to start at its smallest caller node id. Any pointer may be NULL. */
int ue_get_tables(const ue_mesh* m, int64_t* perm_tri, int64_t* edge_caller, int32_t* edge_tri,
                  int32_t* tri_code);

/* Tiles of a UE_REORDER_KD, UE_REORDER_GREEDY or UE_REORDER_GREEDY_RINGS mesh ("Divide and
 * conqueror" section):
 * *n_tiles parts (0 for other orders); tile t holds the stored triangles
 * tile_off[t] .. tile_off[t+1]-1.  tile_off (host, n_tiles + 1 entries) may be NULL to ask the
 * count only.  Host only; UE_ERR_ARG if m or n_tiles is NULL. */
int ue_get_tiles(const ue_mesh* m, int64_t* n_tiles, int64_t* tile_off);

/* FP64 geometry computed on the device, caller numbering (after ue_geometry_build):
 * O[2*n_tris] circumcentres, S[n_tris] areas, elen[n_edges] lengths, d[n_edges] signed dual
 * lengths (NaN on boundary edges).  Any pointer may be NULL. */
int ue_get_geometry(ue_mesh* m, double* O, double* S, double* elen, double* d);

/* Learned spectral radius (device pointers, caller-owned; the paper's eq. 20 sets dt from the
 * highest mode, which the network predicts per triangle).
 * ue_rho_features: X[12*n_tris] (float, stored triangle order) and base[n_tris] = log sqrt(K_jj),
 *   K = -L_E L_B, of a built mesh without a PML frame (UE_ERR_ARG otherwise);
 *   log rho_hat = max_j (z_j + base_j).
 * ue_mlp_forward: z[n] for rows X[12*n]; bf16 = 1 tensor cores (BF16 in, FP32 accumulate),
 *   0 = FP32 debug path.  params: UE_MLP_PARAMS floats on the device.
 * ue_mlp_backward: grad[UE_MLP_PARAMS] = sum over m rows of dz[i] * dz_i/dparams for rows[i]
 *   (same rounding as the forward); work holds m * UE_MLP_PARAMS floats.
 * ue_adam: one Adam step (t >= 1) on n floats.
 * ue_seg_argmax: per segment s of rows [off[s], off[s+1]): best = max (z + base), arg.
 * ue_rho_loss: dz[s] = 2 (best[s] - target[s]), loss[s] = (best[s] - target[s])^2.
 * All asynchronous on `stream`. */
int ue_rho_features(ue_mesh* m, float* X, float* base, void* stream);
int ue_mlp_forward(const float* params, const float* X, int64_t n, int32_t bf16, float* z,
                   void* stream);
int ue_mlp_backward(const float* params, const float* X, const int64_t* rows, const float* dz,
                    int64_t m, int32_t bf16, float* work, float* grad, void* stream);
int ue_adam(float* params, const float* grad, float* m1, float* m2, int32_t n, float lr,
            float beta1, float beta2, float eps, int32_t t, void* stream);
int ue_seg_argmax(const float* z, const float* base, const int64_t* off, int32_t n_seg,
                  float* best, int64_t* arg, void* stream);
int ue_rho_loss(const float* best, const float* target, int32_t n_seg, float* dz, float* loss,
                void* stream);

/* Time the step kernels with CUDA events: n_steps (1..4096) launches one by one on `stream`
 * (no graph), then synchronised; the fields advance.
 * Plain variant: ms[0], ms[1], ms[2] = mean device milliseconds of the E half-step (eq. 3 /
 * eqs. 5-6), source and B half-step (eq. 4) kernels; bytes[0..2] = their algorithmic HBM bytes
 * per launch.  Blocked variant: each launch advances block_depth steps; ms[0] = mean per launch,
 * bytes[0] = algorithmic bytes of the same number of plain steps of the triangles and edges it
 * owns, bytes[1] = bytes the blocked kernel streams per launch (tile records, local field reads,
 * owned writes), ms[1] = the source table; with a frame, ms[2] = the region next to the frame
 * (gather, block_depth plain steps with the frame, scatter) and bytes[2] = the plain-kernel bytes
 * of its local triangles and edges over those steps, else 0. */
int ue_profile_steps(ue_mesh* m, int64_t n_steps, void* stream, double* ms, double* bytes);

/* Mesh generation (Section 3, "Mesh generation"; Fig. 5a): the Delaunay triangulation of a
 * node cloud over its convex hull, with geometry segments restored by flipping the edges that
 * cross them, then every other edge made locally Delaunay again (Lawson), so that the result is
 * the constrained Delaunay triangulation; then the triangles reachable from a hole point
 * without crossing a segment are dropped, and with UE_TRI_DROP_EXTERIOR those reachable from a
 * hull edge that is not a segment.  Orientation and in-circle tests are exact, so the result is
 * unique where no four nodes are cocircular, and the same on every host.
 * xy: n_nodes*2 doubles (n_nodes >= 3, no node repeated, not all collinear); segs: n_segs
 * pairs of node ids (may be NULL when n_segs = 0); holes: n_holes points (x, y) inside the
 * regions to drop.  tris (caller-owned, cap_tris*3 int32): the triangles, counter-clockwise;
 * a triangulation of n nodes has at most 2 n - 5 triangles, so cap_tris = 2 n_nodes always
 * suffices.  *n_tris: the count written (or needed, when cap_tris is too small: UE_ERR_ARG).
 * *n_flips (may be NULL): flips made by the segment refinement.  Host only; no GPU call.
 * Errors: UE_ERR_ARG (sizes, ids, a node on a segment, crossing segments, a hole point outside
 * the hull, cap_tris too small); UE_ERR_DEGENERATE (a repeated node, all nodes collinear). */
#define UE_TRI_DROP_EXTERIOR 1
int ue_triangulate(const double* xy, int64_t n_nodes, const int32_t* segs, int64_t n_segs,
                   const double* holes, int64_t n_holes, int32_t flags, int32_t* tris, int64_t cap_tris,
                   int64_t* n_tris, int64_t* n_flips);

/* Mesh optimisation by the jello model with flip refinement (Section 3, "Mesh generation"):
 * nodes joined by unit springs along the triangle edges (rest length (h_a + h_b)/2) and along
 * the heights (vertex to the midpoint of its opposite edge, rest length sqrt(3)/2 times the
 * triangle's mean rest edge) move by strongly damped first-order steps x += tau F,
 * F = -grad of the spring energy, each step clamped to 0.1 of the node's shortest rest edge and
 * to 0.15 of the smallest height of its triangles (so that no triangle turns over);
 * the boundary nodes (on an edge of one triangle: the input geometry) stay, and so do the
 * n_anchors nodes listed in anchors (the seeding nodes of interior geometry: an object's contour
 * meshed on both sides, a path; may be NULL when n_anchors = 0).  Every flip_every steps
 * (0: never) interior edges that are not locally Delaunay are flipped (Lawson), so the
 * triangulation follows the nodes; boundary edges and the n_segs node-id pairs in segs (the
 * geometry's edges; may be NULL when n_segs = 0) are never flipped.  On a randomly seeded node
 * cloud this lowers rho(M) severalfold, allowing a larger dt (eq. 20); nearly cocircular pairs
 * can remain, so check the result with ue_geometry_build (UE_ERR_DUAL).
 * xy: n_nodes*2 doubles; tris: n_tris*3 int32, either orientation.  h_nodes: NULL (uniform:
 * the edge of an equilateral triangle of the mean area) or n_nodes target sizes > 0.
 * tau in (0, 0.1] (explicit steps of this spring system are stable below about 0.1).
 * xy_out, tris_out (CCW) have the input sizes; node numbering is kept.  *n_flips (may be NULL):
 * flips done.  Host arrays; synchronous; device buffers by cudaMalloc, freed on return.
 * Errors: UE_ERR_ARG (sizes, ids out of range); UE_ERR_DEGENERATE (a zero-area input triangle, or a triangle inverted by
 * the relaxation: lower tau); UE_ERR_CUDA. */
int ue_mesh_relax(const double* xy, int64_t n_nodes, const int32_t* tris, int64_t n_tris,
                  const double* h_nodes, int32_t iters, int32_t flip_every, double tau,
                  const int32_t* anchors, int64_t n_anchors, const int32_t* segs, int64_t n_segs,
                  double* xy_out, int32_t* tris_out, int64_t* n_flips, void* stream);

/* The remesh step of ue_mesh_relax alone, on the host (Section 3): interior edges that are not
 * locally Delaunay (the node across one triangle's edge inside its circle, beyond a relative
 * 1e-10 margin) are flipped until none is left; boundary edges and the n_segs node-id pairs in
 * segs are kept.  xy: n_nodes*2 doubles; tris: n_tris*3 int32, either orientation; tris_out
 * (caller-owned, n_tris*3): the triangles, CCW, in the input's slots.  *n_flips (may be NULL):
 * flips done.  No GPU call.  Errors: UE_ERR_ARG (sizes, ids); UE_ERR_DEGENERATE (a zero-area
 * triangle). */
int ue_mesh_flip(const double* xy, int64_t n_nodes, const int32_t* tris, int64_t n_tris, const int32_t* segs,
                 int64_t n_segs, int32_t* tris_out, int64_t* n_flips);

/* The highest eigenmodes of the semi-discrete system (Section 2): omega_i^2 are the largest
 * eigenvalues of K = -L_E L_B in the S-weighted product, found by the "complex time" method
 * with deflation (each mode iterated while the modes above it are kept from growing back),
 * here with all columns of a block advanced together and re-orthonormalised after every
 * product, then a Rayleigh-Ritz step.  The block holds min(32, 2 n_modes) columns; modes
 * beyond n_modes only guard the convergence of the ones returned.  FP64; the error of omega_i
 * falls like (omega_{m+1} / omega_i)^(4 iters).
 * n_modes in [1, 24], iters >= 1, seed: start vectors (SplitMix64 of the caller triangle id and
 * column).  omega: n_modes doubles, descending.  B: NULL or n_modes * n_tris doubles, mode i
 * at B + i*n_tris in caller triangle order, normalised to sum_j S_j B_j^2 = 1 (sign
 * arbitrary).  Synchronous; the work space, about (2 n_tris + n_interior_edges) * 2 n_modes
 * doubles, comes from the mesh's allocator and is returned.
 * Errors: UE_ERR_ARG (also on a mesh with a PML frame); UE_ERR_ALLOC; UE_ERR_DUAL if the block
 * loses rank; UE_ERR_CUDA. */
int ue_modes(ue_mesh* m, int32_t n_modes, int32_t iters, uint32_t seed, double* omega, double* B,
             void* stream);

/* The lowest eigenmodes (the other end of the spectrum of Section 2, which Fig. 4 plots against
 * the analytic resonator frequencies): omega[0..n_modes) ascending (omega[0] = 0 for the
 * static field B = constant of a PEC cavity) and, if B is not NULL, their B fields (n_modes x
 * n_tris, caller order, S-normalised).  Chebyshev-filtered subspace iteration on a block of
 * min(32, 2 n_modes) columns: each of at most `iters` filters is the degree-`degree` Chebyshev
 * polynomial of K that stays within [-1, 1] on [lo, hi] (hi a Gershgorin bound of the largest
 * eigenvalue, lo the block's largest Ritz value) and grows below lo, followed by Cholesky QR in
 * the S metric and Rayleigh-Ritz; it stops early when the n_modes Ritz values no longer move.
 * FP64, synchronous.  n_modes in [1, 16], degree in [2, 200].  Errors as ue_modes. */
int ue_modes_low(ue_mesh* m, int32_t n_modes, int32_t iters, int32_t degree, uint32_t seed, double* omega,
                 double* B, void* stream);

/* Open boundaries: a PML frame (the paper's conclusion: a mesh with a rectangular boundary tied
 * to a structured frame of rectangular cells carrying PML layers).  The frame is `width` square
 * cells of side h around the mesh's bounding box [X0, X1] x [Y0, Y1], h being the spacing of
 * the mesh's outer boundary nodes, which must be uniform and the same on all four sides (the
 * box a whole number nx x ny of them); holes stay PEC.  Cells carry B at their centres, E lives
 * on their sides (Yee); the mesh's 2 nx + 2 ny outer edges become unknowns coupling a triangle
 * and a frame cell, with dual length d = (O_tri - C_e) . n_in + h/2 (eq. 3; the two centres on
 * the edge's perpendicular bisector).  The frame's own outer boundary is PEC.
 * PML: Berenger's split field B = Bx + By in every frame cell, Bx fed by the cell's vertical
 * sides and decaying at sigma_x(x), By by its horizontal sides at sigma_y(y); E on horizontal
 * sides decays at sigma_y, on vertical sides at sigma_x; sigma(delta) = sigma_max
 * (delta / (width h))^order, delta the distance beyond the box along that axis, taken at the
 * field's position; the decay is trapezoidal in time.  sigma_max < 0 selects
 * (order + 1) ln(1e6) / (2 width h) (a continuous layer reflecting 1e-6 at normal incidence);
 * 0 gives an undamped frame.
 * Host call on a loaded mesh; it takes effect at the next ue_geometry_build (width 0 removes
 * the frame).  A framed mesh steps with UE_VARIANT_PLAIN or, on a tiled mesh, UE_VARIANT_BLOCKED:
 * the tiles whose block_depth rings stay off the outer edges run in the blocked kernel, the
 * others form one region advanced block_depth steps at a time by the plain kernels together
 * with the frame (the same results, bit for bit).  dt modes UE_DT_GIVEN and UE_DT_POWER, the
 * power iteration then covering the whole framed system (eq. 20 for the coupled operator).
 * Its sources must be interior edges.  In plasma media (ue_set_plasma) the current runs on the
 * mesh's interior edges, the frame and the outer edges being vacuum.
 * ue_write_fields zeroes the frame's fields; ue_read_fields returns E on the mesh's outer
 * edges too; the energy watchdog and ue_energy cover the mesh only.
 * width in [1, 256], order in [1, 8].  Errors: UE_ERR_ARG (arguments, a batch, or an outer
 * boundary that is not a uniformly divided axis-aligned rectangle). */
int ue_frame_attach(ue_mesh* m, int32_t width, double sigma_max, int32_t order);

/* Frame layout (host): dims = {width, nx, ny, NX = nx + 2 width, NY = ny + 2 width, n_cells,
 * n_interface}, geom = {h, X0, Y0, sigma_max}.  Frame cells are numbered in strip order: the
 * `width` bottom rows (NX cells each), then per middle row the `width` cells left of the mesh
 * and the `width` right of it, then the `width` top rows; cell (I, J) of the NX x NY grid
 * covers [X0 + (I - width) h, X0 + (I - width + 1) h] x [Y0 + (J - width) h, ...].
 * Either pointer may be NULL.  UE_ERR_ARG without a frame. */
int ue_frame_get(const ue_mesh* m, int64_t* dims, double* geom);

/* The frame's interface edges (host; after ue_frame_attach): for k in [0, n_interface), in the
 * order bottom side (by x), top, left (by y), right: edge[k] = the mesh's caller edge id and
 * cell[k] = the frame cell across it (strip order).  Either pointer may be NULL.  UE_ERR_ARG
 * without a frame. */
int ue_frame_interface(const ue_mesh* m, int64_t* edge, int64_t* cell);

/* Blocked stepping of a framed tiled mesh, planned on the host for a given block_depth k:
 * counts[6] = {tiles, tiles that stay blocked (their rings H_0..H_{k-1} reach no triangle on
 * the outer edges), triangles owned by the region (the other tiles' triangles), the region's
 * local triangles (owned plus k rings), its local edges (those with a triangle within k-1
 * rings), its owned edges (those whose smaller stored triangle it owns)}.  UE_ERR_ARG without a
 * frame or tiles, or for block_depth outside 1..15. */
int ue_frame_region(const ue_mesh* m, int32_t block_depth, int64_t* counts);

/* The frame's own state for checkpoint and resume (synchronous, after ue_geometry_build):
 * Bx, By[n_cells] (strip order), Ex[NX * (NY + 1)], Ey[(NX + 1) * NY] in the layout of
 * ue_frame_fields (E = circulation / h, 0 on sides that are not frame unknowns).  write = 0
 * reads them out, write = 1 sets them (call it after ue_write_fields, which zeroes the frame;
 * the mesh's outer edges travel with ue_read_fields / ue_write_fields).  All four pointers are
 * required.  UE_ERR_ARG without a built frame. */
int ue_frame_state(ue_mesh* m, double* Bx, double* By, double* Ex, double* Ey, int32_t write, void* stream);

/* Frame fields (synchronous, after ue_geometry_build): B[n_cells] = Bx + By per frame cell in
 * strip order; Ex[NX * (NY + 1)]: E on the horizontal side at height J between columns I and
 * I + 1, at Ex[J * NX + I]; Ey[(NX + 1) * NY]: E on the vertical side at column I between rows J
 * and J + 1, at Ey[J * (NX + 1) + I]; sides along +x and +y; 0 on sides that are not frame
 * unknowns (the PEC outer wall, the mesh's outer edges, which ue_read_fields returns, and sides
 * inside the mesh).  Any pointer may be NULL. */
int ue_frame_fields(ue_mesh* m, double* B, double* Ex, double* Ey, void* stream);

/* Power iteration for rho(M) that allocates no device memory.
 * The paper has no counterpart: this exists for callers that cannot allocate device memory
 * while they run (a memory budget fixed up front, a host process that owns the allocator, or
 * code that must avoid cudaMalloc's implicit synchronisation).  It computes the same
 * S-normalised power iteration as ue_geometry_build (same SplitMix64 start vector, iteration
 * count; the reductions follow ue_geometry_build's order, but each element is divided by d and
 * S where ue_geometry_build multiplies by precomputed reciprocals, so the two agree to rounding,
 * not bit for bit), with its work vectors in one file-scope device array of 8.4 MB: at most
 * UE_STATIC_MAX_TRIS triangles and UE_STATIC_MAX_EDGES interior edges.  Larger sizes return
 * UE_ERR_ARG.
 * Device memory: under CUDA's default lazy module loading the array is placed on a device by
 * the first call there, not when the library is loaded, and stays until the process exits.  A
 * caller whose memory budget is fixed at some point makes one warm-up call on each device
 * before it (or runs with CUDA_MODULE_LOADING=EAGER).  After that, calls take no device memory.
 * Inputs are DEVICE pointers owned by the caller, in the stored numbering of ue_get_tables:
 *   edge_tri[2*n_ei] (R, L), int32, 8-byte aligned; elen[n_ei], d[n_ei] (|e| and |O_R O_L| per
 *   stored edge); tri_code[3*n_tris]; S[n_tris]; tri_caller[n_tris] (caller id of each stored
 *   triangle, which keys the start vector).  An edge_tri entry outside [0, n_tris) or a
 *   tri_code entry outside [0, 2 n_ei + 1] is not followed: the call returns UE_ERR_ARG.
 * Output: *rho (host).  Synchronous on `stream`.  All calls share the work array: calls that
 * overlap on the GPU race, so serialise them.  Every call looks up the array's device address
 * (cudaGetSymbolAddress) with the calling device current; the first call on a device also
 * loads the module there, so make it before any stream capture.  No cudaMalloc, cudaFree or
 * allocating routine is used. */
#define UE_STATIC_MAX_TRIS (1 << 18)
#define UE_STATIC_MAX_EDGES (1 << 19)
int ue_power_iteration_static(const int32_t* edge_tri, const double* elen, const double* d,
                              const int32_t* tri_code, const double* S,
                              const int64_t* tri_caller, int64_t n_tris, int64_t n_interior_edges,
                              int32_t iters, uint32_t seed, void* stream, double* rho);

int ue_stats(const ue_mesh* m, ue_stats_t* out);
const char* ue_last_error(void);
void ue_mesh_free(ue_mesh* m);

#ifdef __cplusplus
}
#endif
#endif /* UE_H */
