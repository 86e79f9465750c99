"""Python binding of the C ABI: the same calls, numpy host arrays in and out.

Argument marshalling only: every step of the method runs in libue.so.  Streams are
cudaStream_t handles passed as integers (``torch.cuda.current_stream().cuda_stream``); device
memory comes from PyTorch's caching allocator when ``torch_alloc=True``, else from cudaMalloc.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native as N


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _dptr(a):
    return None if a is None else a.ctypes.data_as(N.PD)


def options(**kw) -> N.Options:
    o = N.Options()
    N.lib().ue_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class _TorchAllocator:
    """Routes the library's device allocations to torch's caching allocator."""

    def __init__(self):
        import torch
        self.torch = torch
        self.dev = torch.cuda.current_device()

        def _alloc(nbytes, stream, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.dev, stream or 0))
            except Exception:
                return None

        def _free(ptr, stream, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self.alloc = N.ALLOC_FN(_alloc)
        self.free = N.FREE_FN(_free)


class Mesh:
    """A loaded mesh (``ue_mesh``).  Methods mirror the C calls of include/ue.h."""

    def __init__(self, xy, tris, reorder: int = N.UE_REORDER_RCM, torch_alloc: bool = False,
                 tile_tris: int = 2048):
        L = N.lib()
        self._xy = np.ascontiguousarray(xy, dtype=np.float64)
        t = np.ascontiguousarray(tris, dtype=np.int32)
        if self._xy.ndim != 2 or self._xy.shape[1] != 2 or t.ndim != 2 or t.shape[1] != 3:
            raise ValueError("xy must be [n,2], tris [m,3]")
        self._allocator = _TorchAllocator() if torch_alloc else None
        h = C.c_void_p()
        o = options(reorder=reorder, tile_tris=tile_tris)
        a = self._allocator.alloc if self._allocator else N.ALLOC_FN()
        f = self._allocator.free if self._allocator else N.FREE_FN()
        N.check(L.ue_mesh_load(_dptr(self._xy), self._xy.shape[0], t.ctypes.data_as(N.PI32),
                               t.shape[0], C.byref(o), a, f, None, C.byref(h)), "ue_mesh_load")
        self._h = h
        nn, nt, ne, nei = (C.c_int64() for _ in range(4))
        N.check(L.ue_get_sizes(h, C.byref(nn), C.byref(nt), C.byref(ne), C.byref(nei)), "ue_get_sizes")
        self.n_nodes, self.n_tris, self.n_edges, self.n_ei = nn.value, nt.value, ne.value, nei.value
        self.precision = N.UE_PREC_FP32

    @classmethod
    def _wrap(cls, handle, keep=()):
        obj = cls.__new__(cls)
        obj._h = handle
        obj._keep = keep
        obj._allocator = None
        nn, nt, ne, nei = (C.c_int64() for _ in range(4))
        N.check(N.lib().ue_get_sizes(handle, C.byref(nn), C.byref(nt), C.byref(ne), C.byref(nei)),
                "ue_get_sizes")
        obj.n_nodes, obj.n_tris, obj.n_edges, obj.n_ei = nn.value, nt.value, ne.value, nei.value
        obj.precision = N.UE_PREC_FP32
        return obj

    def close(self):
        if getattr(self, "_h", None):
            N.lib().ue_mesh_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def geometry_build(self, stream=None, **opts):
        params = opts.pop("mlp_params", None)
        o = options(**opts)
        if params is not None:
            self._mlp_params = np.ascontiguousarray(params, dtype=np.float32)
            if self._mlp_params.shape != (N.UE_MLP_PARAMS,):
                raise ValueError(f"mlp_params must hold {N.UE_MLP_PARAMS} values")
            o.mlp_params = self._mlp_params.ctypes.data_as(C.c_void_p)
        self.precision = o.precision
        N.check(N.lib().ue_geometry_build(self._h, C.byref(o), _stream(stream)), "ue_geometry_build")

    def get_dt(self):
        dt, rho, src = C.c_double(), C.c_double(), C.c_int32()
        N.check(N.lib().ue_get_dt(self._h, C.byref(dt), C.byref(rho), C.byref(src)), "ue_get_dt")
        return dt.value, rho.value, src.value

    def set_plasma(self, n_nodes_density, nu: float):
        n = None if n_nodes_density is None else np.ascontiguousarray(n_nodes_density, np.float64)
        if n is not None and n.shape != (self.n_nodes,):
            raise ValueError("density must have one value per node")
        N.check(N.lib().ue_set_plasma(self._h, _dptr(n), float(nu)), "ue_set_plasma")

    def set_source(self, edge_ids, amp, omega0: float, t0: float, tau: float):
        ids = np.ascontiguousarray(edge_ids, np.int32)
        a = np.ascontiguousarray(amp, np.float64)
        if ids.shape != a.shape:
            raise ValueError("edge_ids and amp must have the same length")
        N.check(N.lib().ue_set_source(self._h, ids.ctypes.data_as(N.PI32), _dptr(a), ids.size,
                                      float(omega0), float(t0), float(tau)), "ue_set_source")

    def write_fields(self, E=None, B=None, j=None, stream=None):
        def chk(x, n):
            if x is None:
                return None
            x = np.ascontiguousarray(x, np.float64)
            if x.shape != (n,):
                raise ValueError(f"expected {n} values")
            return x
        E, B, j = chk(E, self.n_edges), chk(B, self.n_tris), chk(j, self.n_edges)
        N.check(N.lib().ue_write_fields(self._h, _dptr(E), _dptr(B), _dptr(j), _stream(stream)),
                "ue_write_fields")

    def exchange_tris(self, ids, buf, scatter: bool, stream=None):
        """B of the triangles with caller ids `ids` (int32 CUDA tensor) into `buf` (a CUDA tensor
        of the field type, scatter=False) or from it (scatter=True): ue_exchange_tris."""
        N.check(N.lib().ue_exchange_tris(self._h, C.c_void_p(ids.data_ptr()), int(ids.numel()),
                                         C.c_void_p(buf.data_ptr()), 1 if scatter else 0, _stream(stream)),
                "ue_exchange_tris")

    def write_fields_f32(self, E=None, B=None, j=None, stream=None):
        """ue_write_fields_f32: fields as float32 arrays in caller numbering."""
        def chk(x, n):
            if x is None:
                return None
            x = np.ascontiguousarray(x, np.float32)
            if x.shape != (n,):
                raise ValueError(f"expected {n} values")
            return x
        E, B, j = chk(E, self.n_edges), chk(B, self.n_tris), chk(j, self.n_edges)
        N.check(N.lib().ue_write_fields_f32(self._h, *(None if a is None else a.ctypes.data_as(C.c_void_p)
                                                       for a in (E, B, j)), _stream(stream)),
                "ue_write_fields_f32")

    def read_fields_f32(self, E=True, B=True, j=False, stream=None, out=None):
        """ue_read_fields_f32: (E, B, j) as float32 arrays in caller numbering."""
        o = out or {}
        Ea = o.get("E", np.empty(self.n_edges, np.float32)) if E else None
        Ba = o.get("B", np.empty(self.n_tris, np.float32)) if B else None
        ja = o.get("j", np.empty(self.n_edges, np.float32)) if j else None
        for a in (Ea, Ba, ja):
            if a is not None and (a.dtype != np.float32 or not a.flags.c_contiguous):
                raise ValueError("output arrays must be contiguous float32")
        N.check(N.lib().ue_read_fields_f32(self._h, *(None if a is None else a.ctypes.data_as(C.c_void_p)
                                                      for a in (Ea, Ba, ja)), _stream(stream)),
                "ue_read_fields_f32")
        return Ea, Ba, ja

    def step_n(self, n: int, stream=None):
        N.check(N.lib().ue_step_n(self._h, int(n), _stream(stream)), "ue_step_n")

    def step_prepare(self, stream=None):
        """Capture the step graphs now (ue_step_prepare), outside any timed or latency-bound call."""
        N.check(N.lib().ue_step_prepare(self._h, _stream(stream)), "ue_step_prepare")

    def read_fields(self, E=True, B=True, j=False, stream=None, out=None):
        """Return (E, B, j) as float64 arrays in caller numbering (None where not asked)."""
        o = out or {}
        Ea = o.get("E", np.empty(self.n_edges)) if E else None
        Ba = o.get("B", np.empty(self.n_tris)) if B else None
        ja = o.get("j", np.empty(self.n_edges)) if j else None
        N.check(N.lib().ue_read_fields(self._h, _dptr(Ea), _dptr(Ba), _dptr(ja), _stream(stream)),
                "ue_read_fields")
        return Ea, Ba, ja

    def energy(self, stream=None) -> float:
        w = C.c_double()
        N.check(N.lib().ue_energy(self._h, C.byref(w), _stream(stream)), "ue_energy")
        return w.value

    def check(self):
        """(ok, energy at last check, flag); ok is False when the watchdog flagged the run
        (flag 1 or 2) or a grid barrier of the persistent variant timed out (flag 3)."""
        w, f = C.c_double(), C.c_int32()
        rc = N.lib().ue_check(self._h, C.byref(w), C.byref(f))
        if rc not in (0, -7, -8):
            N.check(rc, "ue_check")
        return rc == 0, w.value, f.value

    def get_step(self) -> int:
        v = C.c_int64()
        N.check(N.lib().ue_get_step(self._h, C.byref(v)), "ue_get_step")
        return v.value

    def set_step(self, step: int):
        N.check(N.lib().ue_set_step(self._h, int(step)), "ue_set_step")

    def tables(self):
        perm = np.empty(self.n_tris, np.int64)
        ec = np.empty(self.n_ei, np.int64)
        et = np.empty((self.n_ei, 2), np.int32)
        tc = np.empty((self.n_tris, 3), np.int32)
        N.check(N.lib().ue_get_tables(self._h, perm.ctypes.data_as(N.PI64), ec.ctypes.data_as(N.PI64),
                                      et.ctypes.data_as(N.PI32), tc.ctypes.data_as(N.PI32)),
                "ue_get_tables")
        return dict(perm_tri=perm, edge_caller=ec, edge_tri=et, tri_code=tc, n_ei=self.n_ei)

    def frame_attach(self, width: int, sigma_max: float = -1.0, order: int = 3):
        """PML frame of ``width`` square cells around the rectangular outer boundary
        (ue_frame_attach); takes effect at the next geometry_build.  width 0 removes it."""
        N.check(N.lib().ue_frame_attach(self._h, int(width), float(sigma_max), int(order)),
                "ue_frame_attach")

    def frame_info(self):
        """dict(W, nx, ny, NX, NY, n_cells, n_interface, h, X0, Y0, sigma_max)."""
        d = np.zeros(7, np.int64)
        g = np.zeros(4)
        N.check(N.lib().ue_frame_get(self._h, d.ctypes.data_as(N.PI64), _dptr(g)), "ue_frame_get")
        keys = ("W", "nx", "ny", "NX", "NY", "n_cells", "n_interface")
        out = {k: int(v) for k, v in zip(keys, d)}
        out.update(h=float(g[0]), X0=float(g[1]), Y0=float(g[2]), sigma_max=float(g[3]))
        return out

    def frame_interface(self):
        """(caller edge id, frame cell) per interface edge, in the frame's order."""
        n = self.frame_info()["n_interface"]
        e = np.empty(n, np.int64)
        c = np.empty(n, np.int64)
        N.check(N.lib().ue_frame_interface(self._h, e.ctypes.data_as(N.PI64), c.ctypes.data_as(N.PI64)),
                "ue_frame_interface")
        return e, c

    def frame_region(self, block_depth: int):
        """Host plan of blocked stepping with the frame (ue_frame_region): dict of counts."""
        c = np.zeros(6, np.int64)
        N.check(N.lib().ue_frame_region(self._h, int(block_depth), c.ctypes.data_as(N.PI64)),
                "ue_frame_region")
        keys = ("tiles", "blocked_tiles", "region_owned_tris", "region_tris", "region_edges",
                "region_owned_edges")
        return {k: int(v) for k, v in zip(keys, c)}

    def frame_state(self, state=None, stream=None):
        """Without `state`: the frame's (Bx, By, Ex, Ey) for a checkpoint.  With it: set them
        (after write_fields, which zeroes the frame) (ue_frame_state)."""
        f = self.frame_info()
        if state is None:
            Bx, By = np.empty(f["n_cells"]), np.empty(f["n_cells"])
            Ex, Ey = np.empty((f["NY"] + 1, f["NX"])), np.empty((f["NY"], f["NX"] + 1))
            N.check(N.lib().ue_frame_state(self._h, _dptr(Bx), _dptr(By), _dptr(Ex), _dptr(Ey), 0,
                                           _stream(stream)), "ue_frame_state")
            return Bx, By, Ex, Ey
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in state]
        N.check(N.lib().ue_frame_state(self._h, *(_dptr(a) for a in arrs), 1, _stream(stream)),
                "ue_frame_state")

    def frame_fields(self, stream=None):
        """(B per frame cell in strip order, Ex [NY+1, NX], Ey [NY, NX+1]) (ue_frame_fields)."""
        f = self.frame_info()
        B = np.empty(f["n_cells"])
        Ex = np.empty((f["NY"] + 1, f["NX"]))
        Ey = np.empty((f["NY"], f["NX"] + 1))
        N.check(N.lib().ue_frame_fields(self._h, _dptr(B), _dptr(Ex), _dptr(Ey), _stream(stream)),
                "ue_frame_fields")
        return B, Ex, Ey

    def tiles(self):
        """Tile offsets [n_tiles + 1] of a KD or greedy mesh (empty for other orders)."""
        n = C.c_int64(0)
        N.check(N.lib().ue_get_tiles(self._h, C.byref(n), None), "ue_get_tiles")
        off = np.zeros(n.value + 1 if n.value else 0, np.int64)
        if n.value:
            N.check(N.lib().ue_get_tiles(self._h, C.byref(n), off.ctypes.data_as(N.PI64)), "ue_get_tiles")
        return off

    def geometry(self):
        O = np.empty((self.n_tris, 2))
        S = np.empty(self.n_tris)
        le = np.empty(self.n_edges)
        d = np.empty(self.n_edges)
        N.check(N.lib().ue_get_geometry(self._h, _dptr(O), _dptr(S), _dptr(le), _dptr(d)),
                "ue_get_geometry")
        return dict(O=O, S=S, elen=le, d=d)

    def rho_features(self, X, base, stream=None):
        """Learned-rho features (ue_rho_features) into CUDA tensors X [n_tris, 12] float32 and
        base [n_tris] float32 (log sqrt K_jj), stored triangle order."""
        N.check(N.lib().ue_rho_features(self._h, C.c_void_p(X.data_ptr()), C.c_void_p(base.data_ptr()),
                                        _stream(stream)), "ue_rho_features")

    def profile_steps(self, n: int, stream=None):
        """Mean per-kernel device time (ms) and algorithmic bytes per launch, n plain steps."""
        ms = np.zeros(3)
        by = np.zeros(3)
        N.check(N.lib().ue_profile_steps(self._h, int(n), _stream(stream), _dptr(ms), _dptr(by)),
                "ue_profile_steps")
        return ms, by

    def modes(self, n_modes: int, iters: int = 1000, seed: int = 0, vectors: bool = False, stream=None):
        """The n_modes highest modes (ue_modes): omegas in descending order, and with
        vectors=True their B fields (n_modes x n_tris, caller order, S-normalised)."""
        om = np.zeros(int(n_modes))
        B = np.zeros((int(n_modes), self.n_tris)) if vectors else None
        N.check(N.lib().ue_modes(self._h, int(n_modes), int(iters), int(seed) & 0xFFFFFFFF, _dptr(om),
                                 _dptr(B), _stream(stream)), "ue_modes")
        return (om, B) if vectors else om

    def modes_low(self, n_modes: int, iters: int = 200, degree: int = 24, seed: int = 0, vectors: bool = False,
                  stream=None):
        """The n_modes lowest modes (ue_modes_low): omegas ascending, and with vectors=True their
        B fields (n_modes x n_tris, caller order, S-normalised)."""
        om = np.zeros(int(n_modes))
        B = np.zeros((int(n_modes), self.n_tris)) if vectors else None
        N.check(N.lib().ue_modes_low(self._h, int(n_modes), int(iters), int(degree), int(seed) & 0xFFFFFFFF,
                                     _dptr(om), _dptr(B), _stream(stream)), "ue_modes_low")
        return (om, B) if vectors else om

    def stats(self) -> dict:
        s = N.Stats()
        N.check(N.lib().ue_stats(self._h, C.byref(s)), "ue_stats")
        return {k: getattr(s, k) for k, _ in N.Stats._fields_}


def power_iteration_static(edge_tri, elen, d, tri_code, S, tri_caller, iters: int = 200,
                           seed: int = 0, stream=None) -> float:
    """rho(M) by power iteration without any device allocation (ue_power_iteration_static).

    For callers that cannot allocate device memory while they run.  Arguments are CUDA
    tensors in the stored numbering (see ``Mesh.tables``): edge_tri int32 [n_ei, 2], elen and
    d float64 [n_ei], tri_code int32 [n_tris, 3], S float64 [n_tris], tri_caller int64
    [n_tris].  Sizes are limited to UE_STATIC_MAX_TRIS / UE_STATIC_MAX_EDGES.  Type, shape,
    device, contiguity and alignment are checked here (ValueError); indices that leave the
    arrays are refused by the library (UEError, UE_ERR_ARG).
    """
    import torch
    n_t = int(S.shape[0]) if getattr(S, "ndim", 0) == 1 else -1
    n_ei = int(elen.shape[0]) if getattr(elen, "ndim", 0) == 1 else -1
    want = (("edge_tri", edge_tri, torch.int32, (n_ei, 2)), ("elen", elen, torch.float64, (n_ei,)),
            ("d", d, torch.float64, (n_ei,)), ("tri_code", tri_code, torch.int32, (n_t, 3)),
            ("S", S, torch.float64, (n_t,)), ("tri_caller", tri_caller, torch.int64, (n_t,)))
    for name, x, dtype, shape in want:
        if not isinstance(x, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if x.dtype != dtype or tuple(x.shape) != shape:
            raise ValueError(f"{name} must be {dtype} of shape {shape}, got {x.dtype} {tuple(x.shape)}")
        if not x.is_contiguous() or x.data_ptr() % 8:
            raise ValueError(f"{name} must be contiguous and 8-byte aligned")
    for name, x, _, _ in want:
        if not x.is_cuda or x.device != S.device:
            raise ValueError(f"{name} must be a CUDA tensor on the device of S")
    rho = C.c_double()
    N.check(N.lib().ue_power_iteration_static(
        C.c_void_p(edge_tri.data_ptr()), C.c_void_p(elen.data_ptr()), C.c_void_p(d.data_ptr()),
        C.c_void_p(tri_code.data_ptr()), C.c_void_p(S.data_ptr()), C.c_void_p(tri_caller.data_ptr()),
        n_t, n_ei, int(iters), int(seed), _stream(stream), C.byref(rho)), "ue_power_iteration_static")
    return rho.value


def _pairs(segs):
    return np.ascontiguousarray(np.zeros((0, 2)) if segs is None else segs, np.int32).reshape(-1, 2)


def mesh_relax(xy, tris, iters: int, flip_every: int = 20, tau: float = 0.05, h_nodes=None,
               anchors=None, keep=None, stream=None):
    """Jello-model relaxation with Lawson flips (ue_mesh_relax): (xy, tris CCW, flips).
    anchors: node ids held in place besides the boundary; keep: node-id pairs never flipped."""
    xy = np.ascontiguousarray(xy, np.float64)
    tris = np.ascontiguousarray(tris, np.int32)
    h = None if h_nodes is None else np.ascontiguousarray(h_nodes, np.float64)
    an = np.ascontiguousarray(np.zeros(0) if anchors is None else anchors, np.int32).reshape(-1)
    kp = _pairs(keep)
    if xy.ndim != 2 or xy.shape[1] != 2 or tris.ndim != 2 or tris.shape[1] != 3:
        raise ValueError("xy must be (n, 2) and tris (m, 3)")
    if h is not None and h.shape != (xy.shape[0],):
        raise ValueError("h_nodes must hold one size per node")
    xo = np.empty_like(xy)
    to = np.empty_like(tris)
    nf = C.c_int64()
    N.check(N.lib().ue_mesh_relax(_dptr(xy), xy.shape[0], tris.ctypes.data_as(N.PI32), tris.shape[0],
                                  _dptr(h), int(iters), int(flip_every), float(tau),
                                  an.ctypes.data_as(N.PI32), an.shape[0], kp.ctypes.data_as(N.PI32),
                                  kp.shape[0], _dptr(xo),
                                  to.ctypes.data_as(N.PI32), C.byref(nf), _stream(stream)), "ue_mesh_relax")
    return xo, to, nf.value


def mesh_flip(xy, tris, keep=None):
    """Lawson flips of a triangulation on the host, keeping node-id pairs (ue_mesh_flip):
    (tris CCW, flips)."""
    xy = np.ascontiguousarray(xy, np.float64)
    tris = np.ascontiguousarray(tris, np.int32)
    if xy.ndim != 2 or xy.shape[1] != 2 or tris.ndim != 2 or tris.shape[1] != 3:
        raise ValueError("xy must be (n, 2) and tris (m, 3)")
    kp = _pairs(keep)
    out = np.empty_like(tris)
    nf = C.c_int64()
    N.check(N.lib().ue_mesh_flip(_dptr(xy), xy.shape[0], tris.ctypes.data_as(N.PI32), tris.shape[0],
                                 kp.ctypes.data_as(N.PI32), kp.shape[0], out.ctypes.data_as(N.PI32),
                                 C.byref(nf)), "ue_mesh_flip")
    return out, nf.value


def triangulate(xy, segs=None, holes=None, drop_exterior: bool = False):
    """Constrained Delaunay triangulation of a node cloud (ue_triangulate): (tris CCW, flips)."""
    xy = np.ascontiguousarray(xy, np.float64)
    if xy.ndim != 2 or xy.shape[1] != 2:
        raise ValueError("xy must be (n, 2)")
    sg = _pairs(segs)
    ho = np.ascontiguousarray(np.zeros((0, 2)) if holes is None else holes, np.float64).reshape(-1, 2)
    cap = 2 * xy.shape[0]
    out = np.empty((cap, 3), np.int32)
    nt = C.c_int64()
    nf = C.c_int64()
    N.check(N.lib().ue_triangulate(_dptr(xy), xy.shape[0], sg.ctypes.data_as(N.PI32), sg.shape[0],
                                   _dptr(ho), ho.shape[0], 1 if drop_exterior else 0,
                                   out.ctypes.data_as(N.PI32), cap, C.byref(nt), C.byref(nf)), "ue_triangulate")
    return out[:nt.value].copy(), nf.value


def batch_create(meshes, stream=None) -> Mesh:
    """ue_batch_create: one Mesh object advancing all the given built meshes together.

    Its caller numbering is the mesh-major concatenation of the meshes' nodes, triangles and
    edges; each mesh keeps its own dt and source."""
    arr = (C.c_void_p * len(meshes))(*[m._h.value if isinstance(m._h, C.c_void_p) else m._h
                                      for m in meshes])
    h = C.c_void_p()
    N.check(N.lib().ue_batch_create(arr, len(meshes), _stream(stream), C.byref(h)), "ue_batch_create")
    b = Mesh._wrap(h, keep=tuple(meshes))
    b.precision = meshes[0].precision
    return b


def _p(t):
    return C.c_void_p(t.data_ptr())


def mlp_forward(params, X, z, bf16: bool = True, stream=None):
    """z[i] = MLP(X[i]) on the device (ue_mlp_forward); CUDA tensors."""
    N.check(N.lib().ue_mlp_forward(_p(params), _p(X), int(X.shape[0]), int(bool(bf16)), _p(z),
                                   _stream(stream)), "ue_mlp_forward")


def mlp_backward(params, X, rows, dz, grad, work, bf16: bool = True, stream=None):
    """grad = sum_i dz[i] d z(X[rows[i]]) / d params (ue_mlp_backward); CUDA tensors."""
    N.check(N.lib().ue_mlp_backward(_p(params), _p(X), _p(rows), _p(dz), int(rows.shape[0]),
                                    int(bool(bf16)), _p(work), _p(grad), _stream(stream)),
            "ue_mlp_backward")


def adam(params, grad, m1, m2, t: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
         eps: float = 1e-8, stream=None):
    N.check(N.lib().ue_adam(_p(params), _p(grad), _p(m1), _p(m2), int(params.shape[0]), lr, beta1,
                            beta2, eps, int(t), _stream(stream)), "ue_adam")


def seg_argmax(z, base, off, best, arg, stream=None):
    N.check(N.lib().ue_seg_argmax(_p(z), _p(base), _p(off), int(off.shape[0] - 1), _p(best), _p(arg),
                                  _stream(stream)), "ue_seg_argmax")


def rho_loss(best, target, dz, loss, stream=None):
    N.check(N.lib().ue_rho_loss(_p(best), _p(target), int(best.shape[0]), _p(dz), _p(loss),
                                _stream(stream)), "ue_rho_loss")
