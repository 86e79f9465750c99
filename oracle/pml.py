"""A structured PML frame tied to a triangle mesh (oracle; test infrastructure only).

The paper's conclusion proposes open boundaries for meshes with a rectangular outer boundary: a
frame of rectangular cells around the mesh carries PML layers, the scheme working unchanged on
the mixed triangle + quad mesh.  It prints no formulas for it; the readings here are:

* the frame: square cells of side h, h being the spacing of the mesh's outer boundary nodes (the
  same on all four sides of its bounding box [X0, X1] x [Y0, Y1]), ``width`` cells thick; cell
  (I, J) of the grid of NX x NY cells covers [X0 + (I - W) h, ...] x [Y0 + (J - W) h, ...], the
  cells inside the bounding box being the mesh; the frame's own outer boundary is PEC (E = 0);
* a square's centre is its circumcentre, so every frame side has the dual length of eq. 3 like a
  triangle edge: d = h between two frame cells; on the mesh's outer boundary the two centres sit
  on the side's perpendicular bisector, d = (O_tri - C_e) . n_in + h / 2 (n_in the unit normal
  into the mesh, C_e the side's midpoint);
* frame sides are directed along +x (horizontal) and +y (vertical); the mesh's outer edges keep
  the mesh's direction (low to high node id) and become unknowns;
* PML (Berenger's split field): every frame cell carries B = Bx + By; Bx takes the circulation
  of the cell's two vertical sides and decays at sigma_x(x), By that of its horizontal sides and
  decays at sigma_y(y); E on a horizontal side decays at sigma_y, on a vertical side at sigma_x;
  each sigma is taken at the field's own position;
* sigma(delta) = sigma_max (delta / (W h))^order, delta the distance beyond the bounding box along
  that axis (0 inside it); default sigma_max = (order + 1) ln(1 / R0) / (2 W h), R0 = 1e-6, the
  normal-incidence reflection of the continuous layer;
* decay terms trapezoidal in time, as for the collision term:
  E+ = ((1 - s dt/2) E + dt (L_B B)) / (1 + s dt/2), and the same form for Bx, By.

Unknown order: the inner system's edges, then the 2 nx + 2 ny interface edges (bottom side, top,
left, right; along +x or +y), then the frame sides (horizontal sides row by row, then vertical).
Cells: the inner system's cells, then the frame cells in strip order (the W bottom rows, then per
middle row the W cells left of the mesh and the W right of it, then the W top rows).  The split
state is [inner cells, Bx of the frame cells, By of the frame cells].

With plasma (``step_plasma``) the current of eqs. 5-6 runs on the mesh's interior edges only; the
mesh's outer edges and the frame are vacuum.

Parity: pinned by tests/test_oracle_pml.py (Yee's closed form for every mode of a right-split
lattice framed with sigma = 0, adjointness of the combined operators, exact conservation of the
staggered energy at sigma = 0, and a pulse that stays within 5e-4 of the same mesh in a large
undamped frame until that frame's echo returns, while a layer whose Bx and By decay rates are
swapped is more than 20 times worse).  A PML absorbs travelling waves only: the static charge
its anisotropic decay leaves behind (div E is not kept inside the layer) and the zero-frequency
part of a field stay, so the pins compare fields, not the energy left.  The plasma step is
pinned by the static field: a discrete gradient of a node potential that vanishes on the
boundary never reaches the frame, and with a uniform density n0 and nu = 0 it obeys
E^{n+1} + E^{n-1} = (2 - n0 dt^2) E^n exactly while B stays 0.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .geometry import Geometry
from .mesh import Mesh
from .operators import Operators


def default_sigma_max(h: float, width: int, order: int, r0: float = 1e-6) -> float:
    return (order + 1) * math.log(1.0 / r0) / (2.0 * width * h)


def sigma_profile(delta, h: float, width: int, sigma_max: float, order: int):
    return sigma_max * (np.asarray(delta, np.float64) / (width * h)) ** order


class FramedOperators:
    """Mesh (or merged cells) + PML frame; L_B, L_E (cells), w_E, w_B like ``Operators``."""

    def __init__(self, mesh: Mesh, width: int, sigma_max: float | None = None, order: int = 3,
                 geom: Geometry | None = None, inner=None, tol: float = 1e-9):
        geom = geom if geom is not None else Geometry(mesh)
        inner = inner if inner is not None else Operators(mesh, geom)
        cell_of_tri = getattr(inner, "cell_of_tri", np.arange(mesh.n_tris))
        self.inner = inner
        W = int(width)
        xy = mesh.xy
        X0, X1 = xy[:, 0].min(), xy[:, 0].max()
        Y0, Y1 = xy[:, 1].min(), xy[:, 1].max()
        # outer boundary edges: one triangle, both ends on the same side of the bounding box
        bnd = np.nonzero(~mesh.interior)[0]
        side_edges = {s: [] for s in "btlr"}
        for e in bnd:
            (xa, ya), (xb, yb) = xy[mesh.edges[e, 0]], xy[mesh.edges[e, 1]]
            span = max(X1 - X0, Y1 - Y0)
            on = lambda u, v: abs(u - v) <= tol * span
            if on(ya, Y0) and on(yb, Y0):
                side_edges["b"].append(e)
            elif on(ya, Y1) and on(yb, Y1):
                side_edges["t"].append(e)
            elif on(xa, X0) and on(xb, X0):
                side_edges["l"].append(e)
            elif on(xa, X1) and on(xb, X1):
                side_edges["r"].append(e)
        if any(len(v) == 0 for v in side_edges.values()):
            raise ValueError("outer boundary is not an axis-aligned rectangle")
        h = float(np.median(geom.elen[np.concatenate([np.asarray(v, np.int64) for v in side_edges.values()])]))
        nx = int(round((X1 - X0) / h))
        ny = int(round((Y1 - Y0) / h))
        if abs(nx * h - (X1 - X0)) > tol * nx * h or abs(ny * h - (Y1 - Y0)) > tol * ny * h:
            raise ValueError("bounding box is not a whole number of boundary spacings")
        if len(side_edges["b"]) != nx or len(side_edges["t"]) != nx or \
                len(side_edges["l"]) != ny or len(side_edges["r"]) != ny:
            raise ValueError("outer boundary nodes are not uniformly spaced")
        for s in "btlr":     # every outer node on the grid X0 + i h (Y0 + j h)
            for e in side_edges[s]:
                for v in mesh.edges[e]:
                    u = (xy[v, 0] - X0) if s in "bt" else (xy[v, 1] - Y0)
                    if abs(u / h - round(u / h)) > 1e-6:
                        raise ValueError("outer boundary nodes are not uniformly spaced")
        self.h, self.W, self.nx, self.ny = h, W, nx, ny
        NX, NY = nx + 2 * W, ny + 2 * W
        self.NX, self.NY = NX, NY
        if sigma_max is None:
            sigma_max = default_sigma_max(h, W, order)
        self.sigma_max, self.order = sigma_max, order

        # frame cells in strip order
        cells = [(I, J) for J in range(W) for I in range(NX)]
        cells += [(I, J) for J in range(W, W + ny) for I in list(range(W)) + list(range(W + nx, NX))]
        cells += [(I, J) for J in range(W + ny, NY) for I in range(NX)]
        self.frame_cells = cells
        n_fc = len(cells)
        cid = {c: k for k, c in enumerate(cells)}
        n_in = inner.L_B.shape[1]
        self.n_in, self.n_fc = n_in, n_fc
        self.n_c = n_in + n_fc
        xg = lambda I: X0 + (I - W) * h          # grid line x of column I
        yg = lambda J: Y0 + (J - W) * h

        def delta_x(x):
            return max(0.0, X0 - x, x - X1)

        def delta_y(y):
            return max(0.0, Y0 - y, y - Y1)

        sig = lambda d: float(sigma_profile(d, h, W, sigma_max, order))

        # --- edges
        rows_B, cols_B, vals_B = [], [], []        # L_B entries (edge, cell, value)
        w_E, sigE = [], []
        n_ie = inner.n_ei
        LBi = inner.L_B.tocoo()
        rows_B += LBi.row.tolist()
        cols_B += LBi.col.tolist()
        vals_B += LBi.data.tolist()
        w_E += list(inner.w_E)
        sigE += [0.0] * n_ie
        # interface edges: (edge row, triangle cell, frame cell, triangle is R, |e|) per side
        iface = []
        n_in_dir = {"b": (0.0, 1.0), "t": (0.0, -1.0), "l": (1.0, 0.0), "r": (-1.0, 0.0)}
        for s in "btlr":
            def pos(e):
                a, b = xy[mesh.edges[e, 0]], xy[mesh.edges[e, 1]]
                m = 0.5 * (a + b)
                return m[0] if s in "bt" else m[1]
            for e in sorted(side_edges[s], key=pos):
                a, b = xy[mesh.edges[e, 0]], xy[mesh.edges[e, 1]]
                C = 0.5 * (a + b)
                if s in "bt":
                    I = W + int(math.floor((C[0] - X0) / h))
                    fc = (I, W - 1) if s == "b" else (I, W + ny)
                else:
                    J = W + int(math.floor((C[1] - Y0) / h))
                    fc = (W - 1, J) if s == "l" else (W + nx, J)
                t = mesh.R[e] if mesh.R[e] >= 0 else mesh.L[e]
                tri_is_R = bool(mesh.R[e] >= 0)
                nin = np.array(n_in_dir[s])
                d = float(np.dot(geom.O[t] - C, nin) + 0.5 * h)
                if not d > 0:
                    raise ValueError("non-positive dual length at the frame")
                iface.append((e, int(cell_of_tri[t]), n_in + cid[fc], tri_is_R, float(geom.elen[e]), d, s, fc))
        self.iface = iface
        self.n_if = len(iface)
        for k, (e, tc, fcell, tri_is_R, el, d, s, fc) in enumerate(iface):
            row = n_ie + k
            R, L = (tc, fcell) if tri_is_R else (fcell, tc)
            rows_B += [row, row]
            cols_B += [R, L]
            vals_B += [1.0 / d, -1.0 / d]
            w_E.append(d * el)
            sigE.append(0.0)
        # frame sides: horizontal H(I, J) between (I, J-1) below and (I, J) above; vertical
        # V(I, J) between (I-1, J) left and (I, J) right.  A side is a frame unknown when both
        # neighbours are frame cells.
        fset = set(cells)
        self.H, self.V = {}, {}
        row = n_ie + self.n_if
        for J in range(1, NY):
            for I in range(NX):
                if (I, J - 1) in fset and (I, J) in fset:
                    self.H[(I, J)] = row
                    rows_B += [row, row]
                    cols_B += [n_in + cid[(I, J)], n_in + cid[(I, J - 1)]]   # R above, L below
                    vals_B += [1.0 / h, -1.0 / h]
                    w_E.append(h * h)
                    sigE.append(sig(delta_y(yg(J))))
                    row += 1
        for J in range(NY):
            for I in range(1, NX):
                if (I - 1, J) in fset and (I, J) in fset:
                    self.V[(I, J)] = row
                    rows_B += [row, row]
                    cols_B += [n_in + cid[(I - 1, J)], n_in + cid[(I, J)]]   # R left, L right
                    vals_B += [1.0 / h, -1.0 / h]
                    w_E.append(h * h)
                    sigE.append(sig(delta_x(xg(I))))
                    row += 1
        self.n_ei = row
        self.L_B = sp.csr_matrix((vals_B, (rows_B, cols_B)), shape=(self.n_ei, self.n_c))
        self.w_E = np.asarray(w_E)
        self.sigE = np.asarray(sigE)

        # --- split cells: dB/dt = -(1/S) sum_q s_q |e_q| E_q
        n_s = n_in + 2 * n_fc
        rows_E, cols_E, vals_E = [], [], []
        LEi = inner.L_E.tocoo()
        rows_E += LEi.row.tolist()
        cols_E += LEi.col.tolist()
        vals_E += LEi.data.tolist()
        S_in = np.asarray(inner.w_B)
        iface_of = {}
        for k, (e, tc, fcell, tri_is_R, el, d, s, fc) in enumerate(iface):
            # the triangle runs the edge counter-clockwise iff it is R; the frame cell the reverse
            rows_E.append(tc)
            cols_E.append(n_ie + k)
            vals_E.append(-(1.0 if tri_is_R else -1.0) * el / S_in[tc])
            iface_of[(fc, s)] = (n_ie + k, -1.0 if tri_is_R else 1.0, el)
        S_f = h * h
        sigB = [0.0] * n_s
        for c, (I, J) in enumerate(cells):
            bx, by = n_in + c, n_in + n_fc + c
            xc, yc = X0 + (I - W + 0.5) * h, Y0 + (J - W + 0.5) * h
            sigB[bx] = sig(delta_x(xc))
            sigB[by] = sig(delta_y(yc))
            # sides with their counter-clockwise sign: bottom +, right +, top -, left -
            for side, key, sgn, tgt, iside in (("H", (I, J), 1.0, by, "t"), ("V", (I + 1, J), 1.0, bx, "l"),
                                               ("H", (I, J + 1), -1.0, by, "b"), ("V", (I, J), -1.0, bx, "r")):
                # iside: the mesh side this frame side would face if it were an interface edge
                tab = self.H if side == "H" else self.V
                if key in tab:
                    rows_E.append(tgt)
                    cols_E.append(tab[key])
                    vals_E.append(-sgn * h / S_f)
                elif ((I, J), iside) in iface_of:
                    col, s_cell, el = iface_of[((I, J), iside)]
                    rows_E.append(tgt)
                    cols_E.append(col)
                    vals_E.append(-s_cell * el / S_f)
        self.Ls_E = sp.csr_matrix((vals_E, (rows_E, cols_E)), shape=(n_s, self.n_ei))
        self.sigB = np.asarray(sigB)
        pr = list(range(n_in)) + [n_in + c for c in range(n_fc)] * 2
        self.P = sp.csr_matrix((np.ones(n_s), (pr, np.arange(n_s))), shape=(self.n_c, n_s))
        self.L_E = (self.P @ self.Ls_E).tocsr()
        self.w_B = np.concatenate([S_in, np.full(n_fc, S_f)])
        self.n_s = n_s
        self.n_t = self.n_c

    def start_split(self, B_cells: np.ndarray) -> np.ndarray:
        """Split state from cell values (a frame cell's value goes to Bx, By = 0)."""
        out = np.zeros(self.n_s)
        out[:self.n_in] = B_cells[:self.n_in]
        out[self.n_in:self.n_in + self.n_fc] = B_cells[self.n_in:]
        return out


def step(fo: FramedOperators, E: np.ndarray, Bs: np.ndarray, dt: float, src=None, n: int = 0):
    """One leap-frog step with trapezoidal PML decay; src = (edge rows, amplitudes, g)."""
    aE = (1.0 - 0.5 * dt * fo.sigE) / (1.0 + 0.5 * dt * fo.sigE)
    bE = dt / (1.0 + 0.5 * dt * fo.sigE)
    E = aE * E + bE * (fo.L_B @ (fo.P @ Bs))
    if src is not None:
        rows, amp, g = src
        E[rows] += dt * amp * g((n + 0.5) * dt)
    aB = (1.0 - 0.5 * dt * fo.sigB) / (1.0 + 0.5 * dt * fo.sigB)
    bB = dt / (1.0 + 0.5 * dt * fo.sigB)
    Bs = aB * Bs + bB * (fo.Ls_E @ E)
    return E, Bs


def inner_nbar(fo: FramedOperators, n_nodes: np.ndarray) -> np.ndarray:
    """Mean density of the two end nodes of each of the mesh's interior edges (eq. 5 reading)."""
    e = fo.inner.mesh.edges[fo.inner.ie]
    return 0.5 * (n_nodes[e[:, 0]] + n_nodes[e[:, 1]])


def step_plasma(fo: FramedOperators, E, Bs, j, dt: float, nbar, nu: float, src=None, n: int = 0):
    """One framed step with the cold-plasma current of eqs. 5-6 on the mesh's interior edges,
    in the order and form of the unframed step: j at half steps, trapezoidal in nu, drains E;
    the mesh's outer edges and the frame are vacuum.  Returns (E, Bs, j)."""
    ni = fo.inner.n_ei
    j = ((1.0 - 0.5 * nu * dt) * j + dt * nbar * E[:ni]) / (1.0 + 0.5 * nu * dt)
    aE = (1.0 - 0.5 * dt * fo.sigE) / (1.0 + 0.5 * dt * fo.sigE)
    bE = dt / (1.0 + 0.5 * dt * fo.sigE)
    E = aE * E + bE * (fo.L_B @ (fo.P @ Bs))
    E[:ni] -= dt * j
    if src is not None:
        rows, amp, g = src
        E[rows] += dt * amp * g((n + 0.5) * dt)
    aB = (1.0 - 0.5 * dt * fo.sigB) / (1.0 + 0.5 * dt * fo.sigB)
    bB = dt / (1.0 + 0.5 * dt * fo.sigB)
    Bs = aB * Bs + bB * (fo.Ls_E @ E)
    return E, Bs, j


def run(fo: FramedOperators, E, Bs, dt: float, n_steps: int, src=None, n0: int = 0):
    for k in range(n_steps):
        E, Bs = step(fo, E, Bs, dt, src, n0 + k)
    return E, Bs


def energy_W(fo: FramedOperators, E: np.ndarray, Bs: np.ndarray) -> float:
    B = fo.P @ Bs
    return float(np.dot(fo.w_E, E * E) + np.dot(fo.w_B, B * B))
