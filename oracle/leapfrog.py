"""Leap-frog time stepping of eqs. 4-6 (14, 15), energies of eqs. 7-8, div E (oracle).

Test infrastructure only.  Time levels: E (and its unknown-edge vector) at integer steps
t = n dt, B and the current j at half steps t = (n + 1/2) dt.  One step from n to n+1:

1. current (plasma media, eq. 5, trapezoidal in the collision term):
       j^{n+1/2} = ((1 - nu dt/2) j^{n-1/2} + dt nbar_i E^n) / (1 + nu dt/2)
   with nbar_i the mean of the node density n over the two end nodes of edge i;
2. E (eqs. 6 and 14):  E^{n+1} = E^n + dt (L_B B^{n+1/2} - j^{n+1/2}) + dt a_i g(t_{n+1/2})
   where a_i g(t) is an optional soft source, g(t) = sin(w0 t) exp(-((t - t0)/tau)^2);
3. B (eq. 15):         B^{n+3/2} = B^{n+1/2} + dt L_E E^{n+1}.

Eq. 6 prints "+ j" with eq. 5's "dj/dt = nE"; together they give E'' = +nE, i.e. growth.  The
oracle takes the physical sign (the current drains E), which equals the printed system up to the
sign convention of j.

Parity: pinned by tests/test_oracle_invariants.py (exact conservation of the staggered energy
Q, bounded W of eq. 8, div E flux), tests/test_oracle_spectral.py (leap-frog dispersion
sin(W dt/2) = w dt/2 of eqs. 18-19, cavity TE(m,n) convergence) and tests/test_oracle_plasma.py
(closed-form plasma oscillation and collisional damping).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .operators import Operators


@dataclasses.dataclass
class Plasma:
    n_nodes: np.ndarray     # density n at every caller node (n = omega_p^2, dimensionless)
    nu: float               # collision rate

    def nbar(self, ops: Operators) -> np.ndarray:
        e = ops.mesh.edges[ops.ie]
        return 0.5 * (self.n_nodes[e[:, 0]] + self.n_nodes[e[:, 1]])


@dataclasses.dataclass
class Source:
    edge_ids: np.ndarray    # caller edge ids (interior edges)
    amp: np.ndarray         # a_i, E amplitude per edge
    omega0: float
    t0: float
    tau: float

    def g(self, t: float) -> float:
        return math.sin(self.omega0 * t) * math.exp(-((t - self.t0) / self.tau) ** 2)


@dataclasses.dataclass
class State:
    E: np.ndarray           # unknown-edge vector at t = n dt
    B: np.ndarray           # triangles at t = (n + 1/2) dt
    j: np.ndarray           # unknown edges at t = (n - 1/2) dt (zeros without plasma)
    n: int = 0              # step counter


def initial_state(ops: Operators, E_all=None, B=None, j_all=None) -> State:
    E = ops.restrict(E_all) if E_all is not None else np.zeros(ops.n_ei)
    Bv = np.asarray(B, np.float64).copy() if B is not None else np.zeros(ops.n_t)
    jv = ops.restrict(j_all) if j_all is not None else np.zeros(ops.n_ei)
    return State(E.copy(), Bv, jv.copy(), 0)


def step(ops: Operators, st: State, dt: float, plasma: Plasma | None = None,
         source: Source | None = None, nbar: np.ndarray | None = None,
         src_cols: np.ndarray | None = None) -> State:
    """Advance one leap-frog step (E from n to n+1, B from n+1/2 to n+3/2)."""
    E, B, j = st.E, st.B, st.j
    if plasma is not None:
        nb = nbar if nbar is not None else plasma.nbar(ops)
        j = ((1.0 - 0.5 * plasma.nu * dt) * j + dt * nb * E) / (1.0 + 0.5 * plasma.nu * dt)
    E = E + dt * (ops.L_B @ B - j)
    if source is not None:
        cols = src_cols if src_cols is not None else ops.col_of_edge[source.edge_ids]
        t = (st.n + 0.5) * dt
        E[cols] += dt * source.amp * source.g(t)
    B = B + dt * (ops.L_E @ E)
    return State(E, B, j, st.n + 1)


def run(ops: Operators, st: State, dt: float, n_steps: int, plasma: Plasma | None = None,
        source: Source | None = None, record=None) -> State:
    """n_steps leap-frog steps; ``record(state)`` is called after each step if given."""
    nbar = plasma.nbar(ops) if plasma is not None else None
    cols = ops.col_of_edge[source.edge_ids] if source is not None else None
    for _ in range(n_steps):
        st = step(ops, st, dt, plasma, source, nbar, cols)
        if record is not None:
            record(st)
    return st


def energy_W(ops: Operators, E: np.ndarray, B: np.ndarray) -> float:
    """Eq. 8 with the eq. 7 weights: sum d_i |e_i| E_i^2 + sum S_j B_j^2."""
    return float(np.dot(ops.w_E, E * E) + np.dot(ops.w_B, B * B))


def energy_Q(ops: Operators, E: np.ndarray, B_before: np.ndarray, B_after: np.ndarray) -> float:
    """Staggered leap-frog energy: sum w_E E^n^2 + sum S B^{n-1/2} B^{n+1/2}.

    Exactly invariant under the vacuum leap-frog step (without source or current): with
    A = W_B^{1/2} and the eq. 10 adjointness, Q^{n+1} - Q^n telescopes to zero.
    """
    return float(np.dot(ops.w_E, E * E) + np.dot(ops.w_B, B_before * B_after))


def node_flux(ops: Operators, E: np.ndarray) -> np.ndarray:
    """Flux of E out of each node's Voronoi cell: sum_i sigma_iv d_i E_i (remark after eq. 4).

    sigma_iv = +1 when edge i leaves node v (v is its low end), -1 when it arrives.
    """
    e = ops.mesh.edges[ops.ie]
    f = ops.d * E
    out = np.zeros(ops.mesh.n_nodes)
    np.add.at(out, e[:, 0], f)
    np.add.at(out, e[:, 1], -f)
    return out


def interior_nodes(ops: Operators) -> np.ndarray:
    """Nodes none of whose edges is a boundary edge."""
    mesh = ops.mesh
    on_bnd = np.zeros(mesh.n_nodes, bool)
    be = mesh.edges[~mesh.interior]
    on_bnd[be.reshape(-1)] = True
    return np.nonzero(~on_bnd)[0]
