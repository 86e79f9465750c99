"""Planted mistakes in copies of the oracle (CPU only): each plausible slip must fail the pin
that guards it, so that the pins are known to see it.  The oracle itself is not modified: the
mutant is compiled from its source with one textual change."""
import inspect
import math
import textwrap

import numpy as np
import pytest

import meshgen
from oracle import mesh as om, operators, pml, rcm, spectral


def _mutant(obj, old: str, new: str):
    """obj (function or class) recompiled from its source with `old` replaced by `new`."""
    src = textwrap.dedent(inspect.getsource(obj))
    assert src.count(old) == 1, old
    ns = dict(vars(inspect.getmodule(obj)))
    exec(compile(src.replace(old, new), f"<mutant of {obj.__name__}>", "exec"), ns)
    return ns[obj.__name__]


def test_greedy_small_part_join_is_pinned():
    """Dropping the join of small parts leaves the strip's 2-triangle tail as its own part."""
    bad = _mutant(rcm.greedy_order, "if size[pid] == 0 or size[pid] >= theta:",
                  "if True:")
    ms = meshgen.right_split_lattice(30, 2, 29.0, 1.0)
    m = om.canonicalize(ms.xy, ms.tris)
    order, offs = bad(m, rcm.rcm_order(m), 32)
    assert offs.tolist() != [0, 28, 58]


def _yee_error(cls):
    h, nx, ny = 0.125, 9, 7
    ms = meshgen.right_split_lattice(nx, ny, (nx - 1) * h, (ny - 1) * h)
    m = om.canonicalize(ms.xy, ms.tris)
    fo = cls(m, 3, sigma_max=0.0, inner=operators.MergedOperators(m))
    lam = np.sort(np.linalg.eigvalsh(spectral.symmetric_K(fo)))
    M, N = np.meshgrid(np.arange(fo.NX), np.arange(fo.NY))
    yee = np.sort(((4 / h ** 2) * (np.sin(M * np.pi / (2 * fo.NX)) ** 2
                                   + np.sin(N * np.pi / (2 * fo.NY)) ** 2)).ravel())
    return np.abs(lam - yee).max() / yee.max()


def test_frame_interface_dual_length_is_pinned():
    """The interface edge's dual length with the frame cell's half counted twice
    (d = (O - C) . n + h) breaks Yee's closed form for the framed lattice."""
    assert _yee_error(pml.FramedOperators) < 1e-12
    bad = _mutant(pml.FramedOperators, "d = float(np.dot(geom.O[t] - C, nin) + 0.5 * h)",
                  "d = float(np.dot(geom.O[t] - C, nin) + 1.0 * h)")
    assert _yee_error(bad) > 1e-3


def test_frame_interface_sign_is_pinned():
    """The frame cell taking the triangle's orientation sign for the shared edge (instead of
    the opposite one) breaks the adjointness of the coupled operators."""
    bad = _mutant(pml.FramedOperators, "iface_of[(fc, s)] = (n_ie + k, -1.0 if tri_is_R else 1.0, el)",
                  "iface_of[(fc, s)] = (n_ie + k, 1.0 if tri_is_R else -1.0, el)")
    ms = meshgen.graded_square(1 / 16, 1 / 16, grade=0.0, seed=5)
    m = om.canonicalize(ms.xy, ms.tris)
    for cls, ok in ((pml.FramedOperators, True), (bad, False)):
        fo = cls(m, 4, sigma_max=0.0)
        LB, LE = fo.L_B.toarray(), fo.L_E.toarray()
        adj = np.abs(fo.w_E[:, None] * LB + (fo.w_B[:, None] * LE).T).max() / np.abs(LB).max()
        assert (adj < 1e-12) == ok


def test_framed_plasma_drain_sign_is_pinned():
    """A current that feeds E instead of draining it breaks the static-field closed form."""
    bad = _mutant(pml.step_plasma, "E[:ni] -= dt * j", "E[:ni] += dt * j")
    ms = meshgen.graded_square(1 / 16, 1 / 16, grade=0.0, seed=5)
    m = om.canonicalize(ms.xy, ms.tris)
    fo = pml.FramedOperators(m, 4)
    rng = np.random.default_rng(6)
    bnd = np.zeros(m.n_nodes, bool)
    bnd[m.edges[~m.interior].ravel()] = True
    phi = np.where(bnd, 0.0, rng.standard_normal(m.n_nodes))
    e = m.edges[fo.inner.ie]
    E0 = np.zeros(fo.n_ei)
    E0[:fo.inner.n_ei] = (phi[e[:, 1]] - phi[e[:, 0]]) / fo.inner.elen
    n0 = 3.0e3
    rho, _ = spectral.power_iteration(fo, 300)
    dt = 0.5 * 2.0 / math.sqrt(rho * rho + n0)
    nbar = pml.inner_nbar(fo, np.full(m.n_nodes, n0))

    def resid(step):
        E, Bs, j = E0.copy(), np.zeros(fo.n_s), np.zeros(fo.inner.n_ei)
        hist = [E.copy()]
        for k in range(20):
            E, Bs, j = step(fo, E, Bs, j, dt, nbar, 0.0, n=k)
            hist.append(E.copy())
        H = np.asarray(hist)
        return np.abs(H[2:] + H[:-2] - (2.0 - n0 * dt * dt) * H[1:-1]).max() / np.abs(H).max()

    assert resid(pml.step_plasma) < 1e-12
    assert resid(bad) > 1e-6
