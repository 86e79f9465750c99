"""Pins of the oracle's FP64 geometry (circumcentres, areas, dual lengths, eq. 4's sign)."""
import math

import numpy as np

import meshgen
from oracle import geometry, mesh as om


def test_equilateral_triangle_closed_forms():
    s = 0.37
    xy = np.array([[0.1, 0.2], [0.1 + s, 0.2], [0.1 + s / 2, 0.2 + s * math.sqrt(3) / 2]])
    t = np.array([[0, 1, 2]])
    O = geometry.circumcentres(xy, t)
    np.testing.assert_allclose(O[0], xy.mean(axis=0), rtol=0, atol=1e-15)
    np.testing.assert_allclose(geometry.areas(xy, t), [math.sqrt(3) / 4 * s * s], rtol=1e-14)


def test_right_triangle_circumcentre_is_hypotenuse_midpoint():
    xy = np.array([[0.3, -0.1], [1.7, -0.1], [0.3, 0.45]])
    O = geometry.circumcentres(xy, np.array([[0, 1, 2]]))
    np.testing.assert_allclose(O[0], 0.5 * (xy[1] + xy[2]), atol=1e-15)


def test_circumcentre_is_equidistant_on_random_meshes():
    ms = meshgen.random_delaunay(500, seed=11)
    O = geometry.circumcentres(ms.xy, ms.tris)
    r = [np.hypot(*(O - ms.xy[ms.tris[:, k]]).T) for k in range(3)]
    np.testing.assert_allclose(r[1], r[0], rtol=1e-9)
    np.testing.assert_allclose(r[2], r[0], rtol=1e-9)


def test_dual_length_equals_independent_cotangent_form():
    """|O_R O_L| from circumcentres vs (|e|/2)(cot a_R + cot a_L) from the opposite angles."""
    ms = meshgen.cavity_te11_mesh()
    m = om.canonicalize(ms.xy, ms.tris)
    g = geometry.Geometry(m)
    ie = m.interior_ids
    d_cot = np.zeros(m.n_edges)
    for q in range(3):
        e = m.tri_edge[:, q]
        a = m.xy[m.tris[:, q]]
        b = m.xy[m.tris[:, (q + 1) % 3]]
        o = m.xy[m.tris[:, (q + 2) % 3]]
        u, v = a - o, b - o
        cot = (u * v).sum(1) / np.abs(u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0])
        np.add.at(d_cot, e, 0.5 * np.hypot(*(b - a).T) * cot)
    np.testing.assert_allclose(g.d[ie], d_cot[ie], rtol=1e-10, atol=1e-14)
    assert np.all(g.d[ie] > 0)


def test_equilateral_lattice_dual_length():
    ms = meshgen.equilateral_lattice(6, h=0.25)
    m = om.canonicalize(ms.xy, ms.tris)
    g = geometry.Geometry(m)
    ie = m.interior_ids
    np.testing.assert_allclose(g.d[ie], 0.25 / math.sqrt(3), rtol=1e-13)


def test_areas_sum_to_domain():
    ms = meshgen.cavity_te11_mesh()
    m = om.canonicalize(ms.xy, ms.tris)
    assert abs(geometry.areas(m.xy, m.tris).sum() - 0.5) < 1e-14


def test_literal_sign_agrees_with_orientation_sign_for_acute_opposite_angles():
    """Eq. 4's sgn(y0.(O_j C x e)) equals s(j,q) whenever the angle opposite e is < 89 deg."""
    ms = meshgen.cavity_te11_mesh()
    m = om.canonicalize(ms.xy, ms.tris)
    O = geometry.circumcentres(m.xy, m.tris)
    lit = geometry.literal_signs(m, O)
    ang = np.zeros((m.n_tris, 3))
    for q in range(3):
        a = m.xy[m.tris[:, q]]
        b = m.xy[m.tris[:, (q + 1) % 3]]
        o = m.xy[m.tris[:, (q + 2) % 3]]
        u, v = a - o, b - o
        ang[:, q] = np.degrees(np.arccos((u * v).sum(1) / np.hypot(*u.T) / np.hypot(*v.T)))
    acute = ang < 89.0
    assert np.array_equal(lit[acute], m.tri_sign[acute])
    # where the opposite angle is obtuse the literal factor flips (O_j is across the edge)
    obtuse = ang > 91.0
    if obtuse.any():
        assert np.array_equal(lit[obtuse], -m.tri_sign[obtuse])
