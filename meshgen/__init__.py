"""Seeded synthetic triangle meshes used as inputs by the tests, the benchmark and the oracle.

This package builds meshes only: it places nodes, triangulates them with Qhull
(``scipy.spatial.Delaunay``), carves holes and jitters.  It holds none of the
time-stepping method's arithmetic; its one geometric acceptance test (the Delaunay margin of
each interior edge) is its own code and is used only to accept or redraw node positions.
Both the CUDA library and the oracle consume its output; neither is imported here.
"""
from .core import (  # noqa: F401
    MeshArrays,
    cavity_lattice,
    right_split_lattice,
    equilateral_lattice,
    random_delaunay,
    graded_square,
    polygon_triangle,
    polygon_ellipse,
    polygon_rectangle,
    edge_table,
    delaunay_margin,
)
from .configs import (  # noqa: F401
    cavity_te11_mesh,
    scatterer_mesh,
    plasma_square_mesh,
    batch_meshes,
    batch_specs,
    batch_mesh,
    learned_specs,
    learned_mesh,
    source_line_amplitudes,
    plasma_density_nodes,
    te_mode_b,
    cached,
)
