"""Seeded synthetic inputs shared by the tests, the oracle scripts and bench.py.

This package only draws geometry (island curves on the unit sphere and their
derivatives), point sources, off-curve targets and densities.  It holds none
of the method's arithmetic: no projection, no kernel, no Green's function.
"""
from .star_caps import (  # noqa: F401
    Geometry,
    star_caps,
    config_geometry,
    pair_sources,
    random_pair_sources,
    targets_off_islands,
    random_density,
    rotation_to_pole,
    apply_rotation,
    rotated,
    batch_instances,
    ellipse_islands,
    fibonacci_centres,
)
