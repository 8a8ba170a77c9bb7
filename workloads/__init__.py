"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds only input generation: layered media (interface heights,
wavenumbers, densities) and scatterer boundaries given as closed polygons
(vertex lists).  It contains none of the method's arithmetic -- turning a
polygon into Nystrom elements, Green's functions, expansions and solvers all
live on either side of the comparison (``oracle/`` and the CUDA library),
each in its own code.
"""

from .geometry import (  # noqa: F401
    Medium,
    Workload,
    circle,
    ellipse,
    sine_star,
    l_shape,
    config_c1,
    config_c2,
    config_c3,
    config_c4,
    config_c5_request,
    config_c5_stream,
    example1,
    example2,
    example3,
    random_bodies,
    layered_small,
    layered_wide,
    layered_wide_c3,
)
