"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the solver itself: it only draws the
random numbers and builds the integer phase maps that both the CUDA path
and the CPU oracle take as *inputs* (the paper takes the microstructure,
the material parameters and the grain orientations as given data).

Everything here is deterministic in its seed:

* random draws use ``numpy.random.default_rng(seed)`` (PCG64);
* geometry is decided in exact integer arithmetic on a lattice of 1/256
  voxel, so a phase map is bit-identical on every machine;
* Voronoi ties go to the lowest seed index, sphere membership is inclusive.

Workloads (sizes and recipes) are stated in the repository's design notes.
"""

from .microstructure import (  # noqa: F401
    centred_sphere,
    voronoi,
    random_spheres,
    laminate,
)
from .draws import (  # noqa: F401
    shoemake_quaternions,
    uniform_seeds,
    random_field,
)
from .workloads import (  # noqa: F401
    Material,
    Workload,
    sphere_inclusion_32,
    voronoi_polycrystal,
    x_laminate,
    y_laminate,
    iso_lame,
    bending_load,
    torsion_bending_load,
    sphere_composite_bending,
    cp_polycrystal_torsion_bending,
)
