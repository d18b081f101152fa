"""Seeded synthetic inputs for the fast random-walk Kalman filter.

This package generates the *inputs* of the method and nothing else: cell-centre
point sets, straight-ray travel-time measurement operators (Sec. 4.1.1,
Eq. lineartomography), a random-walk "truth" trajectory and noisy measurements.
It holds none of the filter's arithmetic (no covariance kernel, no Kalman
algebra), so both the CUDA path and the CPU oracle may import it.
"""

from .tomography import (  # noqa: F401
    BASE_SEED,
    Csr,
    grid_points_2d,
    grid_points_3d,
    cross_well_geometry_2d,
    cross_well_geometry_3d,
    trace_rays_2d,
    trace_rays_3d,
    smooth_increment,
    random_walk_truth,
    measurements,
    tomography_workload,
    varying_ray_operators,
    csr_to_dense,
)
