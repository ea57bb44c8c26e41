"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package draws microstructures (voxel phase maps), per-phase parameter
tables, macroscopic load paths and random material-point states.  It holds
none of the method's arithmetic: no constitutive update, no Fourier transform,
no Green operator and no error measure.  Both sides of every parity check
(the CPU oracle and the CUDA library) receive identical arrays from here.

Every generator takes an explicit seed; the convention
``seed = 2409_10774 + 1000 * config + replica`` is used throughout.
"""
from .generators import (  # noqa: F401
    SEED_BASE,
    seed_for,
    PHASE_FIELDS,
    phase_record,
    sphere_map,
    laminate_map,
    rsa_sphere_map,
    voronoi_map,
    random_sphere_map,
    ramp_path,
    two_leg_path,
    workload_centered_sphere,
    workload_rsa_spheres,
    workload_voronoi,
    workload_batch,
    workload_serving_request,
    random_material_states,
)
