"""Seeded synthetic inputs shared by the CPU oracle, the CUDA path's tests and the bench.

This package builds media (an isotropic background plus a per-voxel Voigt
stiffness contrast and a density contrast), moment-tensor sources and
frequency lists with the shapes and value distributions of the paper's
workloads (Sec. 4 and Tables 1-3).  It holds none of the Lippmann-Schwinger
arithmetic: no Green's tensor, no strain, no convolution, no solver.
"""
from .media import (  # noqa: F401
    BASE_SEED,
    Medium,
    iso_lame,
    iso_voigt,
    thomsen_vti,
    bond_rotate_y,
    pack21,
    unpack21,
    gaussian_random_field,
    inclusion_medium,
    layered_vti_medium,
    grf_orthorhombic_medium,
    table2_layers_medium,
    tti_layer_medium,
    random_medium,
)
from .sources import (  # noqa: F401
    voigt_moment,
    explosion,
    clvd,
    double_couple_12,
    double_couple_13,
    random_moment_tensors,
)
from .workloads import WORKLOADS, Workload, get_workload  # noqa: F401
