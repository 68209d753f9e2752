"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This package builds inputs only: the voxelised phantom, the analytic breathing
DVF family, the PCA motion model (x_mean, U) of its training phases, the scan
geometry of each workload, and standard-normal noise draws. It holds none of
the reconstruction arithmetic (DVF synthesis, warp, projection, cost, gradient,
line search, tumor inversion); measured projections are assembled from these
inputs by the oracle (tests) or by the library (benchmark).
"""

from .generate import (  # noqa: F401
    Volume,
    Geometry,
    phantom_volume,
    phantom_point_values,
    MU_BODY, MU_LUNG, MU_TUMOR, MU_SPINE,
    breathing_phase,
    dvf_analytic,
    training_dvfs,
    PCAModel,
    build_pca,
    tumor_centre,
    tumor_truth,
    standard_normal,
    workload_small,
    workload_paper,
    workload_mixed,
    MIXED_SHAPES,
    DETECTORS,
)
