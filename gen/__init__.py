"""Seeded synthetic inputs for the PIRMCut hot path.

This package builds graphs (full symmetric CSR including the terminals s and t)
and nothing else: it holds none of the method's arithmetic. Both the FP64 CPU
oracle (through the tests) and the CUDA library take their inputs from here.
"""
from .graphs import (  # noqa: F401
    Graph,
    csr_from_edges,
    image_disks_2d,
    image_ellipsoid_3d,
    segmentation_grid,
    random_graph,
    chung_lu_instance,
    chung_lu_batch,
    config_graph,
    perturb_capacities,
    capacity_sequence,
    permute_graph,
    CONFIGS,
)
