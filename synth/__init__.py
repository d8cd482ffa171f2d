"""Seeded synthetic inputs for the RGF transmission path.

This module draws random block-tridiagonal nonorthogonal devices, lead
blocks and energy grids.  It holds no transport arithmetic: it only draws
numbers and lays them out.  Both the FP64 oracle (``oracle/``) and the CUDA
path consume what it produces; neither side imports the other.
"""
from .devices import (  # noqa: F401
    Device,
    Lead,
    WORKLOADS,
    chain_device,
    energy_grid,
    make_device,
    make_workload,
    random_device,
)
