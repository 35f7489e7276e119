"""GB300-native 3D-mode cosmic-ray propagation (arXiv:1410.5323, CRPropa 3 hot path).

Thin Python binding of ``libcrp.so`` (C ABI in ``include/crp.h``): argument marshalling
only. Every step of the propagation runs in the library's CUDA kernels; there is no CPU
fallback, and using the binding without the built library raises.

    from paper_1410_5323_gb300 import Field, Tables, Simulation
"""
from __future__ import annotations

from .api import (  # noqa: F401
    BOUNDARY_NONE,
    BOUNDARY_REFLECT,
    COLUMNS,
    FORM_FP64,
    FORM_MIXED,
    GRID_AUTO,
    GRID_CELLS,
    GRID_NODES,
    MAX_SPECIES,
    STATUS_ACTIVE,
    STATUS_DONE,
    STATUS_NAN,
    STATUS_RANGE,
    CrpError,
    Field,
    Lens,
    Simulation,
    Spectrum,
    Tables,
    debug_fail_allocations,
    healpix_ring,
    kernel_runs,
    lib,
    selftest_wait,
)
