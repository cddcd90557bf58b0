"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package holds geometry and load generation only (lattices, jitter,
support and load selection, material tables).  It contains none of the
method's arithmetic (no energy, force, stress, damage or solver code), so
the oracle and the GPU path can both use it without sharing any of the
computation they are compared on.
"""
from .meshes import (  # noqa: F401
    kuhn_box, bcc_ellipsoid, jitter, beam_config, loaf_config, glass_config,
    batch_configs, two_tet_fig4, single_tet, Workload, LOAF_AXES,
)
from .weights import he_normal_weights  # noqa: F401
