"""Seeded synthetic inputs for the TSQBX near-field step.

This package only builds inputs: flat-triangle surfaces with interior
quadrature nodes, QBX centers and targets, densities, and the grouped CSR pair
lists (radius lists, or the GIGAQBX octree Lists 1 / 3 close / 4 close).  It
holds none of the expansion arithmetic.  Both the CPU oracle and the GPU
library consume what it produces; neither is imported here.
"""
from .geometry import Geometry  # noqa: F401
