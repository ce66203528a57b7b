"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module builds meshes and charge sets only. It holds none of the boundary
element arithmetic (no Green's functions, quadrature, operators or solves), so
both the FP64 oracle and the CUDA path can take their inputs from here without
sharing any of the method's code.

Workloads (all seeded, all synthetic):
  * ``kirkwood_sphere``  - icosphere level 3, radius 2 A, one +1 e charge at the
    centre (the Born/Kirkwood closed-form case).
  * ``multi_charge_sphere`` - icosphere level 5, radius 10 A, 20 charges drawn
    uniformly in the ball of radius 8 A with values uniform in [-1, 1] e.
  * ``synthetic_molecule`` - random-walk atoms with a Gaussian-surface mesh
    (see ``synth.molecule``), standing in for the PDB molecules with
    solvent-excluded surfaces used in the paper's scaling study.
"""
from .icosphere import icosphere, uv_ellipsoid
from .charges import ball_charges, kirkwood_sphere, multi_charge_sphere
from .molecule import protein_like_500, protein_like_5000, serving_stream, synthetic_molecule

__all__ = ["icosphere", "uv_ellipsoid", "ball_charges", "kirkwood_sphere", "multi_charge_sphere",
           "protein_like_500", "protein_like_5000", "serving_stream", "synthetic_molecule"]
