"""Shared fixtures of the GPU parity tests: meshes, oracle matrices, the context."""
import functools

import numpy as np

import oracle
from oracle import oracle as O
from synth import icosphere
from synth.charges import ball_charges
from synth.icosphere import uv_ellipsoid

PHYS = O.Physics(4.0, 80.0, 0.125)

# operator name in the oracle -> (PB_OP_*, PB_LAPLACE/PB_YUKAWA)
OPS = {"VL": (0, 0), "KL": (1, 0), "TL": (2, 0), "DL": (3, 0), "VY": (0, 1), "KY": (1, 1), "TY": (2, 1),
       "DY": (3, 1), "M": (4, 0)}


@functools.lru_cache(maxsize=None)
def mesh_case(name):
    """Small meshes the dense oracle handles in seconds. 'uv' is an irregular
    ellipsoid off the origin whose point count leaves ragged tails in every
    tile size (260 triangles, 1560 points at 6 per triangle)."""
    if name == "ico3":
        v, t = icosphere(3, 2.0)
        xq, q = np.zeros((1, 3)), np.ones(1)
    elif name == "ico2":
        v, t = icosphere(2, 2.0)
        xq, q = ball_charges(5, 1.5, 7)
    elif name == "uv":
        v, t = uv_ellipsoid(13, 11, (2.0, 1.6, 1.3), center=(0.3, -0.2, 0.1), twist=0.15)
        xq, q = ball_charges(4, 0.9, 11)
        xq = xq + np.array([0.3, -0.2, 0.1])
    else:
        raise KeyError(name)
    return v, t, xq, q


@functools.lru_cache(maxsize=None)
def oracle_ops(name, far_q=6, n_ss=4):
    v, t, _, _ = mesh_case(name)
    return oracle.assemble(v, t, PHYS.kappa, O.Plan(far_q, n_ss))


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
