"""Seeded point-charge sets and the two sphere workloads."""
import numpy as np

from .icosphere import icosphere


def ball_charges(n: int, radius: float, seed: int, qmax: float = 1.0):
    """n positions uniform in the ball |x| <= radius (rejection sampling from
    the enclosing cube) and charges uniform in [-qmax, qmax], both drawn from
    NumPy's PCG64 stream ``default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    pos = []
    while len(pos) < n:
        p = rng.uniform(-radius, radius, size=3)
        if p @ p <= radius * radius:
            pos.append(p)
    q = rng.uniform(-qmax, qmax, size=n)
    return np.array(pos, dtype=np.float64).reshape(n, 3), q.astype(np.float64)


def kirkwood_sphere(level: int = 3, radius: float = 2.0):
    """Sphere of the given radius with one +1 e charge at its centre."""
    v, f = icosphere(level, radius)
    return v, f, np.zeros((1, 3)), np.ones(1)


def multi_charge_sphere(level: int = 5, radius: float = 10.0, n_charges: int = 20,
                        charge_radius: float = 8.0, seed: int = 2):
    """Sphere with n_charges charges uniform in an inner ball (seed 2 by default)."""
    v, f = icosphere(level, radius)
    xq, q = ball_charges(n_charges, charge_radius, seed)
    return v, f, xq, q
