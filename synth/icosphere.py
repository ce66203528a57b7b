"""Icosphere meshes: a regular icosahedron refined by 4-to-1 midpoint splits,
with every vertex projected back to the sphere after each split.

Level L has 10*4**L + 2 vertices and 20*4**L triangles. Triangles are listed
counter-clockwise as seen from outside, so the right-hand normal points out of
the enclosed volume.
"""
import numpy as np


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
    ], dtype=np.float64)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int64)
    return v, f


def _orient_outward(v, f):
    """Flip any triangle whose right-hand normal points towards the centre."""
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    n = np.cross(b - a, c - a)
    inward = np.einsum("ij,ij->i", n, a + b + c) < 0
    f = f.copy()
    f[inward] = f[inward][:, [0, 2, 1]]
    return f


def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Return (verts float64 [N_v,3], tris int32 [N_t,3]) of an icosphere."""
    if level < 0:
        raise ValueError("level must be >= 0")
    v, f = _icosahedron()
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    f = _orient_outward(v, f)
    for _ in range(level):
        verts = list(v)
        cache = {}

        def mid(i, j):
            key = (i, j) if i < j else (j, i)
            k = cache.get(key)
            if k is None:
                m = 0.5 * (verts[i] + verts[j])
                m = m / np.linalg.norm(m)
                k = len(verts)
                verts.append(m)
                cache[key] = k
            return k

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        v = np.array(verts)
        f = np.array(nf, dtype=np.int64)
    v = v * float(radius) + np.asarray(center, dtype=np.float64)
    return np.ascontiguousarray(v, dtype=np.float64), np.ascontiguousarray(f, dtype=np.int32)


def uv_ellipsoid(n_lon: int, n_lat: int, axes=(1.0, 1.0, 1.0), center=(0.0, 0.0, 0.0), twist: float = 0.0):
    """Latitude-longitude ellipsoid with two pole vertices.

    n_lat - 1 rings of n_lon vertices; 2 n_lon (n_lat - 1) triangles, so the
    triangle count is not a power-of-two multiple (useful for ragged tails).
    ``twist`` rotates each ring by twist * ring index (radians) to make the
    triangles non-symmetric. Counter-clockwise seen from outside."""
    if n_lon < 3 or n_lat < 2:
        raise ValueError("need n_lon >= 3 and n_lat >= 2")
    a = np.asarray(axes, dtype=np.float64)
    verts = [[0.0, 0.0, 1.0]]
    for i in range(1, n_lat):
        th = np.pi * i / n_lat
        for j in range(n_lon):
            ph = 2.0 * np.pi * j / n_lon + twist * i
            verts.append([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    verts.append([0.0, 0.0, -1.0])
    v = np.array(verts) * a + np.asarray(center, dtype=np.float64)
    south = len(verts) - 1

    def ring(i, j):
        return 1 + (i - 1) * n_lon + (j % n_lon)

    f = []
    for j in range(n_lon):
        f.append([0, ring(1, j), ring(1, j + 1)])
    for i in range(1, n_lat - 1):
        for j in range(n_lon):
            p, q, r, s = ring(i, j), ring(i, j + 1), ring(i + 1, j), ring(i + 1, j + 1)
            f.append([p, r, s])
            f.append([p, s, q])
    for j in range(n_lon):
        f.append([south, ring(n_lat - 1, j + 1), ring(n_lat - 1, j)])
    f = np.array(f, dtype=np.int64)
    f = _orient_outward(v - np.asarray(center, dtype=np.float64), f)
    return np.ascontiguousarray(v, dtype=np.float64), np.ascontiguousarray(f, dtype=np.int32)
