"""The seeded input generators: meshes are closed oriented 2-manifolds that
enclose every atom, at the requested vertex density, reproducibly."""
import numpy as np
import pytest

from synth import icosphere, serving_stream, synthetic_molecule
from synth.icosphere import uv_ellipsoid
from synth.molecule import check_closed_manifold, winding_numbers


def _area(v, f):
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)


def _volume(v, f):
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    return np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0


@pytest.mark.parametrize("level", [0, 2, 5])
def test_icosphere_counts_and_orientation(level):
    v, f = icosphere(level, 3.0)
    assert len(v) == 10 * 4 ** level + 2 and len(f) == 20 * 4 ** level
    assert check_closed_manifold(f)
    assert _volume(v, f) > 0
    assert np.allclose(np.linalg.norm(v, axis=1), 3.0)


def test_uv_ellipsoid_is_closed_and_outward():
    v, f = uv_ellipsoid(13, 11, (2.0, 1.6, 1.3), center=(0.3, -0.2, 0.1), twist=0.15)
    assert check_closed_manifold(f) and _volume(v, f) > 0 and len(f) == 260


def test_synthetic_molecule():
    v, f, pos, q, radii = synthetic_molecule(60, 21)
    assert f.dtype == np.int32 and check_closed_manifold(f)
    assert _volume(v, f) > 0
    w = winding_numbers(v, f, pos)
    assert np.all(np.abs(w - 1.0) < 1e-6)  # every atom inside the surface
    assert abs(q.sum() - round(q.sum())) < 1e-12 and np.all(np.abs(q) <= 0.8 + 1.0 / 60)
    assert np.all((radii >= 1.2) & (radii <= 2.0))
    dens = len(v) / _area(v, f).sum()
    assert 3.5 < dens < 4.6
    # the same seed gives the same molecule
    v2, f2, pos2, _, _ = synthetic_molecule(60, 21)
    assert np.array_equal(f, f2) and np.array_equal(v, v2) and np.array_equal(pos, pos2)


def test_serving_stream_mix():
    s = serving_stream(512, 5)
    n = np.array([r["n_atoms"] for r in s])
    assert n.min() >= 50 and n.max() < 3000
    assert set(r["case"] for r in s) == {2, 10, 12, 23}
    assert s == serving_stream(512, 5)
