"""Pins of the oracle's quadrature: triangle rules, the singular-pair maps and
the singular local blocks against an independent polar-coordinate brute force."""
import ctypes
import itertools
import math

import numpy as np
import pytest

from oracle import _clib, pair_blocks, Plan
from oracle.quadrature import gauss_legendre01, triangle_rule


def _tri_moment(a, b):
    """int over the unit right triangle {x,y >= 0, x+y <= 1} of x^a y^b."""
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


@pytest.mark.parametrize("q,deg", [(6, 4), (3, 2), (1, 1)])
def test_triangle_rule_exact_to_its_degree(q, deg):
    pts, w = triangle_rule(q)
    assert abs(w.sum() - 1.0) < 1e-14
    assert np.allclose(pts.sum(axis=1), 1.0, atol=1e-15)
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            # barycentrics (l0, l1, l2): x = l1, y = l2 on the unit right triangle (area 1/2)
            approx = 0.5 * np.sum(w * pts[:, 1] ** a * pts[:, 2] ** b)
            assert abs(approx - _tri_moment(a, b)) < 1e-14, (q, a, b)
    # and it is not exact one degree higher (so the degree is what is claimed)
    errs = [abs(0.5 * np.sum(w * pts[:, 1] ** a * pts[:, 2] ** (deg + 1 - a)) - _tri_moment(a, deg + 1 - a))
            for a in range(deg + 2)]
    assert max(errs) > 1e-6


def _ss_moment(kind, n, a, b, c, d):
    L = _clib.lib()
    L.oracle_ss_moment.restype = ctypes.c_double
    L.oracle_ss_moment.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_int] * 4
    gx, gw = gauss_legendre01(n)
    return L.oracle_ss_moment(kind, n, gx.ctypes.data, gw.ctypes.data, a, b, c, d)


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_singular_maps_tile_the_pair_domain(kind):
    """The regions of each singular kind must cover T^ x T^ exactly once with
    the right Jacobian: then every polynomial moment equals the product of the
    two reference-triangle moments (T^ = {0 <= t <= s <= 1})."""
    def m(p, r):
        return 1.0 / ((r + 1) * (p + r + 2))
    for a, b, c, d in itertools.product(range(3), repeat=4):
        got = _ss_moment(kind, 8, a, b, c, d)
        assert abs(got - m(a, b) * m(c, d)) < 1e-13 * m(a, b) * m(c, d) * 100, (kind, a, b, c, d)


# ---------------------------------------------------------------------------------------------
# Independent brute force for coplanar singular pairs: inner integral in polar coordinates
# about the outer point x (the 1/rho of the kernel cancels the polar Jacobian), outer integral
# by a high-order collapsed Gauss product rule on the test triangle.
# ---------------------------------------------------------------------------------------------

def _collapsed_rule(P, n):
    """Points (in the plane) and weights of an n x n collapsed Gauss rule on triangle P."""
    g, w = gauss_legendre01(n)
    u, v = np.meshgrid(g, g, indexing="ij")
    wu, wv = np.meshgrid(w, w, indexing="ij")
    l1 = u.ravel()
    l2 = (u * v).ravel()        # (s, t) in {0 <= t <= s <= 1}
    jac = (wu * wv * u).ravel()
    A = P[0] + np.outer(l1, P[1] - P[0]) + np.outer(l2, P[2] - P[1])
    e1, e2 = P[1] - P[0], P[2] - P[0]
    area = 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
    return A, jac * 2.0 * area


def _bary(P, x):
    """Barycentric coordinates of 2D points x in triangle P."""
    T = np.array([[P[1][0] - P[0][0], P[2][0] - P[0][0]], [P[1][1] - P[0][1], P[2][1] - P[0][1]]])
    lam12 = np.linalg.solve(T, (x - P[0]).T).T
    return np.column_stack([1.0 - lam12.sum(axis=1), lam12])


def _ray_interval(S, x, d):
    """Entry and exit distance of the ray x + rho d through convex triangle S."""
    hits = []
    for k in range(3):
        p, q = S[k], S[(k + 1) % 3]
        e = q - p
        M = np.array([[d[0], -e[0]], [d[1], -e[1]]])
        det = np.linalg.det(M)
        if abs(det) < 1e-300:
            continue
        rho, s = np.linalg.solve(M, p - x)
        if -1e-12 <= s <= 1 + 1e-12 and rho >= -1e-12:
            hits.append(max(rho, 0.0))
    if not hits:
        return None
    inside = _bary(S, x[None, :]).min() >= -1e-12
    return (0.0 if inside else min(hits)), max(hits)


def _polar_inner(S, x, kappa, n_theta=48, n_rho=24):
    """int_S lambda_b(y) g(|x-y|) dy for b = 0,1,2 with g = 1/(4 pi r) and
    g = e^{-kappa r}/(4 pi r), by polar coordinates about x."""
    ang = np.sort(np.mod([math.atan2(*(S[k] - x)[::-1]) for k in range(3)], 2 * np.pi))
    inside = _bary(S, x[None, :]).min() >= -1e-12
    if inside:
        cuts = [ang[0], ang[1], ang[2], ang[0] + 2 * np.pi]
    else:
        # the wedge subtended by S: the largest gap between vertex angles is outside it
        gaps = np.diff(np.concatenate([ang, [ang[0] + 2 * np.pi]]))
        k = int(np.argmax(gaps))
        start = ang[(k + 1) % 3]
        a2 = [np.mod(ang[(k + 1 + j) % 3] - start, 2 * np.pi) + start for j in range(3)]
        cuts = a2
    gt, wt = gauss_legendre01(n_theta)
    gr, wr = gauss_legendre01(n_rho)
    out = np.zeros((2, 3))
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        for t, wtt in zip(lo + (hi - lo) * gt, (hi - lo) * wt):
            d = np.array([math.cos(t), math.sin(t)])
            iv = _ray_interval(S, x, d)
            if iv is None:
                continue
            r0, r1 = iv
            rho = r0 + (r1 - r0) * gr
            y = x[None, :] + rho[:, None] * d[None, :]
            lam = _bary(S, y)
            base = wtt * (r1 - r0) * wr / (4.0 * np.pi)  # g * rho = 1/(4 pi)
            out[0] += base @ lam
            out[1] += (base * np.exp(-kappa * rho)) @ lam
    return out


def _brute_V(T, S, kappa, n_outer=16):
    X, W = _collapsed_rule(T, n_outer)
    lamx = _bary(T, X)
    V = np.zeros((2, 3, 3))
    for x, w, lx in zip(X, W, lamx):
        inner = _polar_inner(S, x, kappa)
        V += w * lx[None, :, None] * inner[:, None, :]
    return V


def _to3d(P):
    return np.column_stack([P, np.zeros(len(P))])


@pytest.mark.slow
@pytest.mark.parametrize("kind", ["coincident", "edge", "vertex"])
def test_singular_V_blocks_match_polar_brute_force(kind):
    """Coplanar singular pairs: the oracle's V_L and V_Y local blocks (any
    number of Gauss points) converge to an independent polar-coordinate
    brute force; D carries the same kernel, K vanishes (coplanar)."""
    P = np.array([[0.0, 0.0], [1.0, 0.1], [0.3, 0.8], [1.1, 0.9], [-0.6, -0.5], [0.2, -0.9]])
    tris = {"coincident": [[0, 1, 2], [0, 1, 2]],
            "edge": [[0, 1, 2], [1, 3, 2]],
            "vertex": [[0, 1, 2], [0, 4, 5]]}[kind]
    verts = _to3d(P)
    t = np.array(tris, dtype=np.int32)
    kappa = 0.7
    hi = pair_blocks(verts, t, 0, 1, kappa, Plan(far_q=6, n_ss=12))
    lo = pair_blocks(verts, t, 0, 1, kappa, Plan(far_q=6, n_ss=4))
    scale = np.abs(hi[0]).max()
    coarse = _brute_V(P[t[0]], P[t[1]], kappa, n_outer=10)
    fine = _brute_V(P[t[0]], P[t[1]], kappa, n_outer=20)
    e_coarse = np.abs(coarse[0] - hi[0]).max() / scale
    e_fine = np.abs(fine[0] - hi[0]).max() / scale
    # the brute force converges towards the singular rule's value ...
    assert e_fine < 5e-5 and e_fine < e_coarse / 3.0, (e_coarse, e_fine)
    assert np.abs(fine[1] - hi[3]).max() / np.abs(hi[3]).max() < 5e-5
    # ... and the plan's 4-point rule is within its own quadrature error of it
    assert np.abs(lo[0] - hi[0]).max() / scale < 3e-5
    assert np.abs(hi[1]).max() < 1e-15 and np.abs(hi[4]).max() < 1e-15  # (x-y).n_y = 0


def test_far_pair_uses_the_triangle_rule():
    """Two well-separated triangles: the blocks equal the 6-point x 6-point
    rule written out directly (brute force of the definition)."""
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [3, 0, 1], [3, 1, 1.2], [2.5, 0.3, 2.0]], float)
    t = np.array([[0, 1, 2], [3, 4, 5]], dtype=np.int32)
    kappa = 0.3
    blk = pair_blocks(verts, t, 0, 1, kappa)
    rl, rw = triangle_rule(6)
    A, B = verts[t[0]], verts[t[1]]
    at = 0.5 * np.linalg.norm(np.cross(A[1] - A[0], A[2] - A[0]))
    bs = 0.5 * np.linalg.norm(np.cross(B[1] - B[0], B[2] - B[0]))
    ny = np.cross(B[1] - B[0], B[2] - B[0]); ny /= np.linalg.norm(ny)
    V = np.zeros((3, 3)); K = np.zeros((3, 3)); VY = np.zeros((3, 3))
    for i in range(6):
        x = rl[i] @ A
        for j in range(6):
            y = rl[j] @ B
            r = np.linalg.norm(x - y)
            w = rw[i] * rw[j] * at * bs
            V += w * np.outer(rl[i], rl[j]) / (4 * np.pi * r)
            VY += w * np.outer(rl[i], rl[j]) * np.exp(-kappa * r) / (4 * np.pi * r)
            K += w * np.outer(rl[i], rl[j]) * np.dot(x - y, ny) / (4 * np.pi * r ** 3)
    assert np.allclose(blk[0], V, rtol=1e-13, atol=0)
    assert np.allclose(blk[1], K, rtol=1e-12, atol=1e-18)
    assert np.allclose(blk[3], VY, rtol=1e-13, atol=0)


def _shared(t, i, j):
    return len(set(t[i]) & set(t[j]))


def test_per_class_singular_orders():
    """A plan with a singular order per class of pair (coincident, edge,
    vertex) uses, for every pair, the plain plan's rule of its own class's
    order, and nothing else changes: the blocks of a pair of class c under
    (n_coin, n_edge, n_vert) equal its blocks under the plain plan with
    n_ss = n_c, bit for bit; per-class orders all equal to n_ss are the plain
    plan, bit for bit, for the whole assembly."""
    from synth import icosphere
    v, t = icosphere(1, 1.5)
    kappa = 0.125
    by_class = {3: [], 2: [], 1: [], 0: []}
    for i in range(len(t)):
        for j in range(len(t)):
            k = _shared(t, i, j)
            if len(by_class[k]) < 3:
                by_class[k].append((i, j))
    mixed = Plan(6, 4, n_ss_coin=5, n_ss_edge=3, n_ss_vert=2)
    order = {3: 5, 2: 3, 1: 2}
    for k, pairs in by_class.items():
        assert pairs, k
        for i, j in pairs:
            got = pair_blocks(v, t, i, j, kappa, mixed)
            want = pair_blocks(v, t, i, j, kappa, Plan(6, order.get(k, 4)))
            assert np.array_equal(got, want), (k, i, j)
            if k in order:  # and the order matters for that class
                assert not np.array_equal(got, pair_blocks(v, t, i, j, kappa, Plan(6, 4))), (k, i, j)
    import oracle
    a = oracle.assemble(v, t, kappa, Plan(6, 4))
    b = oracle.assemble(v, t, kappa, Plan(6, 4, n_ss_coin=4, n_ss_edge=4, n_ss_vert=4))
    for name in ("VL", "KL", "DL", "VY", "KY", "DY", "M"):
        assert np.array_equal(getattr(a, name), getattr(b, name)), name
