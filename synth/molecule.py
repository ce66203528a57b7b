"""Synthetic protein-like molecules: a seeded random-walk chain of atoms and a
closed triangulated Gaussian surface around it.

Atoms: a walk of fixed step (3.8 A) in uniformly random directions; a step
that lands within `clash` of any earlier non-bonded atom, or outside an
optional confining sphere, is redrawn (up to `retries` times; then the last
draw inside the sphere is kept even if it clashes). Radii are
uniform in [1.2, 2.0] A, charges uniform in [-0.8, 0.8] e, shifted by a common
amount so that the net charge is an integer.

Surface: the level set rho(x) = 1 of rho(x) = sum_k exp(-d (|x - c_k|^2 / R_k^2 - 1))
(a Gaussian molecular surface), extracted by marching tetrahedra on a cubic
grid split into six tetrahedra per cube along the main diagonal (a
consistent simplicial decomposition, so the piecewise-linear level set is a
closed 2-manifold). Surface vertices lie on grid edges and are welded by the
edge they lie on; their position along the edge is kept at least `delta` of
the edge length away from the grid nodes, which bounds the sliver triangles.
Triangles are oriented from the inside (rho > 1) out, and the largest
connected component is kept.
"""
import numpy as np

# the six tetrahedra of a cube along the (0,0,0)-(1,1,1) diagonal: one per
# permutation of the axes; corner c = (x, y, z) bits -> index x + 2y + 4z
_AXES = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _tets():
    out = []
    for a, b, c in _AXES:
        v0 = (0, 0, 0)
        v1 = tuple(1 if k == a else 0 for k in range(3))
        v2 = tuple(1 if k in (a, b) else 0 for k in range(3))
        v3 = (1, 1, 1)
        out.append([p[0] + 2 * p[1] + 4 * p[2] for p in (v0, v1, v2, v3)])
    return np.array(out, dtype=np.int64)


TETS = _tets()


def random_walk_atoms(n, seed, step=3.8, clash=3.0, retries=100, confine=None):
    """Positions [n,3], radii [n], charges [n] of a seeded random-walk chain."""
    rng = np.random.default_rng(seed)
    pos = np.zeros((n, 3))
    cell = clash
    grid = {}

    def key(p):
        return tuple(np.floor(p / cell).astype(np.int64))

    def clashes(p, upto):
        kx, ky, kz = key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for j in grid.get((kx + dx, ky + dy, kz + dz), ()):
                        if j < upto and np.sum((pos[j] - p) ** 2) < clash * clash:
                            return True
        return False

    grid.setdefault(key(pos[0]), []).append(0)
    for i in range(1, n):
        chosen, fallback = None, None
        for _ in range(retries):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            p = pos[i - 1] + step * d
            if confine is not None and np.linalg.norm(p) > confine:
                continue
            fallback = p
            if not clashes(p, i - 1):  # every earlier atom except the bonded one
                chosen = p
                break
        if chosen is None:  # no free spot: a clashing spot inside the sphere, else towards its centre
            if fallback is None:
                d = -pos[i - 1] / max(np.linalg.norm(pos[i - 1]), 1e-12)
                fallback = pos[i - 1] + step * d
            chosen = fallback
        p = chosen
        pos[i] = p
        grid.setdefault(key(p), []).append(i)
    radii = rng.uniform(1.2, 2.0, size=n)
    q = rng.uniform(-0.8, 0.8, size=n)
    q -= (q.sum() - np.round(q.sum())) / n
    return pos, radii, q


def gaussian_density(centers, radii, lo, h, shape, decay=2.3, cutoff=1e-7):
    """rho on the grid lo + h * (i, j, k), summed atom by atom over the box
    where each Gaussian exceeds `cutoff`."""
    rho = np.zeros(shape)
    ext = np.sqrt(1.0 + np.log(1.0 / cutoff) / decay)  # |x - c| / R where the term falls to cutoff
    for c, r in zip(centers, radii):
        rad = ext * r
        i0 = np.maximum(np.floor((c - rad - lo) / h).astype(int), 0)
        i1 = np.minimum(np.ceil((c + rad - lo) / h).astype(int) + 1, np.array(shape))
        xs = [lo[k] + h * np.arange(i0[k], i1[k]) - c[k] for k in range(3)]
        d2 = xs[0][:, None, None] ** 2 + xs[1][None, :, None] ** 2 + xs[2][None, None, :] ** 2
        rho[i0[0]:i1[0], i0[1]:i1[1], i0[2]:i1[2]] += np.exp(-decay * (d2 / (r * r) - 1.0))
    return rho


_OTHERS = np.array([[k for k in range(4) if k != l] for l in range(4)], dtype=np.int64)


def marching_tetrahedra(f, lo, h, delta=0.05):
    """Closed oriented triangle mesh (verts, faces) of the level set f = 0 of a
    grid function f[nx, ny, nz] sampled at lo + h * (i, j, k); the inside is
    f > 0 and faces are counter-clockwise seen from outside."""
    nx, ny, nz = f.shape
    lo = np.asarray(lo, dtype=np.float64)
    f = np.where(f == 0.0, 1e-12, f)  # no grid node exactly on the level set
    inside = f > 0
    offs = np.array([(dx, dy, dz) for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)], dtype=np.int64)
    corner_in = np.stack([inside[dx:nx - 1 + dx, dy:ny - 1 + dy, dz:nz - 1 + dz] for dx, dy, dz in offs], axis=-1)
    cnt = corner_in.sum(axis=-1)
    base = np.stack(np.nonzero((cnt > 0) & (cnt < 8)), axis=1)      # cubes crossed by the level set
    corners = base[:, None, :] + offs[None, :, :]                    # [ncube, 8, 3]
    tc = corners[:, TETS, :].reshape(-1, 4, 3)                       # grid coords of tet vertices
    tv = (tc[..., 0] * ny + tc[..., 1]) * nz + tc[..., 2]            # global node ids
    tf = f.reshape(-1)[tv]
    tin = tf > 0
    nin = tin.sum(axis=1)
    keep = (nin > 0) & (nin < 4)
    tc, tv, tf, tin, nin = tc[keep], tv[keep], tf[keep], tin[keep], nin[keep]
    P = lo + h * tc.astype(np.float64)                               # [ntet, 4, 3]
    nnode = nx * ny * nz

    def ep(r, ai, bi):
        """welding key and position of the level-set point on edge (ai, bi) of tets r"""
        ga, gb = tv[r, ai], tv[r, bi]
        fa, fb = tf[r, ai], tf[r, bi]
        t = np.clip(fa / (fa - fb), delta, 1.0 - delta)
        pa, pb = P[r, ai], P[r, bi]
        return np.minimum(ga, gb) * nnode + np.maximum(ga, gb), pa + t[:, None] * (pb - pa)

    keys, pts, tri, iref, oref = [], [], [], [], []

    def add(tk, tp, ins, outs):
        keys.append(np.concatenate(tk))
        pts.append(np.concatenate(tp))
        tri.append(np.stack(tk, axis=1))
        iref.append(ins)
        oref.append(outs)

    for lone_in in (True, False):  # one vertex on its own side: one triangle
        r = np.nonzero(nin == (1 if lone_in else 3))[0]
        if r.size == 0:
            continue
        l = np.argmax(tin[r] if lone_in else ~tin[r], axis=1)
        oth = _OTHERS[l]
        tk, tp = [], []
        for j in range(3):
            k_, p_ = ep(r, l, oth[:, j])
            tk.append(k_)
            tp.append(p_)
        lone_p = P[r, l]
        rest_p = P[r[:, None], oth].mean(axis=1)
        add(tk, tp, lone_p if lone_in else rest_p, rest_p if lone_in else lone_p)
    r = np.nonzero(nin == 2)[0]
    if r.size:  # two and two: a quad on the four crossed edges, split in two
        order = np.argsort(~tin[r], axis=1, kind="stable")            # inside vertices first
        a0, a1, b0, b1 = order[:, 0], order[:, 1], order[:, 2], order[:, 3]
        tk, tp = [], []
        for u, v in ((a0, b0), (a0, b1), (a1, b1), (a1, b0)):
            k_, p_ = ep(r, u, v)
            tk.append(k_)
            tp.append(p_)
        ins = 0.5 * (P[r, a0] + P[r, a1])
        outs = 0.5 * (P[r, b0] + P[r, b1])
        add([tk[0], tk[1], tk[2]], [tp[0], tp[1], tp[2]], ins, outs)
        add([tk[0], tk[2], tk[3]], [tp[0], tp[2], tp[3]], ins, outs)
    allk = np.concatenate(keys)
    allp = np.concatenate(pts)
    ukeys, first = np.unique(allk, return_index=True)
    verts = allp[first]
    faces = np.searchsorted(ukeys, np.concatenate(tri))
    ins = np.concatenate(iref)
    outs = np.concatenate(oref)
    a, b, c = verts[faces[:, 0]], verts[faces[:, 1]], verts[faces[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(b - a, c - a), outs - ins) < 0
    faces[flip] = faces[flip][:, [0, 2, 1]]
    return verts, faces


def largest_component(verts, faces):
    """Keep the connected component with the most triangles; reindex."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    nv = verts.shape[0]
    e = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]])
    g = sp.coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(nv, nv))
    ncomp, lab = connected_components(g, directed=False)
    tl = lab[faces[:, 0]]
    best = np.bincount(tl, minlength=ncomp).argmax()
    faces = faces[tl == best]
    used = np.unique(faces)
    remap = -np.ones(nv, dtype=np.int64)
    remap[used] = np.arange(len(used))
    return verts[used], remap[faces]


def check_closed_manifold(faces):
    """True if every undirected edge is used by exactly two faces in opposite directions."""
    e = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]]).astype(np.int64)
    n = int(e.max()) + 1
    key = np.minimum(e[:, 0], e[:, 1]) * n + np.maximum(e[:, 0], e[:, 1])
    sign = np.where(e[:, 0] < e[:, 1], 1, -1)
    order = np.argsort(key, kind="stable")
    k, s_ = key[order], sign[order]
    uk, start, counts = np.unique(k, return_index=True, return_counts=True)
    if not np.all(counts == 2):
        return False
    return bool(np.all(s_[start] + s_[start + 1] == 0))


def density_and_gradient(points, centers, radii, decay, cutoff=1e-6, chunk=65536):
    """rho and grad rho at arbitrary points, from the atoms within the cutoff
    distance (k-d tree, fixed neighbour count, vectorised)."""
    from scipy.spatial import cKDTree
    ext = np.sqrt(1.0 + np.log(1.0 / cutoff) / decay) * radii.max()
    tree = cKDTree(centers)
    kmax = int(min(len(centers), max(8, tree.query_ball_point(centers[:1], ext, return_length=True)[0] * 3)))
    rho = np.zeros(len(points))
    grad = np.zeros((len(points), 3))
    for s in range(0, len(points), chunk):
        pts = points[s:s + chunk]
        dist, idx = tree.query(pts, k=kmax, distance_upper_bound=ext)
        if kmax == 1:
            dist, idx = dist[:, None], idx[:, None]
        valid = idx < len(centers)
        idc = np.where(valid, idx, 0)
        d = pts[:, None, :] - centers[idc]
        r2 = np.sum(d * d, axis=2) / radii[idc] ** 2
        e = np.where(valid, np.exp(-decay * (r2 - 1.0)), 0.0)
        rho[s:s + chunk] = e.sum(axis=1)
        grad[s:s + chunk] = np.einsum("pk,pkj->pj", -2.0 * decay * e / radii[idc] ** 2, d)
    return rho, grad


def smooth_on_level_set(verts, faces, centers, radii, decay, iters=4, lam=0.5):
    """Tangential Laplacian smoothing with projection back to rho = 1 (one
    Newton step along the gradient). Vertices of any triangle that would flip
    or nearly collapse keep their previous position."""
    nv = len(verts)
    e = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]])
    e = np.concatenate([e, e[:, ::-1]])
    deg = np.bincount(e[:, 0], minlength=nv)

    def normals(v):
        a, b, c = v[faces[:, 0]], v[faces[:, 1]], v[faces[:, 2]]
        return np.cross(b - a, c - a)

    for _ in range(iters):
        n0 = normals(verts)
        cen = np.zeros_like(verts)
        np.add.at(cen, e[:, 0], verts[e[:, 1]])
        cen /= deg[:, None]
        _, g = density_and_gradient(verts, centers, radii, decay)
        gn = g / np.maximum(np.linalg.norm(g, axis=1), 1e-300)[:, None]
        move = cen - verts
        move -= np.sum(move * gn, axis=1)[:, None] * gn  # tangential part
        cand = verts + lam * move
        rho, g2 = density_and_gradient(cand, centers, radii, decay)
        cand = cand - ((rho - 1.0) / np.maximum(np.sum(g2 * g2, axis=1), 1e-300))[:, None] * g2
        for _fix in range(6):
            n1 = normals(cand)
            bad = np.einsum("ij,ij->i", n0, n1) <= 0.1 * np.linalg.norm(n0, axis=1) * np.linalg.norm(n1, axis=1)
            if not bad.any():
                break
            vb = np.unique(faces[bad])
            cand[vb] = verts[vb]
        verts = cand
    return verts


def winding_numbers(verts, faces, points, chunk=256):
    """Generalised winding number of a closed oriented mesh at points (1 inside,
    0 outside), by the solid angle of each triangle (van Oosterom and Strackee)."""
    a0, b0, c0 = verts[faces[:, 0]], verts[faces[:, 1]], verts[faces[:, 2]]
    out = np.zeros(len(points))
    for s in range(0, len(points), chunk):
        p = points[s:s + chunk, None, :]
        a, b, c = a0[None] - p, b0[None] - p, c0[None] - p
        la, lb, lc = (np.linalg.norm(x, axis=2) for x in (a, b, c))
        num = np.einsum("pij,pij->pi", a, np.cross(b, c))
        den = la * lb * lc + np.einsum("pij,pij->pi", a, b) * lc + np.einsum("pij,pij->pi", b, c) * la + \
            np.einsum("pij,pij->pi", c, a) * lb
        out[s:s + chunk] = 2.0 * np.arctan2(num, den).sum(axis=1) / (4.0 * np.pi)
    return out


def molecule(n_atoms, seed, verts_per_A2=4.0, decay=2.3, inflate=1.0, confine=None, h=None, delta=0.05,
             smooth_iters=4):
    """A synthetic molecule: (verts, tris int32, atom positions, charges, radii).

    The surface uses radii R + inflate (a smooth surface around the van der
    Waals spheres, in the spirit of the solvent-excluded surface) so that one
    closed surface encloses every atom. The grid spacing is calibrated so that
    the mesh has about `verts_per_A2` vertices per square Angstrom."""
    pos, radii, q = random_walk_atoms(n_atoms, seed, confine=confine)
    rs = radii + inflate
    pad = 2.5 * rs.max() + 1.0

    def surface(hh):
        lo = pos.min(axis=0) - pad
        hi = pos.max(axis=0) + pad
        shape = tuple(int(np.ceil((hi[k] - lo[k]) / hh)) + 1 for k in range(3))
        rho = gaussian_density(pos, rs, lo, hh, shape, decay)
        v, f = marching_tetrahedra(rho - 1.0, lo, hh, delta)
        return largest_component(v, f)

    hh = h if h is not None else 0.6
    v, f = surface(hh)
    if h is None:
        for _ in range(2):
            a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
            dens = v.shape[0] / (0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1).sum())
            hh = hh * np.sqrt(dens / verts_per_A2)
            v, f = surface(hh)
    if smooth_iters:
        v = smooth_on_level_set(v, f, pos, rs, decay, iters=smooth_iters)
    return np.ascontiguousarray(v), np.ascontiguousarray(f, dtype=np.int32), pos, q, radii


def synthetic_molecule(n_atoms, seed, compactness=2.1, verts_per_A2=4.0):
    """Protein-like synthetic molecule: the walk is confined to a sphere of
    radius compactness * n_atoms^(1/3) A (compactness 2.1 gives ~40k
    triangles at 500 atoms). Returns (verts, tris, atom positions, charges, radii)."""
    return molecule(n_atoms, seed, verts_per_A2=verts_per_A2, confine=compactness * n_atoms ** (1.0 / 3.0))


def protein_like_500():
    """500 atoms, seed 3 (~40k triangles)."""
    return synthetic_molecule(500, 3, 2.1)


def protein_like_5000():
    """5000 atoms, seed 4, compactness calibrated to ~250k triangles."""
    return synthetic_molecule(5000, 4, 2.25)


def serving_stream(n_requests=512, seed=5, cases=(2, 10, 12, 23)):
    """The request mix of the serving workload: per request an atom count
    floor(exp(U[ln 50, ln 3000])), a Table-1 case drawn uniformly from
    `cases` and the seed of its molecule. Molecules are built on demand with
    synthetic_molecule(n_atoms, mol_seed)."""
    rng = np.random.default_rng(seed)
    n_atoms = np.floor(np.exp(rng.uniform(np.log(50.0), np.log(3000.0), size=n_requests))).astype(int)
    case = rng.choice(np.asarray(cases), size=n_requests)
    mol_seed = 10_000 + np.arange(n_requests)
    return [{"id": i, "n_atoms": int(n_atoms[i]), "case": int(case[i]), "mol_seed": int(mol_seed[i])}
            for i in range(n_requests)]
