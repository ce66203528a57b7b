"""FP64 CPU oracle of the boundary-element Poisson-Boltzmann solve.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use it; the product path never imports it. It shares no code
with the CUDA library (the C core in bem_oracle.c is its own).

It computes the plain definitions, step by step:
  1. dense P1-Galerkin matrices V, K, D (Laplace and Yukawa), T = K^T and M
     (C core, ``assemble``);
  2. the 2x2 block system of each formulation (paper: direct int/ext and the
     permuted variants, CFIE int/ext (alpha, beta), PMCHWT, Mueller, Juffer,
     Lu) with identity -> mass matrix and sources tested against the basis;
  3. the left preconditioner (block diagonal, mass, scaled mass, full and
     half Calderon, scaled half Calderon);
  4. the solve, by dense LU of P^-1 A (the reference) and by unrestarted GMRES
     (modified Gram-Schmidt + Givens rotations) for iteration counts;
  5. the reaction potential at the charges and Delta G = 1/2 sum_j q_j phi_reac(x_j).

Readings of the paper (each listed in the design notes):
  * unknown vector x = [u; v], u = Dirichlet, v = Neumann trace P1 coefficients
    of the formulation's side (interior forms: interior traces; exterior forms:
    exterior traces, converted by u_i = u_e, v_i = (eps_ext/eps_int) v_e);
  * GMRES: x0 = 0, left preconditioning, stop at
    ||P^-1 (b - A x)||_2 <= tol ||P^-1 b||_2;
  * block diagonal preconditioner: per-DOF 2x2 inverse of the diagonals of the
    four weak-form blocks (identity terms included);
  * Calderon products in strong form: every product of two weak-form operators
    carries M^-1 in between, and the outer mass preconditioner on the left.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from . import _clib
from .quadrature import gauss_legendre01, triangle_rule

KCAL_PER_PAPER_UNIT = 4.0 * np.pi * 332.0636  # A12 reading: kcal/mol per e^2/A (1/4pi folded into G)


@dataclass(frozen=True)
class Plan:
    """Quadrature plan: regular triangle rule size and Gauss points per
    dimension of the singular (Sauter-Schwab) rule; optionally a distance band
    (band_eta > 0) inside which pairs that share no vertex take the finer rule
    band_q, the coarse far_q then serving only pairs farther apart than
    band_eta times the sum of their radii. The paper pairs low regular orders
    with far interactions (its FMM runs use order 3 regular, 4 singular); the
    band makes that distinction per triangle pair.

    The right-hand side and the reaction potential use the plan's reference
    rule: band_q with a band, far_q without."""
    far_q: int = 6
    n_ss: int = 4
    band_eta: float = 0.0
    band_q: int = 6
    # Gauss points per dimension of the singular rule for each class of pair
    # (None: n_ss). The paper states one singular order; a per-class order is
    # the same definition with the rule chosen by the pair's class.
    n_ss_coin: int | None = None
    n_ss_edge: int | None = None
    n_ss_vert: int | None = None

    @property
    def ref_q(self) -> int:
        return self.band_q if self.band_eta > 0 else self.far_q

    @property
    def n_ss_classes(self) -> tuple:
        """(coincident, edge, vertex) Gauss points per dimension."""
        return tuple(self.n_ss if n is None else n for n in (self.n_ss_coin, self.n_ss_edge, self.n_ss_vert))


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _mesh_arrays(verts, tris):
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    return v, t


def _rules(plan: Plan):
    """Far triangle rule and the three singular Gauss rules (coincident, edge,
    vertex) one after another, with their sizes."""
    rl, rw = triangle_rule(plan.far_q)
    ns = plan.n_ss_classes
    rules = [gauss_legendre01(n) for n in ns]
    gx = np.ascontiguousarray(np.concatenate([r[0] for r in rules]))
    gw = np.ascontiguousarray(np.concatenate([r[1] for r in rules]))
    ng = np.ascontiguousarray(np.array(ns, dtype=np.int32))
    return rl, rw, ng, gx, gw


def _band(plan: Plan):
    bl, bw = triangle_rule(plan.band_q)
    return float(plan.band_eta), bl.shape[0], bl, bw


@dataclass
class Operators:
    """Dense Galerkin matrices of one mesh (row = test vertex)."""
    VL: np.ndarray
    KL: np.ndarray
    DL: np.ndarray
    VY: np.ndarray
    KY: np.ndarray
    DY: np.ndarray
    M: np.ndarray
    kappa: float

    @property
    def TL(self):
        return self.KL.T

    @property
    def TY(self):
        return self.KY.T

    @property
    def n(self):
        return self.M.shape[0]


def pair_blocks(verts, tris, ti, tj, kappa, plan=Plan()):
    """Six local 3x3 blocks (V_L, K_L, D_L, V_Y, K_Y, D_Y) of one triangle pair."""
    v, t = _mesh_arrays(verts, tris)
    rl, rw, ng, gx, gw = _rules(plan)
    eta, nb, bl, bw = _band(plan)
    out = np.zeros((6, 3, 3))
    _clib.lib().oracle_pair_blocks(_ptr(v), _ptr(t), ti, tj, rl.shape[0], _ptr(rl), _ptr(rw),
                                   _ptr(ng), _ptr(gx), _ptr(gw), float(kappa), eta, nb, _ptr(bl), _ptr(bw),
                                   _ptr(out))
    return out


def assemble(verts, tris, kappa, plan=Plan(), nthreads=0) -> Operators:
    """Dense assembly of all operators (loop over all triangle pairs)."""
    v, t = _mesh_arrays(verts, tris)
    nv, nt = v.shape[0], t.shape[0]
    rl, rw, ng, gx, gw = _rules(plan)
    eta, nb, bl, bw = _band(plan)
    mats = [np.zeros((nv, nv)) for _ in range(7)]
    rc = _clib.lib().oracle_assemble_dense(
        _ptr(v), nv, _ptr(t), nt, rl.shape[0], _ptr(rl), _ptr(rw), _ptr(ng), _ptr(gx),
        _ptr(gw), float(kappa), eta, nb, _ptr(bl), _ptr(bw), int(nthreads), *[_ptr(m) for m in mats])
    if rc < 0:
        raise RuntimeError(f"oracle assembly failed ({rc})")
    return Operators(*mats, kappa=float(kappa))


def assemble_rows(verts, tris, rows, kappa, plan=Plan(), nthreads=0):
    """Selected rows of every operator: dict name -> [len(rows), N_v]."""
    v, t = _mesh_arrays(verts, tris)
    nv, nt = v.shape[0], t.shape[0]
    r = np.ascontiguousarray(rows, dtype=np.int64)
    rl, rw, ng, gx, gw = _rules(plan)
    eta, nb, bl, bw = _band(plan)
    mats = [np.zeros((r.shape[0], nv)) for _ in range(7)]
    _clib.lib().oracle_assemble_rows(
        _ptr(v), nv, _ptr(t), nt, _ptr(r), r.shape[0], rl.shape[0], _ptr(rl), _ptr(rw),
        _ptr(ng), _ptr(gx), _ptr(gw), float(kappa), eta, nb, _ptr(bl), _ptr(bw), int(nthreads),
        *[_ptr(m) for m in mats])
    return dict(zip(["VL", "KL", "DL", "VY", "KY", "DY", "M"], mats))


def band_pair_count(verts, tris, band_eta, nthreads=0):
    """Ordered triangle pairs that share no vertex and whose centroids are
    closer than band_eta times the sum of their radii (largest centroid-vertex
    distance): the pairs a banded plan integrates with its band rule."""
    v, t = _mesh_arrays(verts, tris)
    return int(_clib.lib().oracle_band_pair_count(_ptr(v), _ptr(t), t.shape[0], float(band_eta), int(nthreads)))


def source_projections(verts, tris, xq, q, eps_int, plan=Plan()):
    """(b_D, b_N): the charge potential and its normal derivative tested
    against the P1 basis (paper, source projections phi_D, phi_N)."""
    v, t = _mesh_arrays(verts, tris)
    x = np.ascontiguousarray(xq, dtype=np.float64).reshape(-1, 3)
    qq = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    rl, rw = triangle_rule(plan.ref_q)
    bD = np.zeros(v.shape[0])
    bN = np.zeros(v.shape[0])
    _clib.lib().oracle_rhs(_ptr(v), v.shape[0], _ptr(t), t.shape[0], rl.shape[0], _ptr(rl),
                           _ptr(rw), _ptr(x), _ptr(qq), x.shape[0], float(eps_int), _ptr(bD), _ptr(bN))
    return bD, bN


def reaction_potential(verts, tris, u_int, v_int, xq, plan=Plan()):
    """phi_reac at the points xq from the interior traces (paper, phi_reac
    as single minus double layer potential of the interior traces)."""
    v, t = _mesh_arrays(verts, tris)
    x = np.ascontiguousarray(xq, dtype=np.float64).reshape(-1, 3)
    uu = np.ascontiguousarray(u_int, dtype=np.float64)
    vv = np.ascontiguousarray(v_int, dtype=np.float64)
    rl, rw = triangle_rule(plan.ref_q)
    phi = np.zeros(x.shape[0])
    _clib.lib().oracle_reaction_potential(_ptr(v), v.shape[0], _ptr(t), t.shape[0], rl.shape[0],
                                          _ptr(rl), _ptr(rw), _ptr(uu), _ptr(vv), _ptr(x),
                                          x.shape[0], _ptr(phi))
    return phi


# --------------------------------------------------------------------------------------
# Formulations (paper: "Boundary integral formulations" - direct, CFIE and its cases)
# --------------------------------------------------------------------------------------

INTERIOR_FORMS = {"direct_int", "direct_int_perm", "cfie_int", "pmchwt_int", "muller_int", "juffer"}
EXTERIOR_FORMS = {"direct_ext", "direct_ext_perm", "cfie_ext", "pmchwt_ext", "muller_ext", "lu"}
FORMS = INTERIOR_FORMS | EXTERIOR_FORMS


@dataclass(frozen=True)
class Physics:
    eps_int: float = 4.0
    eps_ext: float = 80.0
    kappa: float = 0.125

    @property
    def r(self):
        """eps_int / eps_ext."""
        return self.eps_int / self.eps_ext


def _rows_int_int(o: Operators):
    """Interior Calderon system in interior unknowns (paper eq. bie:int:int),
    weak form: rows [1/2 M + K_i, -V_i], [-D_i, 1/2 M - T_i]."""
    h = 0.5 * o.M
    return [[h + o.KL, -o.VL], [-o.DL, h - o.TL]]


def _rows_ext_int(o: Operators, r):
    """Exterior system written for interior unknowns (paper eq. bie:ext:int):
    rows [1/2 M - K_e, r V_e], [D_e / r, 1/2 M + T_e]."""
    h = 0.5 * o.M
    return [[h - o.KY, r * o.VY], [o.DY / r, h + o.TY]]


def _rows_ext_ext(o: Operators):
    """Exterior Calderon system in exterior unknowns (paper eq. bie:ext:ext):
    rows [1/2 M - K_e, V_e], [D_e, 1/2 M + T_e]."""
    h = 0.5 * o.M
    return [[h - o.KY, o.VY], [o.DY, h + o.TY]]


def _rows_int_ext(o: Operators, r):
    """Interior system written for exterior unknowns (paper eq. bie:int:ext):
    rows [1/2 M + K_i, -V_i / r], [-r D_i, 1/2 M - T_i]."""
    h = 0.5 * o.M
    return [[h + o.KL, -o.VL / r], [-r * o.DL, h - o.TL]]


def _blocks_to_dense(B):
    return np.block([[B[0][0], B[0][1]], [B[1][0], B[1][1]]])


def form_params(form: str, phys: Physics, alpha=None, beta=None):
    """(alpha, beta, row2_scale) of the CFIE family members."""
    r = phys.r
    if form in ("cfie_int", "cfie_ext"):
        return alpha, beta, 1.0
    if form in ("pmchwt_int", "pmchwt_ext"):
        return -1.0, -1.0, 1.0
    if form in ("muller_int", "muller_ext"):
        return 1.0, 1.0, 1.0
    if form == "juffer":
        return 1.0 / r, r, 1.0
    if form == "lu":
        return r, 1.0 / r, r
    raise ValueError(form)


def system(form: str, o: Operators, phys: Physics, bD, bN, alpha=None, beta=None):
    """Dense 2n x 2n weak-form system matrix and right-hand side of a formulation."""
    n = o.n
    r = phys.r
    z = np.zeros(n)
    if form in ("direct_int", "direct_int_perm"):
        # paper eq. bie:dirichlet:int: first rows of the interior and exterior systems
        B = [_rows_int_int(o)[0], _rows_ext_int(o, r)[0]]
        rhs = [bD, z]
    elif form in ("direct_ext", "direct_ext_perm"):
        # paper eq. bie:dirichlet:ext
        B = [_rows_ext_ext(o)[0], _rows_int_ext(o, r)[0]]
        rhs = [z, bD]
    elif form in INTERIOR_FORMS:
        # paper eq. bie:combined:int: interior system + diag(alpha, beta) exterior system
        a, b, s2 = form_params(form, phys, alpha, beta)
        I, E = _rows_int_int(o), _rows_ext_int(o, r)
        B = [[I[0][0] + a * E[0][0], I[0][1] + a * E[0][1]],
             [I[1][0] + b * E[1][0], I[1][1] + b * E[1][1]]]
        rhs = [bD, bN]
        if form == "pmchwt_int":  # printed with both sides negated (paper eq. bie:pmchwt:int)
            B = [[-B[0][0], -B[0][1]], [-B[1][0], -B[1][1]]]
            rhs = [-bD, -bN]
    else:
        # paper eq. bie:combined:ext: exterior system + diag(alpha, beta) interior system
        a, b, s2 = form_params(form, phys, alpha, beta)
        E, I = _rows_ext_ext(o), _rows_int_ext(o, r)
        B = [[E[0][0] + a * I[0][0], E[0][1] + a * I[0][1]],
             [E[1][0] + b * I[1][0], E[1][1] + b * I[1][1]]]
        rhs = [a * bD, b * r * bN]
        if s2 != 1.0:  # Lu: second row multiplied by eps_int/eps_ext (paper eq. bie:lu:ext)
            B[1] = [s2 * B[1][0], s2 * B[1][1]]
            rhs[1] = s2 * rhs[1]
    if form.endswith("_perm"):  # permuted rows (paper, after eq. bie:dirichlet:ext)
        B = [B[1], B[0]]
        rhs = [rhs[1], rhs[0]]
    return _blocks_to_dense(B), np.concatenate(rhs)


def calderon_blocks(which: str, form: str, o: Operators, phys: Physics):
    """Weak-form Calderon preconditioning operator of a PMCHWT system
    (paper eqs. prec:calderon:int and prec:calderon:ext)."""
    r = phys.r
    if which == "full":
        return None
    if form == "pmchwt_int":
        if which == "int":
            B = [[-o.KL, o.VL], [o.DL, o.TL]]
        else:
            B = [[-o.KY, r * o.VY], [o.DY / r, o.TY]]
    elif form == "pmchwt_ext":
        if which == "ext":
            B = [[-o.KY, o.VY], [o.DY, o.TY]]
        else:
            B = [[-o.KL, o.VL / r], [r * o.DL, o.TL]]
    else:
        raise ValueError("Calderon preconditioning is defined for PMCHWT forms")
    return _blocks_to_dense(B)


def half_calderon_scaling(which: str, form: str, phys: Physics):
    """(a, b) of the scaled-mass matrix on top of a half Calderon preconditioner:
    the accumulation points lambda_half,1 = 1/4 + eps_ext/(4 eps_int) and
    lambda_half,2 = 1/4 + eps_int/(4 eps_ext) (paper eq.
    precond:calderon:eigenval_semi), ordered to the block each one lands on."""
    l1 = 0.25 + phys.eps_ext / (4.0 * phys.eps_int)
    l2 = 0.25 + phys.eps_int / (4.0 * phys.eps_ext)
    interior_on_int = (form == "pmchwt_int" and which == "int")
    exterior_on_ext = (form == "pmchwt_ext" and which == "ext")
    if interior_on_int or (form == "pmchwt_ext" and which == "int"):
        return (l1, l2)
    if exterior_on_ext or (form == "pmchwt_int" and which == "ext"):
        return (l2, l1)
    raise ValueError((form, which))


def preconditioner(kind: str, form: str, A: np.ndarray, o: Operators, phys: Physics,
                   a: float | None = None, b: float | None = None) -> np.ndarray:
    """Dense left preconditioner P^-1 (2n x 2n)."""
    n = o.n
    if kind == "none":
        return np.eye(2 * n)
    if kind == "block_diag":
        # paper, algebraic preconditioners: inverse of the diagonals of each block
        d = [np.diag(A[:n, :n]), np.diag(A[:n, n:]), np.diag(A[n:, :n]), np.diag(A[n:, n:])]
        det = d[0] * d[3] - d[1] * d[2]
        P = np.zeros((2 * n, 2 * n))
        idx = np.arange(n)
        P[idx, idx] = d[3] / det
        P[idx, n + idx] = -d[1] / det
        P[n + idx, idx] = -d[2] / det
        P[n + idx, n + idx] = d[0] / det
        return P
    Minv = np.linalg.inv(o.M)  # plain inverse of the (small, SPD) mass matrix
    Z = np.zeros((n, n))
    if kind == "mass":  # paper eq. prec:mass
        return np.block([[Minv, Z], [Z, Minv]])
    if kind == "scaled_mass":  # paper eq. prec:mass:scaled
        return np.block([[Minv / a, Z], [Z, Minv / b]])
    if kind.startswith("calderon_") or kind.startswith("scaled_calderon_"):
        which = kind.split("_")[-1]
        C = A if which == "full" else calderon_blocks(which, form, o, phys)
        MM = np.block([[Minv, Z], [Z, Minv]])
        P = MM @ C @ MM
        if kind.startswith("scaled_"):
            if a is None:
                a, b = half_calderon_scaling(which, form, phys)
            P = np.concatenate([P[:n] / a, P[n:] / b])
        return P
    raise ValueError(kind)


# Table 1 of the paper: case number -> (formulation, preconditioner)
CASES = {
    1: ("direct_int", "none"), 2: ("direct_int", "block_diag"),
    3: ("direct_ext", "none"), 4: ("direct_ext", "block_diag"),
    5: ("direct_int_perm", "none"), 6: ("direct_int_perm", "block_diag"),
    7: ("direct_ext_perm", "none"), 8: ("direct_ext_perm", "block_diag"),
    9: ("juffer", "mass"), 10: ("juffer", "scaled_mass"),
    11: ("lu", "none"), 12: ("lu", "mass"),
    13: ("muller_int", "mass"), 14: ("muller_ext", "mass"),
    15: ("pmchwt_int", "mass"), 16: ("pmchwt_int", "calderon_full"),
    17: ("pmchwt_int", "calderon_int"), 18: ("pmchwt_int", "calderon_ext"),
    19: ("pmchwt_ext", "mass"), 20: ("pmchwt_ext", "calderon_full"),
    21: ("pmchwt_ext", "calderon_ext"), 22: ("pmchwt_ext", "calderon_int"),
    23: ("pmchwt_int", "scaled_calderon_int"), 24: ("pmchwt_int", "scaled_calderon_ext"),
    25: ("pmchwt_ext", "scaled_calderon_ext"), 26: ("pmchwt_ext", "scaled_calderon_int"),
}


def scaled_mass_constants(phys: Physics):
    """Juffer scaled mass: a = 1 + eps_ext/eps_int, b = 1 + eps_int/eps_ext
    (paper, after eq. prec:mass:scaled)."""
    return 1.0 + phys.eps_ext / phys.eps_int, 1.0 + phys.eps_int / phys.eps_ext


# --------------------------------------------------------------------------------------
# Solvers
# --------------------------------------------------------------------------------------

@dataclass
class GmresResult:
    x: np.ndarray
    iters: int
    converged: bool
    history: list = field(default_factory=list)


def gmres(A: np.ndarray, b: np.ndarray, tol: float, max_it: int) -> GmresResult:
    """Unrestarted GMRES on A x = b with x0 = 0: Arnoldi by modified
    Gram-Schmidt, least squares by Givens rotations, stop when the residual
    estimate |g_{k+1}| <= tol * ||b||. (A and b are already preconditioned.)"""
    n = b.shape[0]
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return GmresResult(np.zeros(n), 0, True, [0.0])
    m = min(max_it, n)
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    cs = np.zeros(m)
    sn = np.zeros(m)
    g = np.zeros(m + 1)
    g[0] = beta
    V[0] = b / beta
    hist = [1.0]
    k = 0
    converged = False
    for j in range(m):
        w = A @ V[j]
        for i in range(j + 1):
            H[i, j] = w @ V[i]
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] > 0.0:
            V[j + 1] = w / H[j + 1, j]
        for i in range(j):  # previous rotations on the new column
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        den = np.hypot(H[j, j], H[j + 1, j])
        cs[j] = H[j, j] / den
        sn[j] = H[j + 1, j] / den
        H[j, j] = den
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        res = abs(g[j + 1]) / beta
        hist.append(res)
        if res <= tol or H[j, j] == 0.0:
            converged = res <= tol
            break
    y = scipy.linalg.solve_triangular(H[:k, :k], g[:k])
    x = V[:k].T @ y
    return GmresResult(x, k, converged, hist)


def interior_traces(form: str, x: np.ndarray, phys: Physics):
    """(u_int, v_int) from a solution vector: exterior forms convert with the
    interface conditions u_i = u_e, eps_int v_i = eps_ext v_e (paper eq.
    poissonboltzmann, last two lines)."""
    n = x.shape[0] // 2
    u, v = x[:n], x[n:]
    if form in EXTERIOR_FORMS:
        return u.copy(), v / phys.r
    return u.copy(), v.copy()


@dataclass
class SolveResult:
    x: np.ndarray
    dG: float          # paper units (e^2/A with the 1/(4 pi) of G)
    dG_kcal: float
    iters: int | None
    A: np.ndarray | None = None
    P: np.ndarray | None = None
    b: np.ndarray | None = None


def solve(verts, tris, xq, q, phys: Physics = Physics(), case: int = 2, plan: Plan = Plan(),
          method: str = "lu", tol: float = 1e-12, max_it: int = 1000, ops: Operators | None = None,
          keep: bool = False, form: str | None = None, prec: str | None = None,
          alpha=None, beta=None, nthreads=0) -> SolveResult:
    """Full FP64 solve of one case of Table 1 (or an explicit form/prec)."""
    if form is None:
        form, prec = CASES[case]
    if ops is None:
        ops = assemble(verts, tris, phys.kappa, plan, nthreads=nthreads)
    bD, bN = source_projections(verts, tris, xq, q, phys.eps_int, plan)
    A, b = system(form, ops, phys, bD, bN, alpha, beta)
    a = bb = None
    if prec == "scaled_mass":
        a, bb = scaled_mass_constants(phys)
    P = preconditioner(prec, form, A, ops, phys, a, bb)
    PA = P @ A
    Pb = P @ b
    iters = None
    if method == "lu":
        x = scipy.linalg.lu_solve(scipy.linalg.lu_factor(PA), Pb)
    else:
        res = gmres(PA, Pb, tol, max_it)
        x, iters = res.x, res.iters
    u, v = interior_traces(form, x, phys)
    phi = reaction_potential(verts, tris, u, v, xq, plan)
    dG = 0.5 * float(np.dot(np.asarray(q, dtype=np.float64), phi))
    return SolveResult(x, dG, dG * KCAL_PER_PAPER_UNIT, iters,
                       A if keep else None, P if keep else None, b if keep else None)
