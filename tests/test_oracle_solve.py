"""Pins of the oracle's solve: Born/Kirkwood closed forms, agreement across
formulations, GMRES against dense LU and SciPy, and the accumulation points
printed in the paper."""
import functools
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
from oracle import closed_forms as cf
from oracle import oracle as O
from synth import icosphere, kirkwood_sphere
from synth.charges import ball_charges

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
PH = O.Physics(GOLD["physics"]["eps_int"], GOLD["physics"]["eps_ext"], GOLD["physics"]["kappa"])


def test_closed_forms_reduce_to_textbook_cases():
    # n = 0 term of the Kirkwood series is the Born energy (centred charge)
    b = cf.born_energy(2.0, 1.0, 4.0, 80.0, 0.125)
    k = cf.kirkwood_energy(2.0, np.zeros((1, 3)), np.ones(1), 4.0, 80.0, 0.125)
    assert abs(k / b - 1) < 1e-14
    # kappa = 0, equal permittivities: no reaction field at all
    assert abs(cf.kirkwood_energy(3.0, [[0.5, 0.2, 0.1]], [1.0], 2.0, 2.0, 0.0)) < 1e-15
    # kappa -> 0 limit is continuous
    xq = np.array([[0.5, 0.2, -0.3], [-0.4, 0.1, 0.6]])
    q = np.array([1.0, -0.6])
    e0 = cf.kirkwood_energy(2.0, xq, q, 4.0, 80.0, 0.0)
    e1 = cf.kirkwood_energy(2.0, xq, q, 4.0, 80.0, 1e-7)
    assert abs(e1 / e0 - 1) < 1e-5
    # classical (kappa = 0) Kirkwood image-series coefficients: C_n = (n+1)(eps_i - eps_e)/(n eps_i + (n+1) eps_e)
    n = 3
    g = -(n + 1.0)
    assert abs(((n + 1) * 4 + 80 * g) / (n * 4 - 80 * g) - (n + 1) * (4 - 80) / (n * 4 + (n + 1) * 80)) < 1e-15
    # config-1 number in kcal/mol
    assert abs(b * O.KCAL_PER_PAPER_UNIT - (-19.9238)) < 1e-3


@pytest.mark.slow
def test_born_energy_converges_at_h2():
    errs = []
    ex = cf.born_energy(2.0, 1.0, PH.eps_int, PH.eps_ext, PH.kappa)
    for lev in (1, 2, 3):
        s = oracle.solve(*kirkwood_sphere(lev, 2.0), PH, case=2)
        errs.append(abs(s.dG / ex - 1))
    assert errs[2] < 5e-3
    assert 3.0 < errs[0] / errs[1] < 5.5 and 3.0 < errs[1] / errs[2] < 5.5, errs


@functools.lru_cache(maxsize=None)
def _setup(level=2, radius=2.0):
    v, t = icosphere(level, radius)
    xq, q = ball_charges(5, 0.75 * radius, 7)
    return v, t, xq, q, oracle.assemble(v, t, PH.kappa)


@pytest.mark.slow
def test_kirkwood_series_off_centre_charges():
    """Five charges off centre: Delta G tends to the Kirkwood series at O(h^2)."""
    errs = []
    for lev in (1, 2, 3):
        v, t = icosphere(lev, 2.0)
        xq, q = ball_charges(5, 1.5, 7)
        ex = cf.kirkwood_energy(2.0, xq, q, PH.eps_int, PH.eps_ext, PH.kappa)
        s = oracle.solve(v, t, xq, q, PH, case=2)
        errs.append(abs(s.dG / ex - 1))
    assert errs[2] < 1e-2
    assert errs[0] / errs[2] > 10.0, errs


@pytest.mark.slow
def test_all_cases_agree_on_delta_G():
    """All 26 cases of Table 1 give the same Delta G to within the
    discretisation spread (the paper reports 0.22% over the 26 cases)."""
    v, t, xq, q, o = _setup()
    vals = np.array([oracle.solve(v, t, xq, q, PH, case=c, ops=o).dG for c in range(1, 27)])
    spread = (vals.max() - vals.min()) / abs(vals.mean())
    gold = GOLD["arginine_dG_spread"]
    assert spread < 5e-3
    assert spread < 2.0 * (gold["max_kcal"] - gold["min_kcal"]) / abs(gold["max_kcal"])
    # formulations that differ only by row order, scaling or preconditioner give the same numbers
    for a, b in [(1, 2), (1, 5), (3, 4), (9, 10), (11, 12), (15, 16), (19, 20), (15, 19)]:
        assert abs(vals[a - 1] / vals[b - 1] - 1) < 1e-9, (a, b)


@pytest.mark.slow
def test_gmres_matches_lu_and_scipy():
    v, t, xq, q, o = _setup()
    for case in (2, 10, 12, 20, 23):
        s = oracle.solve(v, t, xq, q, PH, case=case, ops=o, keep=True)
        g = oracle.solve(v, t, xq, q, PH, case=case, ops=o, method="gmres", tol=1e-12)
        assert np.linalg.norm(g.x - s.x) <= 1e-9 * np.linalg.norm(s.x), case
        # SciPy's GMRES (no restart) on the explicitly preconditioned matrix
        PA, Pb = s.P @ s.A, s.P @ s.b
        for tol in (1e-5, 1e-8):
            mine = oracle.gmres(PA, Pb, tol, 1000)
            count = [0]
            spla.gmres(PA, Pb, rtol=tol, atol=0.0, restart=1000, maxiter=1000,
                       callback=lambda r: count.__setitem__(0, count[0] + 1), callback_type="pr_norm")
            assert abs(mine.iters - count[0]) <= 1, (case, tol, mine.iters, count[0])
            r = np.linalg.norm(Pb - PA @ mine.x) / np.linalg.norm(Pb)
            assert r <= 1.01 * tol


def _evs(case, level=3):
    v, t = icosphere(level, 2.0)
    o = _ops3(level)
    xq, q = np.zeros((1, 3)), np.ones(1)
    s = oracle.solve(v, t, xq, q, PH, case=case, ops=o, keep=True)
    return np.sort(np.linalg.eigvals(s.P @ s.A).real)


@functools.lru_cache(maxsize=None)
def _ops3(level):
    v, t = icosphere(level, 2.0)
    return oracle.assemble(v, t, PH.kappa)


@pytest.mark.slow
def test_accumulation_points_printed_in_the_paper():
    """Eigenvalue clusters of the preconditioned systems sit at the points the
    paper predicts (within 5%, level-3 sphere): the medians of the upper and
    lower halves for two-point cases, the median for one-point cases."""
    ap = GOLD["accumulation_points"]
    n = 642

    def halves(ev):
        return np.median(ev[n:]), np.median(ev[:n])
    hi, lo = halves(_evs(9))          # Juffer + mass
    assert abs(hi / ap["juffer_mass"][0] - 1) < 0.05 and abs(lo / ap["juffer_mass"][1] - 1) < 0.05
    assert abs(np.median(_evs(12)) / ap["lu_mass"][0] - 1) < 0.05        # Lu + mass
    # Juffer + scaled mass with the printed constants a = 1 + eps_e/eps_i, b = 1 + eps_i/eps_e:
    # both identity coefficients 1/2(1 + ...) land on 1/2 (one cluster; a global factor
    # that leaves the GMRES iterates unchanged)
    hi, lo = halves(_evs(10))
    assert abs(hi / (0.5 * ap["scaled"][0]) - 1) < 0.05 and abs(lo / (0.5 * ap["scaled"][0]) - 1) < 0.05
    for case in (16, 20):                                                 # full Calderon
        assert abs(np.median(_evs(case)) / ap["calderon_full"][0] - 1) < 0.05
    for case in (17, 18, 21, 22):                                         # half Calderon
        hi, lo = halves(_evs(case))
        assert abs(hi / ap["calderon_half"][0] - 1) < 0.05 and abs(lo / ap["calderon_half"][1] - 1) < 0.05
    for case in (23, 24, 25, 26):                                         # scaled half Calderon
        assert abs(np.median(_evs(case)) / ap["scaled"][0] - 1) < 0.05


def test_interior_trace_conversion():
    """Exterior unknowns convert with the interface conditions (u_i = u_e,
    eps_int v_i = eps_ext v_e), so interior and exterior direct forms give
    identical interior traces."""
    v, t, xq, q, o = _setup(level=1)
    si = oracle.solve(v, t, xq, q, PH, case=1, ops=o)
    se = oracle.solve(v, t, xq, q, PH, case=3, ops=o)
    ui, vi = O.interior_traces("direct_int", si.x, PH)
    ue, ve = O.interior_traces("direct_ext", se.x, PH)
    assert np.allclose(ui, ue, rtol=1e-9, atol=1e-14) and np.allclose(vi, ve, rtol=1e-9, atol=1e-14)


def test_block_diagonal_preconditioner_inverts_the_per_dof_blocks():
    """Pin of the block-diagonal preconditioner (paper, "Algebraic
    preconditioners": the inverse of the diagonals of each block). For every
    DOF i, P restricted to rows and columns (i, n+i) times A restricted to the
    same positions is the 2x2 identity, and P has no entry anywhere else. A
    wrong inverse (a swapped or mis-signed term, a transposed block) fails the
    first check; a fill outside the per-DOF pattern fails the second. Cases 2,
    4, 6 and 8 (direct and permuted forms, interior and exterior) on the
    level-2 sphere."""
    v, t, xq, q, o = _setup()
    n = o.n
    idx = np.arange(n)
    mask = np.zeros((2 * n, 2 * n), dtype=bool)
    for r0 in (0, n):
        for c0 in (0, n):
            mask[r0 + idx, c0 + idx] = True
    for case in (2, 4, 6, 8):
        s = oracle.solve(v, t, xq, q, PH, case=case, ops=o, keep=True)
        P, A = s.P, s.A
        assert np.all(P[~mask] == 0.0), case
        # the 2x2 blocks of P and of A at (i, n+i), stacked per DOF
        Pb = np.stack([[P[idx, idx], P[idx, n + idx]], [P[n + idx, idx], P[n + idx, n + idx]]]).transpose(2, 0, 1)
        Ab = np.stack([[A[idx, idx], A[idx, n + idx]], [A[n + idx, idx], A[n + idx, n + idx]]]).transpose(2, 0, 1)
        prod = Pb @ Ab
        err = np.abs(prod - np.eye(2)[None]).max()
        assert err < 1e-13, (case, err)
        # and the 2x2 restriction of P A (not only of A) is the identity too: P A's
        # diagonal blocks pick up nothing from A's off-diagonal entries
        PA = P @ A
        PAb = np.stack([[PA[idx, idx], PA[idx, n + idx]], [PA[n + idx, idx], PA[n + idx, n + idx]]])
        assert np.abs(PAb.transpose(2, 0, 1) - np.eye(2)[None]).max() < 1e-13, case


def test_stored_sphere_traces_agree_with_the_stored_samples():
    """The whole traces stored for the full-size GPU parity tests (npz) and the
    samples, M-norms' companions and energies stored with them (json) come
    from the same oracle solves: the traces at the sampled vertices and Delta G
    must agree to rounding."""
    here = os.path.join(os.path.dirname(__file__), "golden")
    js = json.load(open(os.path.join(here, "multi_charge_sphere_oracle.json")))
    tr = np.load(os.path.join(here, "multi_charge_sphere_traces.npz"))
    idx = np.asarray(js["sample_vertices"])
    for case in (2, 10, 20):
        ref = js["cases"][str(case)]
        assert abs(float(tr[f"dG_kcal_{case}"]) / ref["dG_kcal"] - 1) < 1e-12
        for name in ("u", "v"):
            full = tr[f"{name}_int_{case}"]
            samp = np.asarray(ref[f"{name}_int_sample"])
            assert np.abs(full[idx] - samp).max() <= 1e-10 * np.abs(samp).max(), (case, name)
