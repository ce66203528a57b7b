"""The oracle's distance-band quadrature plan.

A plan with a band uses the coarse far rule only on pairs that share no vertex
and whose centroids lie at least band_eta times the sum of their radii apart;
closer pairs take the finer band rule. Pins:
- limits: a band that holds every pair is the fine plan, bit for bit; no band
  is the coarse plan, bit for bit;
- classification: the banded matrices equal the coarse matrices plus, for every
  pair the criterion selects (found here by brute force over all pairs), the
  difference of its fine and coarse blocks; the oracle's count of band pairs
  (which the GPU tests hold the device search to) is the brute-force count;
- convergence: Delta G of the banded plan approaches the reference plan's as
  the band widens (the coarse rule's error falls with distance).
"""
import numpy as np
import pytest

import oracle
from oracle import oracle as O
from synth import icosphere, multi_charge_sphere, uv_ellipsoid

KAPPA = 0.125
NAMES = ("VL", "KL", "DL", "VY", "KY", "DY", "M")


def _mats(ops):
    return [getattr(ops, n) for n in NAMES]


@pytest.fixture(scope="module")
def ellipsoid():
    return uv_ellipsoid(14, 9, (1.6, 1.1, 0.8), (0.1, -0.2, 0.05), 0.3)


def test_band_limits_are_the_plain_plans(ellipsoid):
    v, t = ellipsoid
    fine = _mats(oracle.assemble(v, t, KAPPA, O.Plan(6, 4)))
    coarse = _mats(oracle.assemble(v, t, KAPPA, O.Plan(3, 4)))
    all_in = _mats(oracle.assemble(v, t, KAPPA, O.Plan(3, 4, band_eta=1e6, band_q=6)))
    none_in = _mats(oracle.assemble(v, t, KAPPA, O.Plan(3, 4, band_eta=0.0, band_q=6)))
    for a, b in zip(all_in, fine):
        assert np.array_equal(a, b)
    for a, b in zip(none_in, coarse):
        assert np.array_equal(a, b)
    # the reference rule of a banded plan is its band rule
    xq, q = np.array([[0.1, 0.0, 0.05], [-0.3, 0.2, 0.0]]), np.array([0.7, -0.4])
    for a, b in zip(O.source_projections(v, t, xq, q, 4.0, O.Plan(3, 4, 2.0, 6)),
                    O.source_projections(v, t, xq, q, 4.0, O.Plan(6, 4))):
        assert np.array_equal(a, b)


def _band_pairs(v, t, eta):
    """Every ordered pair sharing no vertex with |c_s - c_t| < eta (rho_s + rho_t)."""
    p = v[t]
    c = p.sum(axis=1) / 3.0
    rho = np.sqrt(((p - c[:, None, :]) ** 2).sum(axis=2).max(axis=1))
    d2 = ((c[:, None, :] - c[None, :, :]) ** 2).sum(axis=2)
    lim = eta * (rho[:, None] + rho[None, :])
    share = (t[:, None, :, None] == t[None, :, None, :]).any(axis=(2, 3))
    return np.argwhere((d2 < lim * lim) & ~share)


@pytest.mark.parametrize("eta", [1.5, 2.5])
def test_band_blocks_are_the_fine_rule_on_selected_pairs(ellipsoid, eta):
    v, t = ellipsoid
    plan_b = O.Plan(3, 4, band_eta=eta, band_q=6)
    banded = _mats(oracle.assemble(v, t, KAPPA, plan_b))
    expect = _mats(oracle.assemble(v, t, KAPPA, O.Plan(3, 4)))
    pairs = _band_pairs(v, t, eta)
    assert 0 < len(pairs) < len(t) * (len(t) - 1)
    for i, j in pairs:
        d = O.pair_blocks(v, t, i, j, KAPPA, O.Plan(6, 4)) - O.pair_blocks(v, t, i, j, KAPPA, O.Plan(3, 4))
        for k in range(6):
            expect[k][np.ix_(t[i], t[j])] += d[k]
        # the single-pair entry point applies the same criterion
        assert np.array_equal(O.pair_blocks(v, t, i, j, KAPPA, plan_b), O.pair_blocks(v, t, i, j, KAPPA, O.Plan(6, 4)))
    for a, b in zip(banded, expect):
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


@pytest.mark.parametrize("eta", [0.0, 1.0, 2.5, 4.0, 1e6])
def test_band_pair_count_is_the_brute_force_count(ellipsoid, eta):
    """The oracle's band-pair count (a C loop over all pairs) against the
    brute-force list above; the widest band holds every pair sharing no
    vertex, counted here from the vertex incidences."""
    v, t = ellipsoid
    n = oracle.band_pair_count(v, t, eta)
    assert n == len(_band_pairs(v, t, eta))
    if eta == 0.0:
        assert n == 0
    if eta == 1e6:
        nt = len(t)
        inc = np.zeros((nt, len(v)), dtype=np.int64)
        inc[np.repeat(np.arange(nt), 3), t.ravel()] = 1
        sharing = int(((inc @ inc.T) > 0).sum())  # ordered pairs with a common vertex, (t, t) included
        assert n == nt * nt - sharing


def test_band_delta_G_approaches_the_reference_plan():
    v, t, xq, q = multi_charge_sphere(level=2, radius=10.0, n_charges=20, charge_radius=8.0, seed=2)
    phys = O.Physics()
    ref = O.solve(v, t, xq, q, phys, case=10).dG
    errs = []
    for eta in (2.0, 3.0, 4.0):
        plan = O.Plan(3, 4, band_eta=eta, band_q=6)
        d = O.solve(v, t, xq, q, phys, case=10, plan=plan).dG
        errs.append(abs(d / ref - 1))
    coarse = abs(O.solve(v, t, xq, q, phys, case=10, plan=O.Plan(3, 4)).dG / ref - 1)
    print("coarse everywhere", coarse, "banded", errs)
    assert coarse > errs[0] > errs[1] > errs[2]
    assert errs[1] < 2e-6
