"""Distance-band quadrature plans on the GPU, against the oracle under the same
plan (through the C ABI).

Plan (3, 4, eta, 6): 3-point far rule for pairs farther apart than eta times
the sum of their radii, the 6-point rule inside the band, 4^4 singular rule,
6-point right-hand side and energy. Tolerances as for the reference plan:
FP64 operators 1e-12, FP32 2e-5 and split-coordinate FP32 2e-6, FP64 solves
Delta G 1e-8 and potential 1e-7 (M-norm), mixed 1e-5. At the benchmark's full
size (20-charge sphere, 20,480 triangles) the banded plan's Delta G is checked
against the stored reference-plan oracle within the benchmark's 1e-5.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import oracle as O
from tests.gpu_common import OPS, PHYS, mesh_case, rel

pytestmark = pytest.mark.gpu

BAND = (3, 4, 2.5, 6)


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10481_gb300 as pb
    return pb


@pytest.fixture(scope="module")
def ctx(pb):
    return pb.pb_init(0)


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def plan(p):
    return O.Plan(far_q=p[0], n_ss=p[1], band_eta=p[2], band_q=p[3])


_CACHE = {}


def gpu(pb, ctx, name, p=BAND):
    if (name, p) not in _CACHE:
        v, t, _, _ = mesh_case(name)
        m = pb.pb_mesh_load(ctx, v, t, far_q=p[0], n_ss=p[1], band_eta=p[2], band_q=p[3])
        _CACHE[(name, p)] = (m, pb.pb_near_build(ctx, m, PHYS.kappa))
    return _CACHE[(name, p)]


_ORC = {}


def orc(name, p=BAND):
    if (name, p) not in _ORC:
        v, t, _, _ = mesh_case(name)
        _ORC[(name, p)] = oracle.assemble(v, t, PHYS.kappa, plan(p))
    return _ORC[(name, p)]


@pytest.mark.parametrize("name", ["ico3", "uv"])
def test_band_operators_match_oracle(pb, ctx, name):
    m, nf = gpu(pb, ctx, name)
    o = orc(name)
    x = np.random.default_rng(21).standard_normal(o.n)
    for op in ("VL", "KL", "TL", "DL", "VY", "KY", "TY", "DY"):
        A = getattr(o, op)
        code, kern = OPS[op]
        ref = A @ x
        y64 = pb.pb_op_apply(ctx, m, nf, code, kern, pb.PB_F64, cuda(x)).cpu().numpy()
        y32 = pb.pb_op_apply(ctx, m, nf, code, kern, pb.PB_F32, cuda(x)).cpu().numpy()
        yac = pb.pb_op_apply(ctx, m, nf, code, kern, pb.PB_F32_ACCURATE, cuda(x)).cpu().numpy()
        e64, e32, eac = rel(y64, ref), rel(y32, ref), rel(yac, ref)
        print(f"{name} {op} band f64 {e64:.1e} f32 {e32:.1e} accurate {eac:.1e}")
        assert e64 < 1e-12 and e32 < 2e-5 and eac < 2e-6


def test_band_differs_from_both_plain_plans(pb, ctx):
    """The banded operator is neither the coarse nor the fine plan's (the band is not empty and not everything)."""
    v, t, _, _ = mesh_case("uv")
    o_b, o_c, o_f = orc("uv"), oracle.assemble(v, t, PHYS.kappa, O.Plan(3, 4)), oracle.assemble(v, t, PHYS.kappa)
    m, nf = gpu(pb, ctx, "uv")
    x = np.random.default_rng(22).standard_normal(o_b.n)
    y = pb.pb_op_apply(ctx, m, nf, 0, 1, pb.PB_F64, cuda(x)).cpu().numpy()
    assert rel(y, o_b.VY @ x) < 1e-12
    assert rel(y, o_c.VY @ x) > 1e-8 and rel(y, o_f.VY @ x) > 1e-8
    mc, _ = gpu(pb, ctx, "uv", (3, 4, 0.0, 6))
    ib, ic = m.info(), mc.info()
    print("band mesh", ib, "coarse mesh", ic)
    assert ib["n_pairs"] > ic["n_pairs"] and ib["nnz"] > ic["nnz"] and ib["n_points"] == ic["n_points"]


@pytest.mark.parametrize("p,ref", [((3, 4, 64.0, 6), (6, 4, 0.0, 6)), ((3, 4, 0.3, 6), None)])
def test_band_limits(pb, ctx, p, ref):
    """A band holding every pair is the fine plan; a band holding none is the
    coarse far rule with the fine right-hand side rule."""
    name = "ico2"
    m, nf = gpu(pb, ctx, name, p)
    o = orc(name, p)
    if ref is not None:
        o_ref = orc(name, ref)
        assert all(np.array_equal(getattr(o, k), getattr(o_ref, k)) for k in ("VL", "KL", "DL", "VY", "KY", "DY"))
    x = np.random.default_rng(23).standard_normal(o.n)
    for op in ("KL", "DY"):
        code, kern = OPS[op]
        y = pb.pb_op_apply(ctx, m, nf, code, kern, pb.PB_F64, cuda(x)).cpu().numpy()
        assert rel(y, getattr(o, op) @ x) < 1e-12


@pytest.mark.parametrize("case", [2, 10, 20])
def test_band_solve_matches_oracle_lu(pb, ctx, case):
    name = "uv"
    v, t, xq, q = mesh_case(name)
    m, nf = gpu(pb, ctx, name)
    ref = oracle.solve(v, t, xq, q, PHYS, case=case, plan=plan(BAND), ops=orc(name))
    P = pb.Params(PHYS.eps_int, PHYS.eps_ext, PHYS.kappa)
    form, prec = pb.CASES[case]
    rhs = pb.pb_rhs_charges(ctx, m, cuda(xq), cuda(q), P, form)
    bD, bN = oracle.source_projections(v, t, xq, q, PHYS.eps_int, plan(BAND))
    _, b = O.system(form, orc(name), PHYS, bD, bN)
    assert rel(rhs.cpu().numpy(), b) < 1e-13
    x, info = pb.pb_solve(ctx, m, nf, P, form, prec, rhs, opts=pb.solve_opts(tol=1e-12, max_it=400))
    _, dG = pb.pb_energy(ctx, m, x, form, cuda(xq), cuda(q), P)
    o = orc(name)
    u_ref, _ = O.interior_traces(form, ref.x, PHYS)
    u, _ = O.interior_traces(form, x.cpu().numpy(), PHYS)
    mn = np.sqrt((u - u_ref) @ o.M @ (u - u_ref) / (u_ref @ o.M @ u_ref))
    print(f"band case {case}: dG {dG:.10f} oracle {ref.dG_kcal:.10f} rel {abs(dG / ref.dG_kcal - 1):.1e} potential {mn:.1e}")
    assert abs(dG / ref.dG_kcal - 1) < 1e-8 and mn < 1e-7
    x2, _ = pb.pb_solve(ctx, m, nf, P, form, prec, rhs, opts=pb.solve_opts(tol=1e-6, max_it=400,
                                                                             precision=pb.PB_MIXED))
    _, dG2 = pb.pb_energy(ctx, m, x2, form, cuda(xq), cuda(q), P)
    assert abs(dG2 / dG - 1) < 1e-5


def test_near_kernels_are_profiled(pb, ctx):
    """The near-field kernels report their timed launches per build (the adjacent-pair kernel one per
    class: edge- and vertex-adjacent pairs), with their point-pair counts."""
    v, t, _, _ = mesh_case("uv")
    m = pb.pb_mesh_load(ctx, v, t, far_q=3, n_ss=4, band_eta=2.5, band_q=6)
    pb.pb_profile(ctx, True)
    nf = pb.pb_near_build(ctx, m, PHYS.kappa)
    stats = {k: pb.pb_profile_read(ctx, k) for k in (pb.PB_KERNEL_NEAR_ADJ, pb.PB_KERNEL_NEAR_COIN,
                                                      pb.PB_KERNEL_NEAR_BAND)}
    pb.pb_profile(ctx, False)
    info = m.info()
    for k, st in stats.items():
        want = 2 if k == pb.PB_KERNEL_NEAR_ADJ else 1
        assert st["launches"] == want and st["ms"] > 0 and st["pairs"] > 0 and st["ops"] > st["pairs"], (k, st)
    # coincident pairs: one per triangle, 3 regions of 4^4 points and 15 far-rule pairs (3-point rule: 3)
    assert stats[pb.PB_KERNEL_NEAR_COIN]["pairs"] == info["n_tris"] * (3 * 256 + 3)
    del nf


@pytest.mark.parametrize("name,eta", [("uv", 2.5), ("ico3", 3.0), ("protein500", 3.0)])
def test_band_search_finds_the_oracle_pairs(pb, ctx, name, eta):
    """The device band search (FP32 prefilter, then the exact FP64 test) lists
    as many pairs as the oracle's loop over all pairs selects: the banded mesh
    holds that many pairs more than the plain one."""
    if name == "protein500":
        from synth import protein_like_500
        v, t, _, _, _ = protein_like_500()
    else:
        v, t, _, _ = mesh_case(name)
    mb = pb.pb_mesh_load(ctx, v, t, far_q=3, n_ss=4, band_eta=eta, band_q=6)
    m0 = pb.pb_mesh_load(ctx, v, t, far_q=3, n_ss=4, band_eta=0.0, band_q=6)
    n_gpu = mb.info()["n_pairs"] - m0.info()["n_pairs"]
    n_orc = oracle.band_pair_count(v, t, eta)
    print(f"{name} eta {eta}: band pairs GPU {n_gpu} oracle {n_orc}")
    assert n_gpu == n_orc > 0


def test_band_plan_errors(pb, ctx):
    v, t, _, _ = mesh_case("ico2")
    for bad in [dict(far_q=6, band_eta=2.0, band_q=6), dict(far_q=3, band_eta=-1.0), dict(far_q=3, band_eta=2.0,
                                                                                          band_q=4)]:
        with pytest.raises(pb.PBError):
            pb.pb_mesh_load(ctx, v, t, **bad)


def test_band_full_size_within_metric_tolerance(pb, ctx):
    """The 20-charge sphere with the 3-point far rule beyond 3 radii: mixed-precision
    Delta G within 1e-5 of the reference-plan oracle (stored dense-LU result)."""
    from synth import multi_charge_sphere
    with open(os.path.join(os.path.dirname(__file__), "golden", "multi_charge_sphere_oracle.json")) as f:
        gold = json.load(f)
    v, t, xq, q = multi_charge_sphere()
    m = pb.pb_mesh_load(ctx, v, t, far_q=3, n_ss=4, band_eta=3.0, band_q=6)
    nf = pb.pb_near_build(ctx, m, PHYS.kappa)
    P = pb.Params(PHYS.eps_int, PHYS.eps_ext, PHYS.kappa)
    for case in (10, 2, 20):
        form, prec = pb.CASES[case]
        rhs = pb.pb_rhs_charges(ctx, m, cuda(xq), cuda(q), P, form)
        x, info = pb.pb_solve(ctx, m, nf, P, form, prec, rhs,
                              opts=pb.solve_opts(tol=1e-6, max_it=400, precision=pb.PB_MIXED))
        _, dG = pb.pb_energy(ctx, m, x, form, cuda(xq), cuda(q), P)
        e = abs(dG / gold["cases"][str(case)]["dG_kcal"] - 1)
        print(f"band (3,4,3,6) case {case}: {info['iters']} iterations, dG {dG:.8f}, vs reference-plan oracle {e:.1e}")
        assert e < 1e-5
