"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: FP64 operator application 1e-12 relative; FP64 solve Delta G
1e-8 relative and surface potential 1e-7 in the M-norm (GMRES at 1e-12 on the
GPU against dense LU in the oracle); mixed precision 1e-5 relative in Delta G
against the FP64 GPU solve. FP32 pair sums: per-pair rounding of ~1e-7
relative, amplified for the closest point pairs by |x|/|x - y| when the
coordinates are rounded (the split-coordinate variant removes that), hence
2e-5 (fast) and 2e-6 (split coordinates, FP64 tile sums) relative in the
L2 norm on these meshes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import oracle as O
from tests.gpu_common import OPS, PHYS, mesh_case, oracle_ops, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10481_gb300 as pb
    return pb


@pytest.fixture(scope="module")
def ctx(pb):
    return pb.pb_init(0)


_MESHES = {}


def gpu_mesh(pb, ctx, name, far_q=6, n_ss=4):
    key = (name, far_q, n_ss)
    if key not in _MESHES:
        v, t, _, _ = mesh_case(name)
        m = pb.pb_mesh_load(ctx, v, t, far_q=far_q, n_ss=n_ss)
        nf = pb.pb_near_build(ctx, m, PHYS.kappa)
        _MESHES[key] = (m, nf)
    return _MESHES[key]


def params(pb):
    return pb.Params(PHYS.eps_int, PHYS.eps_ext, PHYS.kappa)


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("name", ["ico3", "uv"])
@pytest.mark.parametrize("op", list(OPS))
def test_op_apply_f64(pb, ctx, name, op):
    m, nf = gpu_mesh(pb, ctx, name)
    o = oracle_ops(name)
    A = o.M if op == "M" else getattr(o, op)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(A.shape[0])
    code, kern = OPS[op]
    y = pb.pb_op_apply(ctx, m, nf, code, kern, pb.PB_F64, cuda(x)).cpu().numpy()
    ref = A @ x
    e = rel(y, ref)
    print(f"{name} {op} f64 rel {e:.2e}")
    assert e < 1e-12
    assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max() * 10


@pytest.mark.parametrize("name", ["ico3", "uv"])
@pytest.mark.parametrize("op", ["VL", "KL", "TL", "DL", "VY", "KY", "TY", "DY"])
def test_op_apply_f32(pb, ctx, name, op):
    m, nf = gpu_mesh(pb, ctx, name)
    o = oracle_ops(name)
    A = getattr(o, op)
    x = np.random.default_rng(6).standard_normal(A.shape[0])
    code, kern = OPS[op]
    ref = A @ x
    y32 = pb.pb_op_apply(ctx, m, nf, code, kern, pb.PB_F32, cuda(x)).cpu().numpy()
    yacc = pb.pb_op_apply(ctx, m, nf, code, kern, pb.PB_F32_ACCURATE, cuda(x)).cpu().numpy()
    e32, eacc = rel(y32, ref), rel(yacc, ref)
    print(f"{name} {op} f32 rel {e32:.2e} accurate {eacc:.2e}")
    assert e32 < 2e-5
    assert eacc < 2e-6


SYSTEM_FORMS = ["direct_int", "direct_ext", "direct_int_perm", "juffer", "lu", "muller_int", "muller_ext",
                "pmchwt_int", "pmchwt_ext", "cfie_int", "cfie_ext"]


@pytest.mark.parametrize("form", SYSTEM_FORMS)
def test_system_apply_and_rhs(pb, ctx, form):
    name = "uv"
    m, nf = gpu_mesh(pb, ctx, name)
    o = oracle_ops(name)
    v, t, xq, q = mesh_case(name)
    bD, bN = oracle.source_projections(v, t, xq, q, PHYS.eps_int)
    alpha, beta = (0.7, -1.3) if form.startswith("cfie") else (None, None)
    A, b = O.system(form, o, PHYS, bD, bN, alpha, beta)
    x = np.random.default_rng(7).standard_normal(A.shape[0])
    a_, b_ = (alpha or 0.0), (beta or 0.0)
    y = pb.pb_system_apply(ctx, m, nf, params(pb), form, cuda(x), pb.PB_F64, a_, b_).cpu().numpy()
    assert rel(y, A @ x) < 1e-12
    rhs = pb.pb_rhs_charges(ctx, m, cuda(xq), cuda(q), params(pb), form, a_, b_).cpu().numpy()
    assert rel(rhs, b) < 1e-13


@pytest.mark.parametrize("form", ["direct_int", "juffer", "pmchwt_ext"])
def test_split_fp32_charge_sums(pb, ctx, form):
    """The right-hand side and the energy with FP32 pair arithmetic on split
    coordinates (PB_F32_ACCURATE, the mixed-precision path) against the
    oracle's FP64 projections and reaction potential: 1e-6 relative (per-pair
    FP32 rounding of about 6e-8, summed with FP64 tile sums)."""
    name = "uv"
    m, nf = gpu_mesh(pb, ctx, name)
    o = oracle_ops(name)
    v, t, xq, q = mesh_case(name)
    bD, bN = oracle.source_projections(v, t, xq, q, PHYS.eps_int)
    _, b = O.system(form, o, PHYS, bD, bN)
    rhs = pb.pb_rhs_charges(ctx, m, cuda(xq), cuda(q), params(pb), form, prec=pb.PB_F32_ACCURATE).cpu().numpy()
    e_rhs = rel(rhs, b)
    x = np.random.default_rng(17).standard_normal(2 * len(v))
    u, w = O.interior_traces(form, x, PHYS)
    phi_ref = oracle.reaction_potential(v, t, u, w, xq)
    phi = torch.empty(len(q), dtype=torch.float64, device="cuda")
    _, dG32 = pb.pb_energy(ctx, m, cuda(x), form, cuda(xq), cuda(q), params(pb), phi=phi, prec=pb.PB_F32_ACCURATE)
    _, dG64 = pb.pb_energy(ctx, m, cuda(x), form, cuda(xq), cuda(q), params(pb))
    e_phi = rel(phi.cpu().numpy(), phi_ref)
    print(f"{form}: split FP32 rhs rel {e_rhs:.1e}, phi_reac rel {e_phi:.1e}, dG rel {abs(dG32 / dG64 - 1):.1e}")
    assert e_rhs < 1e-6 and e_phi < 1e-6 and abs(dG32 / dG64 - 1) < 1e-6


def _solve_gpu(pb, ctx, name, case, precision, tol=1e-12, far_q=6):
    m, nf = gpu_mesh(pb, ctx, name, far_q=far_q)
    v, t, xq, q = mesh_case(name)
    form, prec = pb.CASES[case]
    P = params(pb)
    rhs = pb.pb_rhs_charges(ctx, m, cuda(xq), cuda(q), P, form)
    x, info = pb.pb_solve(ctx, m, nf, P, form, prec, rhs,
                          opts=pb.solve_opts(tol=tol, max_it=600, precision=precision, inner_tol=1e-4))
    dG, dGk = pb.pb_energy(ctx, m, x, form, cuda(xq), cuda(q), P)
    return x.cpu().numpy(), dG, info


@pytest.mark.parametrize("name", ["ico2", "uv"])
@pytest.mark.parametrize("case", [1, 2, 4, 6, 9, 10, 12, 13, 14, 16, 19, 20, 22, 23, 25])
def test_solve_f64_matches_oracle_lu(pb, ctx, name, case):
    v, t, xq, q = mesh_case(name)
    ref = oracle.solve(v, t, xq, q, PHYS, case=case, ops=oracle_ops(name))
    x, dG, info = _solve_gpu(pb, ctx, name, case, pb.PB_F64)
    form = pb.CASES[case][0]
    n = len(v)
    M = oracle_ops(name).M
    u_ref, _ = O.interior_traces(form, ref.x, PHYS)
    u_gpu, _ = O.interior_traces(form, x, PHYS)
    mnorm = np.sqrt((u_gpu - u_ref) @ M @ (u_gpu - u_ref) / (u_ref @ M @ u_ref))
    print(f"{name} case {case}: iters {info['iters']} dG {dG:.12e} ref {ref.dG:.12e} "
          f"rel {abs(dG / ref.dG - 1):.1e} potential {mnorm:.1e}")
    assert abs(dG / ref.dG - 1) < 1e-8
    assert mnorm < 1e-7
    assert info["rel_residual"] <= 1e-12


@pytest.mark.parametrize("case", [2, 10, 12, 20, 23])
def test_mixed_matches_f64(pb, ctx, case):
    name = "ico2"
    _, dG64, _ = _solve_gpu(pb, ctx, name, case, pb.PB_F64, tol=1e-10)
    _, dGm, info = _solve_gpu(pb, ctx, name, case, pb.PB_MIXED, tol=1e-6)
    print(f"mixed case {case}: outer {info['outer_iters']} inner iters {info['iters']} "
          f"rel {abs(dGm / dG64 - 1):.1e}")
    assert abs(dGm / dG64 - 1) < 1e-5


def test_kirkwood_sphere_host_entry(pb, ctx):
    """Config 1 end to end from host buffers (pb_solvation_energy): the
    oracle's LU solution to 1e-8 and the Born closed form to the
    discretisation error of level 3."""
    from oracle import closed_forms as cf
    from synth import kirkwood_sphere
    v, t, xq, q = kirkwood_sphere(3, 2.0)
    ref = oracle.solve(v, t, xq, q, PHYS, case=2)
    dGk, info = pb.pb_solvation_energy(ctx, v, t, xq, q, params(pb), "direct_int", "block_diag",
                                       opts=pb.solve_opts(tol=1e-12, max_it=500))
    assert abs(dGk / ref.dG_kcal - 1) < 1e-8
    born = cf.born_energy(2.0, 1.0, 4.0, 80.0, 0.125) * O.KCAL_PER_PAPER_UNIT
    assert abs(dGk / born - 1) < 5e-3


def test_deterministic_applies(pb, ctx):
    m, nf = gpu_mesh(pb, ctx, "uv")
    x = cuda(np.random.default_rng(9).standard_normal(2 * mesh_case("uv")[0].shape[0]))
    for prec in (pb.PB_F64, pb.PB_F32, pb.PB_F32_ACCURATE):
        y1 = pb.pb_system_apply(ctx, m, nf, params(pb), "pmchwt_ext", x, prec)
        y2 = pb.pb_system_apply(ctx, m, nf, params(pb), "pmchwt_ext", x, prec)
        assert torch.equal(y1, y2)


def test_relaxed_plan_matches_oracle(pb, ctx):
    """A different quadrature plan (3-point far rule, 3 Gauss points) is
    matched just as exactly: parity is per plan."""
    name = "uv"
    m, nf = gpu_mesh(pb, ctx, name, far_q=3, n_ss=3)
    o = oracle_ops(name, 3, 3)
    x = np.random.default_rng(8).standard_normal(o.n)
    for op in ("VY", "KL", "DY"):
        code, kern = OPS[op]
        y = pb.pb_op_apply(ctx, m, nf, code, kern, pb.PB_F64, cuda(x)).cpu().numpy()
        assert rel(y, getattr(o, op) @ x) < 1e-12


@pytest.mark.parametrize("orders", [(3, 5, 2), (5, 2, 3), (2, 4, 5)])
def test_per_class_singular_orders_match_oracle(pb, ctx, orders):
    """Plans with a singular order per class of pair (coincident, edge,
    vertex; the edge and vertex classes take their own launches and outer
    tables, with and without the fixed-size inner loop) against the oracle
    assembled with the same plan: every FP64 operator to 1e-12."""
    name = "uv"
    nc, ne, nv_ = orders
    v, t, _, _ = mesh_case(name)
    m = pb.pb_mesh_load(ctx, v, t, far_q=6, n_ss=4, n_ss_coin=nc, n_ss_edge=ne, n_ss_vert=nv_)
    nf = pb.pb_near_build(ctx, m, PHYS.kappa)
    o = oracle.assemble(v, t, PHYS.kappa, O.Plan(6, 4, n_ss_coin=nc, n_ss_edge=ne, n_ss_vert=nv_))
    x = np.random.default_rng(9).standard_normal(o.n)
    for op in ("VL", "KL", "DL", "VY", "KY", "DY", "TY"):
        code, kern = OPS[op]
        y = pb.pb_op_apply(ctx, m, nf, code, kern, pb.PB_F64, cuda(x)).cpu().numpy()
        e = rel(y, getattr(o, op) @ x)
        assert e < 1e-12, (orders, op, e)


def test_errors_are_reported(pb, ctx):
    from synth import icosphere
    v, t = icosphere(1, 1.0)
    with pytest.raises(pb.PBError) as e:  # open surface
        pb.pb_mesh_load(ctx, v, t[:-1])
    assert e.value.code == -2
    with pytest.raises(pb.PBError) as e:  # inward orientation
        pb.pb_mesh_load(ctx, v, t[:, ::-1].copy())
    assert e.value.code == -2
    bad = t.copy()
    bad[3, 1] = len(v) + 5
    with pytest.raises(pb.PBError) as e:
        pb.pb_mesh_load(ctx, v, bad)
    assert e.value.code == -2
    with pytest.raises(pb.PBError) as e:  # no triangles at all
        pb.pb_mesh_load(ctx, v, t[:0])
    assert e.value.code == -2
    with pytest.raises(pb.PBError) as e:
        pb.pb_mesh_load(ctx, v, t, far_q=5)
    assert e.value.code == -1
    with pytest.raises(pb.PBError) as e:  # a per-class singular order out of range
        pb.pb_mesh_load(ctx, v, t, n_ss_vert=13)
    assert e.value.code == -1
    m, nf = gpu_mesh(pb, ctx, "ico2")
    vv, tt, xq, q = mesh_case("ico2")
    P = params(pb)
    rhs = pb.pb_rhs_charges(ctx, m, cuda(xq), cuda(q), P, "direct_int")
    with pytest.raises(pb.PBError) as e:  # Calderon needs a PMCHWT form
        pb.pb_solve(ctx, m, nf, P, "direct_int", "calderon_full", rhs)
    assert e.value.code == -1
    x, info = pb.pb_solve(ctx, m, nf, P, "direct_int", "block_diag", rhs,
                          opts=pb.solve_opts(tol=1e-12, max_it=1), raise_on_noconv=False)
    assert info["status"] == -4 and info["iters"] == 1 and info["rel_residual"] < 1.0
    with pytest.raises(pb.PBError) as e:
        pb.pb_rhs_charges(ctx, m, cuda(xq[:0]), cuda(q[:0]), P, "direct_int")
    assert e.value.code == -1
    with pytest.raises(pb.PBError) as e:  # the charge sums take PB_F64 or PB_F32_ACCURATE only
        pb.pb_rhs_charges(ctx, m, cuda(xq), cuda(q), P, "direct_int", prec=pb.PB_F32)
    assert e.value.code == -1
