"""Fast Calderon preconditioning (paper, "Fast Calderon preconditioning",
Cases 20b and 23b): the preconditioner's operator is assembled with relaxed
quadrature (the 1-point far rule and 3 singular Gauss points per dimension)
while the system keeps the reference plan.

- The solution is the system's, whatever the preconditioner: FP64 GPU solves
  against the oracle's dense LU of the reference plan (Delta G 1e-8, surface
  potential 1e-7 in the M-norm), mixed precision within 1e-5.
- The preconditioner is the relaxed one: the GPU's GMRES iteration count
  matches the oracle's GMRES on the same fast-Calderon-preconditioned matrix
  (within one iteration).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import oracle as O
from tests.gpu_common import PHYS, mesh_case, oracle_ops

pytestmark = pytest.mark.gpu

PC_PLAN = (1, 3)  # relaxed far rule and singular rule of the preconditioner


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


_GPU = {}


def meshes(pb, ctx, name):
    if name not in _GPU:
        v, t, _, _ = mesh_case(name)
        m = pb.pb_mesh_load(ctx, v, t)
        mc = pb.pb_mesh_load(ctx, v, t, far_q=PC_PLAN[0], n_ss=PC_PLAN[1])
        _GPU[name] = (m, pb.pb_near_build(ctx, m, PHYS.kappa), mc, pb.pb_near_build(ctx, mc, PHYS.kappa))
    return _GPU[name]


def oracle_fast_iterations(name, case, tol):
    """GMRES iterations of the oracle on P_fast A x = P_fast b."""
    v, t, xq, q = mesh_case(name)
    form, prec = O.CASES[case]
    ops = oracle_ops(name)
    ops_pc = oracle_ops(name, *PC_PLAN)
    bD, bN = oracle.source_projections(v, t, xq, q, PHYS.eps_int)
    A, b = O.system(form, ops, PHYS, bD, bN)
    A_pc, _ = O.system(form, ops_pc, PHYS, bD, bN)
    P = O.preconditioner(prec, form, A_pc, ops_pc, PHYS)
    return O.gmres(P @ A, P @ b, tol, 1000).iters


@pytest.mark.parametrize("name", ["ico3", "uv"])
@pytest.mark.parametrize("case", [20, 23])
def test_fast_calderon_solution_and_iterations(pb, ctx, name, case):
    v, t, xq, q = mesh_case(name)
    m, nf, mc, nc = meshes(pb, ctx, name)
    P = pb.Params(PHYS.eps_int, PHYS.eps_ext, PHYS.kappa)
    form, prec = pb.CASES[case]
    rhs = pb.pb_rhs_charges(ctx, m, cuda(xq), cuda(q), P, form)
    ref = oracle.solve(v, t, xq, q, PHYS, case=case, ops=oracle_ops(name))
    x, info = pb.pb_solve_pc(ctx, m, nf, mc, nc, P, form, prec, rhs, opts=pb.solve_opts(tol=1e-12, max_it=400))
    _, dG = pb.pb_energy(ctx, m, x, form, cuda(xq), cuda(q), P)
    o = oracle_ops(name)
    u_ref, _ = O.interior_traces(form, ref.x, PHYS)
    u, _ = O.interior_traces(form, x.cpu().numpy(), PHYS)
    mn = np.sqrt((u - u_ref) @ o.M @ (u - u_ref) / (u_ref @ o.M @ u_ref))
    assert abs(dG / ref.dG_kcal - 1) < 1e-8 and mn < 1e-7
    # iterations at a moderate tolerance against the oracle's GMRES on the same preconditioned matrix
    _, i_fast = pb.pb_solve_pc(ctx, m, nf, mc, nc, P, form, prec, rhs, opts=pb.solve_opts(tol=1e-8, max_it=400))
    _, i_full = pb.pb_solve(ctx, m, nf, P, form, prec, rhs, opts=pb.solve_opts(tol=1e-8, max_it=400))
    it_orc = oracle_fast_iterations(name, case, 1e-8)
    print(f"{name} case {case}b: dG rel {abs(dG / ref.dG_kcal - 1):.1e}, potential {mn:.1e}, iterations "
          f"fast {i_fast['iters']} (oracle {it_orc}), standard Calderon {i_full['iters']}")
    assert abs(i_fast["iters"] - it_orc) <= 1
    xm, _ = pb.pb_solve_pc(ctx, m, nf, mc, nc, P, form, prec, rhs,
                           opts=pb.solve_opts(tol=1e-6, max_it=400, precision=pb.PB_MIXED))
    _, dGm = pb.pb_energy(ctx, m, xm, form, cuda(xq), cuda(q), P)
    assert abs(dGm / dG - 1) < 1e-5


def test_fast_calderon_argument_errors(pb, ctx):
    m, nf, mc, nc = meshes(pb, ctx, "uv")
    m2, nf2, _, _ = meshes(pb, ctx, "ico3")
    v, t, xq, q = mesh_case("uv")
    P = pb.Params(PHYS.eps_int, PHYS.eps_ext, PHYS.kappa)
    rhs = pb.pb_rhs_charges(ctx, m, cuda(xq), cuda(q), P, "pmchwt_ext")
    with pytest.raises(pb.PBError):  # not a Calderon preconditioner
        pb.pb_solve_pc(ctx, m, nf, mc, nc, P, "pmchwt_ext", "mass", rhs)
    with pytest.raises(pb.PBError):  # another surface
        pb.pb_solve_pc(ctx, m, nf, m2, nf2, P, "pmchwt_ext", "calderon_full", rhs)
    with pytest.raises(pb.PBError):  # near field of another mesh
        pb.pb_solve_pc(ctx, m, nf, mc, nf, P, "pmchwt_ext", "calderon_full", rhs)
