"""Several right-hand sides of one system (pb_solve_many): charge sets on the
same atoms, as in pKa calculations. Each solution equals, bit for bit, the
one-at-a-time pb_solve of the same right-hand side (same kernels in the same
order; the set-up, workspace and captured graphs are shared), and matches the
oracle's dense LU (Delta G 1e-8)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from tests.gpu_common import PHYS, mesh_case, oracle_ops

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10481_gb300 as pb
    return pb


def charge_sets(q, k):
    rng = np.random.default_rng(31)
    return [q * (1.0 + 0.5 * rng.standard_normal(q.shape)) for _ in range(k)]


@pytest.mark.parametrize("case,precision", [(2, "f64"), (10, "mixed"), (20, "f64")])
def test_many_rhs_equal_one_at_a_time(pb, case, precision):
    ctx = pb.pb_init(0)
    v, t, xq, q = mesh_case("uv")
    m = pb.pb_mesh_load(ctx, v, t)
    nf = pb.pb_near_build(ctx, m, PHYS.kappa)
    P = pb.Params(PHYS.eps_int, PHYS.eps_ext, PHYS.kappa)
    form, prec = pb.CASES[case]
    prc = pb.PB_F64 if precision == "f64" else pb.PB_MIXED
    opts = pb.solve_opts(tol=1e-12 if prc == pb.PB_F64 else 1e-6, max_it=400, precision=prc)
    qs = charge_sets(q, 4)
    dxq = torch.as_tensor(xq, device="cuda")
    rhs = torch.stack([pb.pb_rhs_charges(ctx, m, dxq, torch.as_tensor(qk, device="cuda"), P, form) for qk in qs])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, infos = pb.pb_solve_many(ctx, m, nf, P, form, prec, rhs, opts=opts)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    singles = [pb.pb_solve(ctx, m, nf, P, form, prec, rhs[k].clone(), opts=opts) for k in range(len(qs))]
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for k, (xk, ik) in enumerate(singles):
        assert torch.equal(X[k], xk)
        assert infos[k]["iters"] == ik["iters"] and infos[k]["status"] == 0
    print(f"case {case} {precision}: {len(qs)} right-hand sides in {1e3 * (t1 - t0):.1f} ms together, "
          f"{1e3 * (t2 - t1):.1f} ms one at a time; iterations {[i['iters'] for i in infos]}")
    if prc == pb.PB_F64:
        k = 2
        ref = oracle.solve(v, t, xq, qs[k], PHYS, case=case, ops=oracle_ops("uv"))
        _, dG = pb.pb_energy(ctx, m, X[k], form, dxq, torch.as_tensor(qs[k], device="cuda"), P)
        assert abs(dG / ref.dG_kcal - 1) < 1e-8
