"""GPU path on synthetic protein-like molecules (through the C ABI).

- a 12-atom molecule (3,700 triangles): FP64 solves against the oracle's dense
  LU (Delta G 1e-8 relative, potential 1e-7 in the M-norm) and mixed precision
  against the FP64 GPU solve (1e-5);
- the 500-atom molecule (~40k triangles; no closed form, the dense oracle is
  too large for a test): operator rows against the oracle's row sample
  (FP64 1e-12, split-coordinate FP32 2e-6), the residual of the mixed-precision
  solution on sampled rows of the oracle's system, and agreement of Delta G
  across formulations within the discretisation spread.
"""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import oracle as O
from tests.gpu_common import OPS, PHYS

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


@functools.lru_cache(maxsize=None)
def small():
    from synth import synthetic_molecule
    v, t, pos, q, _ = synthetic_molecule(12, 7)
    return v, t, pos, q


@functools.lru_cache(maxsize=None)
def p500():
    from synth import protein_like_500
    v, t, pos, q, _ = protein_like_500()
    return v, t, pos, q


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def P(pb):
    return pb.Params(PHYS.eps_int, PHYS.eps_ext, PHYS.kappa)


def solve(pb, ctx, m, nf, xq, q, case, precision, tol):
    form, prec = pb.CASES[case]
    rhs = pb.pb_rhs_charges(ctx, m, cuda(xq), cuda(q), P(pb), form)
    x, info = pb.pb_solve(ctx, m, nf, P(pb), form, prec, rhs,
                          opts=pb.solve_opts(tol=tol, max_it=800, precision=precision, inner_tol=1e-4))
    dG, _ = pb.pb_energy(ctx, m, x, form, cuda(xq), cuda(q), P(pb))
    return x.cpu().numpy(), dG, info, rhs.cpu().numpy()


@pytest.mark.parametrize("case", [2, 10, 20])
def test_small_molecule_matches_oracle_lu(pb, ctx, case):
    v, t, xq, q = small()
    ops = _small_ops()
    ref = oracle.solve(v, t, xq, q, PHYS, case=case, ops=ops)
    m = pb.pb_mesh_load(ctx, v, t)
    nf = pb.pb_near_build(ctx, m, PHYS.kappa)
    x, dG, info, _ = solve(pb, ctx, m, nf, xq, q, case, pb.PB_F64, 1e-12)
    form = pb.CASES[case][0]
    u_ref, _ = O.interior_traces(form, ref.x, PHYS)
    u, _ = O.interior_traces(form, x, PHYS)
    mn = np.sqrt((u - u_ref) @ ops.M @ (u - u_ref) / (u_ref @ ops.M @ u_ref))
    print(f"small molecule case {case}: {info['iters']} iterations, dG rel {abs(dG / ref.dG - 1):.1e}, potential {mn:.1e}")
    assert abs(dG / ref.dG - 1) < 1e-8 and mn < 1e-7
    _, dGm, infom, _ = solve(pb, ctx, m, nf, xq, q, case, pb.PB_MIXED, 1e-6)
    assert abs(dGm / dG - 1) < 1e-5


@functools.lru_cache(maxsize=None)
def _small_ops():
    v, t, _, _ = small()
    return oracle.assemble(v, t, PHYS.kappa)


@functools.lru_cache(maxsize=None)
def _p500_gpu(pb, ctx):
    v, t, _, _ = p500()
    m = pb.pb_mesh_load(ctx, v, t)
    nf = pb.pb_near_build(ctx, m, PHYS.kappa)
    return m, nf


@functools.lru_cache(maxsize=None)
def _p500_rows():
    v, t, _, _ = p500()
    rows = np.sort(np.random.default_rng(3).choice(len(v), size=12, replace=False))
    return rows, oracle.assemble_rows(v, t, rows, PHYS.kappa)


def test_protein_like_500_operator_rows(pb, ctx):
    v, t, _, _ = p500()
    m, nf = _p500_gpu(pb, ctx)
    rows, R = _p500_rows()
    x = np.random.default_rng(4).standard_normal(len(v))
    for op in ("VL", "KL", "DL", "VY", "KY", "DY"):
        code, kern = OPS[op]
        ref = R[op] @ x
        yacc = pb.pb_op_apply(ctx, m, nf, code, kern, pb.PB_F32_ACCURATE, cuda(x)).cpu().numpy()[rows]
        e = np.linalg.norm(yacc - ref) / np.linalg.norm(ref)
        print(f"p500 {op} split-coordinate FP32 rows rel {e:.1e}")
        assert e < 2e-6
    # one FP64 system application (direct form: V and K of both kernels, and M)
    xx = np.random.default_rng(5).standard_normal(2 * len(v))
    y = pb.pb_system_apply(ctx, m, nf, P(pb), "direct_int", cuda(xx), pb.PB_F64).cpu().numpy()
    n = len(v)
    r = PHYS.r
    ref1 = (0.5 * R["M"] + R["KL"]) @ xx[:n] - R["VL"] @ xx[n:]
    ref2 = (0.5 * R["M"] - R["KY"]) @ xx[:n] + r * R["VY"] @ xx[n:]
    e1 = np.linalg.norm(y[rows] - ref1) / np.linalg.norm(ref1)
    e2 = np.linalg.norm(y[n + rows] - ref2) / np.linalg.norm(ref2)
    print(f"p500 direct_int FP64 rows rel {e1:.1e} {e2:.1e}")
    assert e1 < 1e-12 and e2 < 1e-12


def test_protein_like_500_solve(pb, ctx):
    """Mixed-precision solution of the direct form: its residual on the
    oracle's sampled rows; Delta G of the direct and Juffer forms agree
    within the discretisation spread."""
    v, t, xq, q = p500()
    m, nf = _p500_gpu(pb, ctx)
    rows, R = _p500_rows()
    x2, dG2, info2, rhs2 = solve(pb, ctx, m, nf, xq, q, 2, pb.PB_MIXED, 1e-6)
    n = len(v)
    r = PHYS.r
    res1 = (0.5 * R["M"] + R["KL"]) @ x2[:n] - R["VL"] @ x2[n:] - rhs2[rows]
    res2 = (0.5 * R["M"] - R["KY"]) @ x2[:n] + r * R["VY"] @ x2[n:] - rhs2[n + rows]
    scale = np.abs(rhs2[:n]).max()
    print(f"p500 case 2 mixed: {info2['iters']} iterations, {info2['outer_iters']} sweeps, "
          f"row residual {np.abs(res1).max() / scale:.1e} {np.abs(res2).max() / scale:.1e}, dG {dG2:.6e}")
    assert np.abs(res1).max() < 1e-5 * scale and np.abs(res2).max() < 1e-5 * scale
    _, dG10, info10, _ = solve(pb, ctx, m, nf, xq, q, 10, pb.PB_MIXED, 1e-6)
    print(f"p500 case 10 mixed: {info10['iters']} iterations, dG {dG10:.6e}, spread {abs(dG10 / dG2 - 1):.1e}")
    assert abs(dG10 / dG2 - 1) < 5e-3
