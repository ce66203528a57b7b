"""Accuracy of the mixed-precision path on the large synthetic molecules.

- the 5,000-atom molecule (about 223k triangles, the benchmark's workload):
  the mixed solve at the benchmark's tolerance (1e-6) against the same path
  refined to its own accuracy limit (sweeps until the split-coordinate outer
  residual reaches 1e-10 or stops falling), Delta G within 1e-5 relative, for
  the Juffer form with scaled mass (Case 10) and the direct form with the
  block-diagonal preconditioner (Case 2); for Case 2 also the residual of both
  solutions on 12 rows of the FP64 oracle's system (operator rows by
  assemble_rows, right-hand side rows from the triangles around those
  vertices), which measures the refined solution's error against the FP64
  definition directly;
- the 500-atom molecule (about 40k triangles): the mixed solve against the
  plain FP64 GPU solve (tol 1e-8), Delta G within 1e-5 relative (Case 10).

Both use the benchmark's distance-band plan (3-point far rule beyond 3 radii,
6-point rule inside; 4 singular Gauss points), on both sides of every check.
"""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import oracle as O
from tests.gpu_common import PHYS

pytestmark = pytest.mark.gpu

PLAN = {"far_q": 3, "n_ss": 4, "band_eta": 3.0, "band_q": 6}
ORACLE_PLAN = O.Plan(3, 4, 3.0, 6)


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
def p5000():
    from synth import protein_like_5000
    v, t, pos, q, _ = protein_like_5000()
    return v, t, pos, q


@functools.lru_cache(maxsize=None)
def p500():
    from synth import protein_like_500
    v, t, pos, q, _ = protein_like_500()
    return v, t, pos, q


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _params(pb):
    return pb.Params(PHYS.eps_int, PHYS.eps_ext, PHYS.kappa)


_GPU = {}


def _mesh(pb, ctx, name):
    if name not in _GPU:
        v, t, _, _ = p5000() if name == "p5000" else p500()
        m = pb.pb_mesh_load(ctx, v, t, **PLAN)
        nf = pb.pb_near_build(ctx, m, PHYS.kappa)
        _GPU[name] = (m, nf)
    return _GPU[name]


def _solve(pb, ctx, name, case, opts, raise_on_noconv=True):
    v, t, xq, q = p5000() if name == "p5000" else p500()
    m, nf = _mesh(pb, ctx, name)
    form, prec = pb.CASES[case]
    rhs = pb.pb_rhs_charges(ctx, m, cuda(xq), cuda(q), _params(pb), form)
    x, info = pb.pb_solve(ctx, m, nf, _params(pb), form, prec, rhs, opts=opts, raise_on_noconv=raise_on_noconv)
    _, dG = pb.pb_energy(ctx, m, x, form, cuda(xq), cuda(q), _params(pb))
    return x.cpu().numpy(), dG, info


def _mixed(pb, tol=1e-6):
    return pb.solve_opts(tol=tol, max_it=600, precision=pb.PB_MIXED, inner_tol=1e-4)


def _refined(pb):
    return pb.solve_opts(tol=1e-10, max_it=600, precision=pb.PB_MIXED, inner_tol=1e-4, max_outer=12)


def test_config4_mixed_matches_refined_case10(pb, ctx):
    _, dG, info = _solve(pb, ctx, "p5000", 10, _mixed(pb))
    _, dGr, infor = _solve(pb, ctx, "p5000", 10, _refined(pb), raise_on_noconv=False)
    e = abs(dG / dGr - 1)
    print(f"p5000 case 10: mixed {info['iters']} iterations / {info['outer_iters']} sweeps, dG {dG:.10f}; refined "
          f"{infor['outer_iters']} sweeps to residual {infor['rel_residual']:.1e}, dG {dGr:.10f}; rel {e:.1e}")
    assert info["status"] == 0
    # the refinement stops where its split-coordinate outer residual stops falling (its own
    # accuracy, about 2e-8 here: FP32 pair arithmetic on FP32-rounded source densities)
    assert infor["rel_residual"] < 1e-7
    assert e < 1e-5


@functools.lru_cache(maxsize=None)
def _p5000_rows():
    """12 seeded vertex rows of every operator and of the charge projections
    under the band plan, from the FP64 oracle."""
    v, t, xq, q = p5000()
    rows = np.sort(np.random.default_rng(44).choice(len(v), size=12, replace=False))
    R = oracle.assemble_rows(v, t, rows, PHYS.kappa, ORACLE_PLAN)
    # the projections of vertex i only involve the triangles around i, so the
    # oracle's loop over just those triangles gives rows i exactly
    around = np.any(np.isin(t, rows), axis=1)
    bD, bN = oracle.source_projections(v, t[around], xq, q, PHYS.eps_int, ORACLE_PLAN)
    return rows, R, bD[rows], bN[rows]


def test_config4_direct_form_residual_on_oracle_rows(pb, ctx):
    """Case 2 (direct interior form, V and K rows): the residual b - A x of the
    GPU solutions on 12 rows of the oracle's FP64 system, relative to the
    largest right-hand side entry."""
    v, t, xq, q = p5000()
    n = len(v)
    r = PHYS.r
    rows, R, bD, bN = _p5000_rows()
    x, dG, info = _solve(pb, ctx, "p5000", 2, _mixed(pb))
    xr, dGr, infor = _solve(pb, ctx, "p5000", 2, _refined(pb), raise_on_noconv=False)
    # interior direct form: [1/2 M + K_L, -V_L; 1/2 M - K_Y, r V_Y] [u; v] = [b_D; 0]
    scale = np.abs(bD).max()

    def residual(z):
        r1 = (0.5 * R["M"] + R["KL"]) @ z[:n] - R["VL"] @ z[n:] - bD
        r2 = (0.5 * R["M"] - R["KY"]) @ z[:n] + r * R["VY"] @ z[n:]
        return max(np.abs(r1).max(), np.abs(r2).max()) / scale

    res, resr = residual(x), residual(xr)
    e = abs(dG / dGr - 1)
    print(f"p5000 case 2: mixed {info['iters']} iterations, dG {dG:.10f}, oracle-row residual {res:.1e}; refined "
          f"{infor['outer_iters']} sweeps (library residual {infor['rel_residual']:.1e}), dG {dGr:.10f}, "
          f"oracle-row residual {resr:.1e}; dG rel {e:.1e}")
    assert res < 1e-5
    assert resr < 1e-6
    assert e < 1e-5


def test_config3_mixed_matches_f64_gpu(pb, ctx):
    _, dG, info = _solve(pb, ctx, "p500", 10, _mixed(pb))
    _, dG64, info64 = _solve(pb, ctx, "p500", 10, pb.solve_opts(tol=1e-8, max_it=600))
    e = abs(dG / dG64 - 1)
    print(f"p500 case 10: mixed {info['iters']} iterations dG {dG:.10f}; FP64 {info64['iters']} iterations in "
          f"{info64['time_ms'] / 1e3:.1f} s dG {dG64:.10f}; rel {e:.1e}")
    assert e < 1e-5
