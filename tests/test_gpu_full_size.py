"""Parity at the benchmark's full size: the 20-charge sphere (icosphere level 5,
10,242 vertices, 20,480 triangles, 122,880 far-rule points), against the FP64
oracle's dense-LU solutions stored in tests/golden/multi_charge_sphere_oracle.json
(written by tests/golden/make_sphere_oracle.py, which runs only the oracle).

- FP64 GPU solves (tol 1e-10): Delta G within 1e-8 relative; the M-norm of the
  interior Dirichlet trace within 1e-7 (a lower bound of the M-norm error) and
  the traces at 64 sampled vertices within 1e-6 of the trace's RMS value;
- mixed precision (tol 1e-6, the benchmark's setting) for every case the
  sphere workload runs: Delta G within 1e-5 relative;
- for Cases 2, 10 and 20, the whole interior traces of the oracle's solution
  (tests/golden/multi_charge_sphere_traces.npz, same script): the M-norm of
  the difference of the FP64 GPU traces (tol 1e-10) from them within 1e-7 of
  the oracle traces' M-norm, for the Dirichlet and the Neumann trace.
"""
import json
import os
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "multi_charge_sphere_oracle.json")
TRACES = os.path.join(os.path.dirname(__file__), "golden", "multi_charge_sphere_traces.npz")


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10481_gb300 as pb
    return pb


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def setup(pb):
    from synth import multi_charge_sphere
    ctx = pb.pb_init(0)
    v, t, xq, q = multi_charge_sphere()
    m = pb.pb_mesh_load(ctx, v, t)
    nf = pb.pb_near_build(ctx, m, 0.125)
    return ctx, m, nf, torch.as_tensor(xq, device="cuda"), torch.as_tensor(q, device="cuda"), len(v)


def _solve(pb, setup, case, precision, tol):
    ctx, m, nf, xq, q, nv = setup
    P = pb.Params(4.0, 80.0, 0.125)
    form, prec = pb.CASES[case]
    rhs = pb.pb_rhs_charges(ctx, m, xq, q, P, form)
    t0 = time.perf_counter()
    x, info = pb.pb_solve(ctx, m, nf, P, form, prec, rhs,
                          opts=pb.solve_opts(tol=tol, max_it=600, precision=precision, inner_tol=1e-4))
    dG_paper, dG_kcal = pb.pb_energy(ctx, m, x, form, xq, q, P)
    torch.cuda.synchronize()
    return x, info, dG_kcal, time.perf_counter() - t0


def _interior_u(pb, x, form, nv):
    # the Dirichlet trace is continuous across the interface (u_int = u_ext)
    return x[:nv]


@pytest.mark.parametrize("case", [2, 10, 20])
def test_f64_matches_oracle_at_full_size(pb, golden, setup, case):
    ctx, m, nf, xq, q, nv = setup
    ref = golden["cases"][str(case)]
    x, info, dG, dt = _solve(pb, setup, case, pb.PB_F64, 1e-10)
    form = pb.CASES[case][0]
    u = _interior_u(pb, x, form, nv)
    Mu = pb.pb_op_apply(ctx, m, nf, pb.PB_OP_M, pb.PB_LAPLACE, pb.PB_F64, u.contiguous())
    area = float(pb.pb_op_apply(ctx, m, nf, pb.PB_OP_M, pb.PB_LAPLACE, pb.PB_F64,
                                torch.ones(nv, dtype=torch.float64, device="cuda")).sum())
    unorm = float(torch.sqrt(u @ Mu))
    idx = np.asarray(golden["sample_vertices"])
    us = u.cpu().numpy()[idx]
    rms = ref["u_int_M_norm"] / np.sqrt(area)
    e_dG = abs(dG / ref["dG_kcal"] - 1)
    e_norm = abs(unorm / ref["u_int_M_norm"] - 1)
    e_pt = np.abs(us - np.asarray(ref["u_int_sample"])).max() / rms
    print(f"case {case} f64: {info['iters']} iterations in {dt:.1f} s, dG {dG:.10f} (oracle {ref['dG_kcal']:.10f}) "
          f"rel {e_dG:.1e}, ||u||_M rel {e_norm:.1e}, sampled u {e_pt:.1e} of rms")
    assert e_dG < 1e-8
    assert e_norm < 1e-7
    assert e_pt < 1e-6


@pytest.mark.parametrize("case", [2, 10, 12, 13, 14, 15, 19, 20, 23])
def test_mixed_matches_oracle_at_full_size(pb, golden, setup, case):
    ref = golden["cases"][str(case)]
    x, info, dG, dt = _solve(pb, setup, case, pb.PB_MIXED, 1e-6)
    e = abs(dG / ref["dG_kcal"] - 1)
    print(f"case {case} mixed: {info['iters']} iterations, {info['outer_iters']} sweeps in {1e3 * dt:.0f} ms, "
          f"dG rel {e:.1e}")
    assert e < 1e-5


@pytest.mark.parametrize("case", [2, 10, 20])
def test_f64_traces_match_oracle_in_the_m_norm(pb, setup, case):
    """||x_gpu - x_oracle||_M / ||x_oracle||_M <= 1e-7 for both interior traces."""
    ctx, m, nf, xq, q, nv = setup
    ref = np.load(TRACES)
    x, info, dG, dt = _solve(pb, setup, case, pb.PB_F64, 1e-10)
    form = pb.CASES[case][0]
    u = x[:nv].contiguous()
    w = x[nv:].contiguous()
    if form in ("direct_ext", "direct_ext_perm", "cfie_ext", "pmchwt_ext", "muller_ext", "lu"):
        w = w * (80.0 / 4.0)  # interface condition: eps_int v_int = eps_ext v_ext
    for name, a in (("u", u), ("v", w)):
        r = torch.as_tensor(ref[f"{name}_int_{case}"], device="cuda")
        d = (a - r).contiguous()
        Md = pb.pb_op_apply(ctx, m, nf, pb.PB_OP_M, pb.PB_LAPLACE, pb.PB_F64, d)
        Mr = pb.pb_op_apply(ctx, m, nf, pb.PB_OP_M, pb.PB_LAPLACE, pb.PB_F64, r.contiguous())
        e = float(torch.sqrt((d @ Md) / (r @ Mr)))
        print(f"case {case} f64 {name}_int: M-norm of the difference {e:.1e} of the oracle's")
        assert e < 1e-7, (case, name, e)
