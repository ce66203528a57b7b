"""Treecode far field (FP32 applications): accuracy against the exact operator,
convergence with the interpolation order, and mixed-precision solves that
reach the direct solution because the outer residual stays exact.

Tolerance: order 6 with theta 0.7 is a ~1e-5 relative approximation of the
direct far sum (interpolation error of the Chebyshev proxies); the test
bounds the system application's relative L2 error by 1e-4 against the FP64
direct application, requires order 6 to be more accurate than order 3, and
bounds Delta G of a mixed solve by 1e-5 against the FP64 direct solve.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10481_gb300 as pb
    return pb


@pytest.fixture(scope="module")
def sphere(pb):
    from synth import multi_charge_sphere
    ctx = pb.pb_init(0)
    v, t, xq, q = multi_charge_sphere()
    m = pb.pb_mesh_load(ctx, v, t)
    nf = pb.pb_near_build(ctx, m, 0.125)
    return ctx, m, nf, torch.as_tensor(xq, device="cuda"), torch.as_tensor(q, device="cuda")


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("form", ["direct_int", "juffer", "pmchwt_ext"])
def test_tree_application_accuracy(pb, sphere, form):
    ctx, m, nf, _, _ = sphere
    P = pb.Params(4.0, 80.0, 0.125)
    x = torch.randn(2 * m.info()["n_verts"], dtype=torch.float64, device="cuda")
    ref = pb.pb_system_apply(ctx, m, nf, P, form, x, pb.PB_F64)
    pb.pb_set_treecode(ctx, False)
    direct32 = pb.pb_system_apply(ctx, m, nf, P, form, x, pb.PB_F32)
    errs = {}
    for order in (3, 6):
        pb.pb_set_treecode(ctx, True, order, 0.7, 0)
        y = pb.pb_system_apply(ctx, m, nf, P, form, x, pb.PB_F32)
        errs[order] = rel(y, ref)
        # the split-coordinate and FP64 applications stay direct
        assert rel(pb.pb_system_apply(ctx, m, nf, P, form, x, pb.PB_F32_ACCURATE), ref) < 2e-6
    pb.pb_set_treecode(ctx, False)
    info = pb.pb_tree_info(m)
    npts = m.info()["n_points"]
    print(f"{form}: direct FP32 {rel(direct32, ref):.1e}, treecode order 3 {errs[3]:.1e}, order 6 {errs[6]:.1e}; "
          f"tree {info}, pairs {info['direct_pairs'] + info['proxy_pairs']:.3e} of {npts ** 2:.3e}")
    assert errs[6] < 1e-4
    assert errs[6] < errs[3]
    assert info["direct_pairs"] + info["proxy_pairs"] < npts * npts
    # every split leaves a multiple of 128 points on the left: the leaves are full but one per path,
    # ceil(points / 128) of them
    assert info["leaves"] == -(-npts // 128)


def test_tree_mixed_solve_reaches_direct_solution(pb, sphere):
    ctx, m, nf, xq, q = sphere
    P = pb.Params(4.0, 80.0, 0.125)
    form, prec = pb.CASES[10]
    rhs = pb.pb_rhs_charges(ctx, m, xq, q, P, form)
    x64, _ = pb.pb_solve(ctx, m, nf, P, form, prec, rhs, opts=pb.solve_opts(tol=1e-10, max_it=300))
    _, dG64 = pb.pb_energy(ctx, m, x64, form, xq, q, P)
    pb.pb_set_treecode(ctx, True, 6, 0.7, 0)
    for _ in range(2):  # the second solve replays its captured iterations
        x, info = pb.pb_solve(ctx, m, nf, P, form, prec, rhs,
                              opts=pb.solve_opts(tol=1e-6, max_it=300, precision=pb.PB_MIXED))
        _, dG = pb.pb_energy(ctx, m, x, form, xq, q, P)
        print(f"treecode mixed: {info['iters']} iterations, {info['outer_iters']} sweeps, dG rel {abs(dG / dG64 - 1):.1e}")
        assert abs(dG / dG64 - 1) < 1e-5
    pb.pb_set_treecode(ctx, False)


def test_tree_arguments(pb, sphere):
    ctx = sphere[0]
    for bad in [(True, 1, 0.7, 0), (True, 8, 0.7, 0), (True, 6, 0.0, 0), (True, 6, 1.5, 0), (True, 6, 0.7, -1)]:
        with pytest.raises(pb.PBError):
            pb.pb_set_treecode(ctx, *bad)
