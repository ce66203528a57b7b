"""The autotuner (launch choice and quadrature plan)."""
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


def test_launch_tuning_keeps_results(pb):
    from synth import icosphere
    v, t = icosphere(4, 5.0)
    ctx = pb.pb_init(0)
    P = pb.Params(4.0, 80.0, 0.125)
    m = pb.pb_mesh_load(ctx, v, t)
    nf = pb.pb_near_build(ctx, m, P.kappa)
    x = torch.as_tensor(np.random.default_rng(1).standard_normal(2 * len(v)), device="cuda")
    ref = pb.pb_system_apply(ctx, m, nf, P, "juffer", x, pb.PB_F64)
    rr = pb.pb_autotune(ctx, m, nf, P, "juffer")
    print("tuned", rr)
    for r in rr.values():
        assert r["kernel"] in (1, 2) and r["split_scale"] in (0.5, 1.0, 2.0) and 0 <= r["shape"] < 4
        assert r["tile_records"] in (32, 64, 128) and r["targets_per_thread"] in (2, 4)
        assert r["tiles_per_fp64_sum"] in (1, 2, 4)
        assert 0 < r["best_ms"] <= r["default_ms"]
    for prec in (pb.PB_F32, pb.PB_F32_ACCURATE):
        y = pb.pb_system_apply(ctx, m, nf, P, "juffer", x, prec)
        assert float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref)) < 2e-5


def test_plan_tuning_follows_the_rule(pb):
    """The relaxed far rule is accepted only within the stated Delta G change."""
    from synth import kirkwood_sphere
    v, t, xq, q = kirkwood_sphere(3, 2.0)
    ctx = pb.pb_init(0)
    P = pb.Params(4.0, 80.0, 0.125)
    opts = pb.solve_opts(tol=1e-10, max_it=300)
    strict, ch = pb.pb_autotune_plan(ctx, v, t, xq, q, P, "direct_int", "block_diag", tol_dG=1e-9, opts=opts)
    assert strict == {"far_q": 6, "n_ss": 4, "band_eta": 0.0, "band_q": 6, "n_ss_coin": 4, "n_ss_edge": 4,
                      "n_ss_vert": 4} and ch == 0.0
    loose, ch2 = pb.pb_autotune_plan(ctx, v, t, xq, q, P, "direct_int", "block_diag", tol_dG=5e-2, opts=opts)
    print("plans", strict, loose, ch2)
    assert loose["far_q"] == 3 and loose["band_eta"] > 0.0 and loose["band_q"] == 6 and 0.0 < ch2 <= 5e-2
    # a loose tolerance also takes one Gauss point off every class's singular rule
    assert (loose["n_ss_coin"], loose["n_ss_edge"], loose["n_ss_vert"]) == (3, 3, 3)
    # and the reported change is that of the returned plan
    d_ref, _ = pb.pb_solvation_energy(ctx, v, t, xq, q, P, "direct_int", "block_diag", opts=opts)
    d_new, _ = pb.pb_solvation_energy(ctx, v, t, xq, q, P, "direct_int", "block_diag", opts=opts, **loose)
    assert abs(abs(d_new / d_ref - 1) - ch2) < 1e-9
