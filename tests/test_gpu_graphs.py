"""CUDA-graph replay of GMRES iterations launches the same kernels as the
kernel-by-kernel path: solutions, iteration counts, launch counts and the
profiled pair-kernel launches are identical with graphs on and off, for FP64,
mixed-precision and Calderon solves and for the request server."""
import time

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
def ctx(pb):
    return pb.pb_init(0)


@pytest.fixture(scope="module")
def sphere(pb, ctx):
    from synth import multi_charge_sphere
    v, t, xq, q = multi_charge_sphere(level=3, radius=10.0, n_charges=20, charge_radius=8.0, seed=2)
    m = pb.pb_mesh_load(ctx, v, t)
    nf = pb.pb_near_build(ctx, m, 0.125)
    return m, nf, torch.as_tensor(xq, device="cuda"), torch.as_tensor(q, device="cuda")


def _solve(pb, ctx, sphere, case, precision, graphs, profile=False):
    m, nf, xq, q = sphere
    P = pb.Params(4.0, 80.0, 0.125)
    form, prec = pb.CASES[case]
    rhs = pb.pb_rhs_charges(ctx, m, xq, q, P, form)
    pb.pb_set_graphs(ctx, graphs)
    pb.pb_profile(ctx, profile)
    torch.cuda.synchronize()
    n0 = pb.pb_launch_count()
    t0 = time.perf_counter()
    x, info = pb.pb_solve(ctx, m, nf, P, form, prec, rhs,
                          opts=pb.solve_opts(tol=1e-8 if precision == pb.PB_F64 else 1e-6, max_it=300,
                                             precision=precision))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    launches = pb.pb_launch_count() - n0
    prof = pb.pb_profile_read(ctx, pb.PB_KERNEL_PAIR32) if profile else None
    pb.pb_profile(ctx, False)
    pb.pb_set_graphs(ctx, True)
    return x.cpu().numpy(), info, launches, dt, prof


@pytest.mark.parametrize("case,mixed", [(2, False), (10, True), (20, False), (23, True)])
def test_graph_replay_is_bitwise_the_same(pb, ctx, sphere, case, mixed):
    prec = pb.PB_MIXED if mixed else pb.PB_F64
    _solve(pb, ctx, sphere, case, prec, True)  # warm-up (workspaces, tuning table)
    x0, i0, l0, t0, _ = _solve(pb, ctx, sphere, case, prec, False)
    x1, i1, l1, t1, _ = _solve(pb, ctx, sphere, case, prec, True)
    print(f"case {case} {'mixed' if mixed else 'f64'}: {i1['iters']} iterations, {l1} kernels, "
          f"{1e3 * t0:.1f} ms kernel by kernel, {1e3 * t1:.1f} ms from graphs")
    assert i0["iters"] == i1["iters"] and i0["outer_iters"] == i1["outer_iters"]
    assert i0["system_applies"] == i1["system_applies"]
    assert np.array_equal(x0, x1)
    assert l0 == l1


def test_profiled_launches_are_credited_per_replay(pb, ctx, sphere):
    _, i0, _, _, p0 = _solve(pb, ctx, sphere, 10, pb.PB_MIXED, False, profile=True)
    _, i1, _, _, p1 = _solve(pb, ctx, sphere, 10, pb.PB_MIXED, True, profile=True)
    assert p0["launches"] == p1["launches"] > 2
    assert p0["pairs"] == p1["pairs"]
    assert 0.5 < p1["ms"] / p0["ms"] < 2.0


def test_server_same_with_and_without_graphs(pb, ctx):
    from synth import synthetic_molecule
    mols = [(synthetic_molecule(n, 300 + i)[:4], case) for i, (n, case) in enumerate([(16, 2), (22, 23), (12, 12)])]
    P = pb.Params(4.0, 80.0, 0.125)
    opts = pb.solve_opts(tol=1e-6, max_it=300, precision=pb.PB_MIXED, inner_tol=1e-4)
    res = []
    for graphs in (False, True):
        pb.pb_set_graphs(ctx, graphs)
        srv = pb.pb_server_create(ctx, 8 << 30, 4)
        for i, ((v, t, xq, q), case) in enumerate(mols):
            form, prec = pb.CASES[case]
            pb.pb_submit(srv, v, t, xq, q, P, form, prec, opts=opts, tag=i)
        out = {}
        steps = 0
        while len(out) < len(mols):
            pb.pb_server_step(srv)
            for r in pb.pb_poll(srv):
                out[r["tag"]] = r
            steps += 1
            assert steps < 100000
        srv.free()
        res.append(out)
    pb.pb_set_graphs(ctx, True)
    for i in range(len(mols)):
        a, b = res[0][i], res[1][i]
        assert a["status"] == 0 and b["status"] == 0
        assert a["dG_kcal"] == b["dG_kcal"] and a["iters"] == b["iters"]
