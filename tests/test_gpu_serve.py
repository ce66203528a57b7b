"""The request server: each result is the same alone and in the mix.

Five synthetic molecules of different sizes with different formulations run
(i) one at a time on a fresh server and (ii) all submitted together on a
server whose device-memory budget admits only part of them at once (the rest
queue and enter as memory frees). The energies must be identical (the batched
pair kernel keeps every request's own decomposition and fixed reduction
order), every request must converge, and each must agree with pb_solve of the
same molecule within the mixed-precision tolerance (1e-5 relative). Each
served Delta G is also checked against the FP64 oracle's dense-LU solve of
the same molecule and case (1e-5 relative), so that a fault common to the
server and pb_solve cannot pass."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

CASES = [(14, 2), (40, 10), (25, 12), (60, 23), (18, 10)]  # (atoms, Table-1 case)


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10481_gb300 as pb
    return pb


@pytest.fixture(scope="module")
def molecules():
    from synth import synthetic_molecule
    return [synthetic_molecule(n, 100 + i)[:4] for i, (n, _) in enumerate(CASES)]


def _run(pb, ctx, mols, idx, budget, max_active=8):
    srv = pb.pb_server_create(ctx, budget, max_active)
    P = pb.Params(4.0, 80.0, 0.125)
    opts = pb.solve_opts(tol=1e-6, max_it=300, precision=pb.PB_MIXED, inner_tol=1e-4)
    for i in idx:
        v, t, xq, q = mols[i]
        form, prec = pb.CASES[CASES[i][1]]
        pb.pb_submit(srv, v, t, xq, q, P, form, prec, opts=opts, tag=i)
    out = {}
    steps, max_active_seen = 0, 0
    while len(out) < len(idx):
        a, p = pb.pb_server_step(srv)
        max_active_seen = max(max_active_seen, a)
        for r in pb.pb_poll(srv):
            out[r["tag"]] = r
        steps += 1
        assert steps < 100000
    srv.free()
    return out, max_active_seen


@pytest.fixture(scope="module")
def served(pb, molecules):
    ctx = pb.pb_init(0)
    alone = {}
    for i in range(len(CASES)):
        r, _ = _run(pb, ctx, molecules, [i], 8 << 30)
        alone.update(r)
    # a budget that holds roughly two of these molecules at a time
    mixed, seen = _run(pb, ctx, molecules, list(range(len(CASES))), 600 << 20, max_active=3)
    return ctx, alone, mixed, seen


def test_server_results_alone_equal_in_mix(pb, molecules, served):
    ctx, alone, mixed, seen = served
    for i in range(len(CASES)):
        a, m = alone[i], mixed[i]
        print(f"request {i}: atoms {CASES[i][0]} case {CASES[i][1]} dG {a['dG_kcal']:.8f} / {m['dG_kcal']:.8f} "
              f"iters {a['iters']}/{m['iters']} latency {m['latency_ms']:.1f} ms queue {m['queue_ms']:.1f} ms")
        assert a["status"] == 0 and m["status"] == 0
        assert a["dG_kcal"] == m["dG_kcal"] and a["iters"] == m["iters"]
    assert 1 <= seen <= 3
    # and the same as the one-call solve
    P = pb.Params(4.0, 80.0, 0.125)
    for i in range(len(CASES)):
        v, t, xq, q = molecules[i]
        form, prec = pb.CASES[CASES[i][1]]
        m_ = pb.pb_mesh_load(ctx, v, t)
        nf = pb.pb_near_build(ctx, m_, 0.125)
        dxq, dq = torch.as_tensor(xq, device="cuda"), torch.as_tensor(q, device="cuda")
        rhs = pb.pb_rhs_charges(ctx, m_, dxq, dq, P, form)
        x, info = pb.pb_solve(ctx, m_, nf, P, form, prec, rhs,
                              opts=pb.solve_opts(tol=1e-6, max_it=300, precision=pb.PB_MIXED))
        _, dGk = pb.pb_energy(ctx, m_, x, form, dxq, dq, P)
        assert abs(mixed[i]["dG_kcal"] / dGk - 1) < 1e-5, (i, mixed[i]["dG_kcal"], dGk)


def test_served_results_match_the_oracle(pb, molecules, served):
    """Every served Delta G against the FP64 oracle (dense assembly, dense LU
    of the preconditioned system) of the same molecule, case and plan."""
    import oracle
    _, _, mixed, _ = served
    phys = oracle.Physics(4.0, 80.0, 0.125)
    for i, (atoms, case) in enumerate(CASES):
        v, t, xq, q = molecules[i]
        ref = oracle.solve(v, t, xq, q, phys, case=case)
        e = abs(mixed[i]["dG_kcal"] / ref.dG_kcal - 1)
        print(f"request {i}: atoms {atoms} case {case} ({len(t)} tris): served {mixed[i]['dG_kcal']:.8f}, "
              f"oracle {ref.dG_kcal:.8f}, rel {e:.1e}")
        assert e < 1e-5, (i, mixed[i]["dG_kcal"], ref.dG_kcal)


def test_server_rejects_what_cannot_fit(pb, molecules):
    ctx = pb.pb_init(0)
    srv = pb.pb_server_create(ctx, 1 << 20, 4)  # 1 MiB
    v, t, xq, q = molecules[0]
    with pytest.raises(pb.PBError) as e:
        pb.pb_submit(srv, v, t, xq, q, pb.Params(), "direct_int", "block_diag")
    assert e.value.code == -3
    srv.free()
