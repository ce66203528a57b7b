"""The allocation-free system application against the ordinary one and the oracle.

pb_system_apply_noalloc exists for callers that cannot call cudaMalloc (a
process whose device memory another allocator has reserved, or a loop that
cannot take cudaMalloc's device-wide synchronisation). It keeps its
temporaries in one static device array. This test calls it twice in a row
through the C ABI and compares each result with pb_system_apply in FP32 and
with the FP64 oracle's dense system, within the FP32 tolerance of the parity
tests (2e-5 relative); it checks that the device's free memory is the same
before and after a call, and that a mesh too large for the array is refused
with PB_EINVAL. The file is named to be collected last so that a run stopping
at the first failure has already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_noalloc_matches_system_apply_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_2108_10481_gb300 as pb
    from oracle import oracle as O
    from tests.gpu_common import PHYS, mesh_case, oracle_ops

    v, t, xq, q = mesh_case("uv")
    ctx = pb.pb_init(0)
    P = pb.Params(4.0, 80.0, 0.125)
    m = pb.pb_mesh_load(ctx, v, t)
    nf = pb.pb_near_build(ctx, m, P.kappa)
    o = oracle_ops("uv")
    bD, bN = oracle.source_projections(v, t, xq, q, PHYS.eps_int)
    rng = np.random.default_rng(21)
    for form in ("direct_int", "pmchwt_ext"):
        A, _ = O.system(form, o, PHYS, bD, bN)
        xs = [rng.standard_normal(2 * len(v)) for _ in range(2)]
        xd = [torch.as_tensor(x, device="cuda") for x in xs]
        refs = [pb.pb_system_apply(ctx, m, nf, P, form, x, pb.PB_F32) for x in xd]
        ys = [torch.full_like(x, float("nan")) for x in xd]
        torch.cuda.synchronize()
        for call in range(2):
            free0 = torch.cuda.mem_get_info()[0]
            pb.pb_system_apply_noalloc(ctx, m, nf, P, form, xd[call], ys[call])
            torch.cuda.synchronize()
            free1 = torch.cuda.mem_get_info()[0]
            y = ys[call]
            err = float(torch.linalg.norm(y - refs[call]) / torch.linalg.norm(refs[call]))
            exact = A @ xs[call]
            err_orc = float(np.linalg.norm(y.cpu().numpy() - exact) / np.linalg.norm(exact))
            print(f"{form} call {call}: rel diff {err:.2e} vs pb_system_apply, {err_orc:.2e} vs oracle, "
                  f"free memory {free0} -> {free1}")
            assert err < 2e-5, (form, call, err)
            assert err_orc < 2e-5, (form, call, err_orc)
            # the first call on the device may map the static array; later calls change nothing
            if call > 0 or form != "direct_int":
                assert free1 == free0, (form, call, free0, free1)


def test_noalloc_refuses_a_mesh_beyond_its_array():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10481_gb300 as pb
    from synth import icosphere

    v, t = icosphere(5, 10.0)  # 20,480 triangles, 122,880 points with the 6-point rule
    ctx = pb.pb_init(0)
    P = pb.Params(4.0, 80.0, 0.125)
    m = pb.pb_mesh_load(ctx, v, t)
    nf = pb.pb_near_build(ctx, m, P.kappa)
    x = torch.ones(2 * len(v), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(pb.PBError) as e:
        pb.pb_system_apply_noalloc(ctx, m, nf, P, "direct_int", x, y)
    assert e.value.code == pb.PB_EINVAL
    assert "scratch" in str(e.value)
    assert float(y.abs().max()) == 0.0  # nothing ran
