"""The allocation-free system application against the ordinary one.

pb_system_apply_noalloc exists for callers that cannot call cudaMalloc (a
process whose device memory another allocator has reserved, or a loop that
cannot take cudaMalloc's device-wide synchronisation). It keeps its
temporaries in one static device array. This test calls it twice in a row
through the C ABI and compares each result with pb_system_apply in FP32,
within the FP32 tolerance of the parity tests (2e-5 relative). The file is
named to be collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_noalloc_matches_system_apply_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10481_gb300 as pb
    from synth.icosphere import uv_ellipsoid

    v, t = uv_ellipsoid(13, 11, (2.0, 1.6, 1.3), center=(0.3, -0.2, 0.1), twist=0.15)
    ctx = pb.pb_init(0)
    P = pb.Params(4.0, 80.0, 0.125)
    m = pb.pb_mesh_load(ctx, v, t)
    nf = pb.pb_near_build(ctx, m, P.kappa)
    rng = np.random.default_rng(21)
    for form in ("direct_int", "pmchwt_ext"):
        for call in range(2):
            x = torch.as_tensor(rng.standard_normal(2 * len(v)), device="cuda")
            ref = pb.pb_system_apply(ctx, m, nf, P, form, x, pb.PB_F32)
            y = torch.full_like(x, float("nan"))
            pb.pb_system_apply_noalloc(ctx, m, nf, P, form, x, y)
            torch.cuda.synchronize()
            err = float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref))
            print(f"{form} call {call}: rel diff {err:.2e}")
            assert err < 2e-5, (form, call, err)
