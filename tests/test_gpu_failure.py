"""Failure detection without a GPU fault: a bounded device wait that runs out
(a barrier nothing completes) reports PB_ETIMEOUT through the status word,
the kernel returns normally and the context keeps working."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10481_gb300 as pb
    from synth import icosphere
    ctx = pb.pb_init(0)
    assert pb.pb_selftest_wait(ctx, 4096) == -7  # PB_ETIMEOUT
    torch.cuda.synchronize()
    v, t = icosphere(2, 1.0)
    m = pb.pb_mesh_load(ctx, v, t)
    nf = pb.pb_near_build(ctx, m, 0.125)
    x = torch.ones(len(v), dtype=torch.float64, device="cuda")
    y = pb.pb_op_apply(ctx, m, nf, pb.PB_OP_M, pb.PB_LAPLACE, pb.PB_F64, x)
    area = float(y.sum())
    assert abs(area / (4 * np.pi) - 1) < 0.05
