"""The exponential of the FP64 near-field kernels (the Yukawa factor
e^{-kappa r}): a table-driven e^x for x <= 0 after Tang (ACM TOMS 15(2), 1989),
written from the method. It must agree with CUDA's own exp (torch.exp on the
device) and with the host libm within 2 units in the last place over the range
the kernels meet, give exactly 1 at 0 and 0 below -700."""
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


def ulps(y, ref):
    return np.abs(y - ref) / np.spacing(np.abs(ref))


def test_exp_within_two_ulp(pb):
    ctx = pb.pb_init(0)
    rng = np.random.default_rng(5)
    ln2_32 = np.log(2.0) / 32
    x = np.concatenate([
        -np.linspace(0.0, 60.0, 400001),                   # kappa r of near and band pairs and beyond
        -rng.uniform(0.0, 700.0, 200000),                  # the whole normal range
        -np.arange(0, 20000) * ln2_32,                     # reduction boundaries n ln2/32
        -(np.arange(0, 20000) + 0.5) * ln2_32,             # and the points halfway between
        -np.logspace(-300, 0, 2000),                       # tiny arguments
    ])
    x = x[x >= -700.0]
    dx = torch.as_tensor(x, device="cuda")
    y = pb.pb_selftest_exp(ctx, dx).cpu().numpy()
    cuda_ref = torch.exp(dx).cpu().numpy()
    host_ref = np.exp(x)
    e_cuda, e_host = ulps(y, cuda_ref).max(), ulps(y, host_ref).max()
    print(f"{x.size} arguments: max {e_cuda:.2f} ulp from CUDA exp, {e_host:.2f} ulp from host exp")
    assert e_cuda <= 2.0 and e_host <= 2.0


def test_exp_special_values(pb):
    ctx = pb.pb_init(0)
    x = torch.tensor([0.0, -0.0, -700.0, -700.0000001, -1e4, -np.inf], dtype=torch.float64, device="cuda")
    y = pb.pb_selftest_exp(ctx, x).cpu().numpy()
    assert y[0] == 1.0 and y[1] == 1.0
    assert abs(y[2] / np.exp(-700.0) - 1) < 1e-15
    assert y[3] == 0.0 and y[4] == 0.0 and y[5] == 0.0
