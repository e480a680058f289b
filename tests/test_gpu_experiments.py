"""The experiments module at reduced sizes: FP32 against FP64 drift is
reported and small, and the physics goes the way Sec. 2 says."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_flat_interface_static_and_drift_small():
    from paper_1907_13415_gb300 import experiments as ex
    r = ex.flat(2.7, steps=1500, lx=128, ly=8, every=100)
    assert abs(r["x_iface_fp64"] - 63.5) < 1e-3
    assert r["fp32_vs_fp64"]["max_dQ_rel"] < 1e-3
    assert abs(r["fp32_vs_fp64"]["x_iface_drift_max"]) < 1e-2


@pytest.mark.parametrize("delta,sign", [(-0.03, -1), (0.03, 1)])
def test_disc_grows_above_and_shrinks_below_the_shift(delta, sign):
    """Sec. 2.2: a circular nematic domain shrinks at coexistence and needs a
    positive temperature shift to stand still; well above it grows."""
    from paper_1907_13415_gb300 import experiments as ex
    r = ex.disc(delta, steps=3000, n=64, radius=14, every=250)
    assert r["dRdt_fp64"] * sign > 0
    assert r["fp32_vs_fp64"]["max_dQ_rel"] < 1e-2
