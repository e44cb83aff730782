"""Host-side argument checks of the Python binding's newer entry points (kick,
drift, pm_accel, TreePMStepper): tensors that are not CUDA float64 / float32
of the right shape are refused with ValueError before the library is called,
so these run without a GPU."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def og():
    import __graft_entry__
    from paper_2606_17145_gb300 import build as b
    b.build()
    import paper_2606_17145_gb300 as m
    return m


def test_kick_and_drift_refuse_host_tensors(og):
    v = torch.zeros(4, 3, dtype=torch.float64)
    a = torch.zeros(4, 3, dtype=torch.float32)
    with pytest.raises(ValueError, match="CUDA"):
        og.kick(v, a, None, 0.1)
    with pytest.raises(ValueError, match="CUDA"):
        og.drift(v, v, 0.1)


def test_pm_accel_refuses_host_tensors(og):
    pos = torch.zeros(4, 3, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        og.pm_accel(None, pos, torch.ones(4, dtype=torch.float64), 1.0, 0.05)


def test_stepper_refuses_host_tensors(og):
    pos = torch.zeros(4, 3, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        og.TreePMStepper(pos, pos.clone(), torch.ones(4, dtype=torch.float64), 0.01, 1.0, 0.05, 0.5, 16)
