"""Host logic of schedule learning: the interpolation and the schedule model."""
import numpy as np
import pytest
import torch

from paper_2505_22631_gb300.learn import ScheduleModel, interp_matrix


def test_interp_matrix_is_linear_interpolation():
    M = interp_matrix(11, 3).numpy()
    assert M.shape == (11, 3)
    assert np.allclose(M.sum(axis=1), 1.0)
    knots = np.array([2.0, -1.0, 5.0])
    y = M @ knots
    assert y[0] == 2.0 and y[-1] == 5.0 and y[5] == -1.0
    assert np.allclose(y, np.interp(np.arange(11), [0, 5, 10], knots))
    with pytest.raises(ValueError):
        interp_matrix(10, 1)


def test_schedule_model_starts_at_the_hand_schedules():
    m = ScheduleModel(101, 6, [0.25, 0.05], K0=16.0, Ks_max0=2.0, Kn0=0.1)
    K, Ks, Kn = m()
    assert K.shape == Ks.shape == Kn.shape == (2, 101) and K.dtype == torch.float32
    assert torch.allclose(K[0], torch.full((101,), 4.0), rtol=1e-5)
    assert torch.allclose(K[1], torch.full((101,), 0.8), rtol=1e-5)
    assert torch.allclose(Ks[0], torch.linspace(0, 2, 101), atol=2e-4)
    assert torch.allclose(Kn, torch.full((2, 101), 0.1), rtol=1e-5)
    # gradients reach every knot
    (K.sum() + Ks.sum() + Kn.sum()).backward()
    assert all(p.grad is not None and torch.all(p.grad > 0) for p in m.parameters())
