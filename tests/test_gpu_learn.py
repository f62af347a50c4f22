"""Schedule learning through the library's adjoint: the training loss falls and
the learned curves carry over to held-out graphs of the same family."""
import numpy as np
import pytest

from gpu_common import require_gpu
from workloads import erdos_renyi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _batch(seeds, n=120, p=0.08):
    from paper_2505_22631_gb300 import Problem
    graphs = [erdos_renyi(n, p, s, "pm1") for s in seeds]
    return graphs, Problem.batch([Problem.from_graph(g, 2) for g in graphs])


def test_learned_schedules_lower_the_relaxed_energy():
    from paper_2505_22631_gb300.learn import ScheduleModel, learn_schedules, normalised_loss
    T, R, dt = 200, 32, 0.01
    train, ptrain = _batch([1, 2, 3, 4])
    test, ptest = _batch([101, 102, 103])
    model, hist = learn_schedules(ptrain, train, T, R, dt, iters=12, lr=0.1, knots=6, seed=5,
                                  K0=4.0, Ks_max0=0.5, checkpoint_every=50, fresh_noise=False)
    assert np.all(np.isfinite(hist))
    assert hist[-1] < hist[0] - 0.01, hist
    # held-out graphs, unseen noise: the learned curves beat the initial ones
    init = ScheduleModel(T, 6, [1.0], K0=4.0, Ks_max0=0.5)
    l_init = float(normalised_loss(ptest, test, init, dt, R, 77, 50).detach())
    l_fit = float(normalised_loss(ptest, test, model, dt, R, 77, 50).detach())
    assert l_fit < l_init, (l_fit, l_init)
