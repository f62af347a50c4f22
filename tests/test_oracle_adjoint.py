"""Pin the oracle adjoint to FP64 central finite differences of the loss.

The loss is L = mean_r E(theta_T^r) (Eq. 6 on the final phases); the finite
differences re-run the forward simulation with one schedule entry perturbed,
with the same noise, and never touch the adjoint code.
"""
import numpy as np
import pytest

from workloads import erdos_renyi


def loss(orc, g, q, K, Ks, Kn, dt, T, R, seed):
    th, _ = orc.run(g, q, K, Ks, Kn, dt, T, R, seed)
    return orc.energy(g, th).mean()


@pytest.mark.parametrize("q", [2, 3])
def test_adjoint_matches_finite_differences(orc, q):
    g = erdos_renyi(9, 0.5, 21, "pm1")
    T, R, dt, seed = 40, 2, 0.01, 5
    rng = np.random.default_rng(q)
    K = 0.3 + 0.2 * rng.random(T)
    Ks = np.linspace(0.0, 1.5, T)
    Kn = 0.1 + 0.05 * rng.random(T)
    L, dK, dKs, dKn = orc.adjoint(g, q, K, Ks, Kn, dt, T, R, seed)
    assert abs(L - loss(orc, g, q, K, Ks, Kn, dt, T, R, seed)) < 1e-12
    h = 1e-6
    for t in [0, 7, 23, T - 1]:
        for arr, grad in [(K, dK), (Ks, dKs), (Kn, dKn)]:
            up, dn = arr.copy(), arr.copy()
            up[t] += h
            dn[t] -= h
            args = {id(K): 0, id(Ks): 1, id(Kn): 2}[id(arr)]
            sched_up = [K, Ks, Kn]
            sched_dn = [K, Ks, Kn]
            sched_up[args] = up
            sched_dn[args] = dn
            fd = (loss(orc, g, q, *sched_up, dt, T, R, seed)
                  - loss(orc, g, q, *sched_dn, dt, T, R, seed)) / (2 * h)
            assert abs(fd - grad[t]) <= 1e-6 * (1 + abs(fd)), (t, fd, grad[t])
