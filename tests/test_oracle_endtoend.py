"""End-to-end pins of the oracle: the simulated machine solves tiny instances.

A wrong sign anywhere in the coupling or the injection term turns the machine
into a min-cut or a colour-merging solver, which these catch.
"""
import numpy as np
import pytest

from workloads import erdos_renyi, linear_ramp, constant, planted_partition


def best_over_run(orc, g, q, R, T, seed, c):
    K = constant(T, c / g.mean_degree)
    th, trace = orc.run(g, q, K, linear_ramp(T, 0, 2), constant(T, 0.1), 0.01, T, R, seed,
                        readout_every=T // 10, nthreads=4)
    return trace


@pytest.mark.parametrize("seed", range(6))
def test_maxcut_reaches_bruteforce_optimum(orc, seed):
    g = erdos_renyi(16, 0.35, 100 + seed, "+1")
    opt, _ = orc.bruteforce_maxcut(g)
    trace = best_over_run(orc, g, 2, 16, 800, seed, 16.0)
    assert trace.max() <= opt
    assert trace[:, -1].max() == opt


@pytest.mark.parametrize("seed", range(4))
def test_maxcut_pm1_weights_reaches_optimum(orc, seed):
    g = erdos_renyi(16, 0.4, 200 + seed, "pm1")
    opt, _ = orc.bruteforce_maxcut(g)
    trace = best_over_run(orc, g, 2, 16, 800, seed, 16.0)
    assert trace.max() <= opt
    assert trace[:, -1].max() == opt


@pytest.mark.parametrize("seed", range(4))
def test_planted_colouring_found(orc, seed):
    g = planted_partition(15, 3, 3.0, 300 + seed)
    opt, _ = orc.bruteforce_min_conflicts(g, 3)
    assert opt == 0
    trace = best_over_run(orc, g, 3, 16, 1500, seed, 8.0)
    assert trace.min() >= opt
    assert trace[:, -1].min() == 0


def test_run_trace_matches_final_readout(orc):
    g = erdos_renyi(30, 0.2, 1, "pm1")
    T = 200
    th, trace = orc.run(g, 2, 0.5, 1.0, 0.1, 0.01, T, 4, seed=3, readout_every=50)
    assert trace.shape == (4, 4)
    assert np.array_equal(trace[:, -1], orc.scores(g, 2, orc.readout_f64(2, th)))
