"""Pins for readout, scores, energy and the exhaustive solvers of the oracle."""
import os

import numpy as np
import pytest

from workloads import (complete, complete_bipartite, csr_from_edges, cycle, erdos_renyi,
                       petersen, planted_partition)

HERE = os.path.dirname(os.path.abspath(__file__))


def test_table1_accuracy_definition(orc):
    rows = 0
    for line in open(os.path.join(HERE, "golden", "table1_maxcut_accuracy.txt")):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        best, cut, acc = int(parts[2]), int(parts[3]), float(parts[4])
        tol = 0.02 if parts[-1] == "garbled" else 0.01 + 1e-9
        assert abs(orc.accuracy_percent(cut, best) - acc) <= tol, parts[0]
        rows += 1
    assert rows == 30


@pytest.mark.parametrize("q", [2, 3, 4, 5])
def test_readout_lattice_points(orc, q):
    k = np.arange(q)
    for eps in [0.0, 1e-4, -1e-4, 0.49 / q, -0.49 / q]:
        th = (k / q + eps) % 1.0
        assert np.array_equal(orc.readout_f64(q, th[None])[0], k)
        assert np.array_equal(orc.readout_f32(q, th.astype(np.float32)[None])[0], k)


def test_readout_fp32_boundaries(orc):
    f = np.float32

    def f32_spin(q, x):   # floor(q*theta + 1/2) mod q, each operation rounded to FP32
        return int(np.floor(f(f(q) * f(x)) + f(0.5))) % q

    th = np.array([[0.25, np.nextafter(f(0.25), f(0)), 0.75, np.nextafter(f(0.75), f(0)),
                    np.nextafter(f(1.0), f(0)), 0.0, np.nextafter(f(0.25), f(0)) - f(2**-26)]],
                  dtype=np.float32)
    got = orc.readout_f32(2, th)[0].tolist()
    assert got == [f32_spin(2, x) for x in th[0]]
    # 1/4 rounds up to spin 1 and 3/4 up to spin 0; just below 1/4 the FP32 sum
    # 1 - 2^-25 is a tie that rounds to 1.0, so that phase reads as spin 1 too
    assert got == [1, 1, 0, 1, 0, 0, 0]
    th3 = np.array([[f(1) / f(6), 0.5, f(5) / f(6), 0.999, np.nextafter(f(0.5), f(0))]],
                   dtype=np.float32)
    assert orc.readout_f32(3, th3)[0].tolist() == [f32_spin(3, x) for x in th3[0]]


def test_scores_hand_counted(orc):
    # path 0-1-2-3 with weights 1, 2, -1 and a chord 0-2 with weight 3
    g = csr_from_edges(4, [0, 1, 2, 0], [1, 2, 3, 2], [1.0, 2.0, -1.0, 3.0])
    s = np.array([[0, 1, 1, 0], [0, 0, 0, 0], [1, 0, 1, 0]], dtype=np.int8)
    # cut: edges whose ends differ
    assert orc.scores(g, 2, s).tolist() == [1 - 1 + 3, 0, 1 + 2 - 1]
    # conflicts: edges whose ends agree
    assert orc.scores(g, 3, s).tolist() == [2, 1 + 2 - 1 + 3, 3]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_energy_lattice_identities(orc, seed):
    g = erdos_renyi(60, 0.15, seed, "pm1")
    rng = np.random.default_rng(seed)
    W = g.total_weight()
    s2 = rng.integers(0, 2, size=(5, 60)).astype(np.int8)
    # Eq. 6 at the Ising lattice: E = W_tot - 2 * cut
    assert np.allclose(orc.energy(g, s2 / 2.0), W - 2 * orc.scores(g, 2, s2), atol=1e-9)
    s3 = rng.integers(0, 3, size=(5, 60)).astype(np.int8)
    # at the 3-state lattice cos(2 pi k / 3) = -1/2 for k != 0: E = sum w (1.5 delta - 0.5)
    assert np.allclose(orc.energy(g, s3 / 3.0), 1.5 * orc.scores(g, 3, s3) - 0.5 * W, atol=1e-9)


def test_bruteforce_known_maxcuts(orc):
    assert orc.bruteforce_maxcut(cycle(10))[0] == 10
    assert orc.bruteforce_maxcut(cycle(11))[0] == 10
    assert orc.bruteforce_maxcut(complete(9))[0] == 20        # floor(81 / 4)
    assert orc.bruteforce_maxcut(complete_bipartite(4, 6))[0] == 24
    assert orc.bruteforce_maxcut(petersen())[0] == 12
    v, best = orc.bruteforce_maxcut(cycle(12))
    assert orc.scores(cycle(12), 2, best[None])[0] == v


def test_bruteforce_known_colourings(orc):
    assert orc.bruteforce_min_conflicts(complete(4), 3)[0] == 1
    assert orc.bruteforce_min_conflicts(cycle(7), 2)[0] == 1
    assert orc.bruteforce_min_conflicts(petersen(), 3)[0] == 0
    assert orc.bruteforce_min_conflicts(petersen(), 2)[0] == 3   # 15 edges - max cut 12
    g = planted_partition(12, 3, 3.0, 4)
    v, best = orc.bruteforce_min_conflicts(g, 3)
    assert v == 0 and orc.scores(g, 3, best[None])[0] == 0
