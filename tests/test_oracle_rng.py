"""Pins for the oracle's random streams (Philox4x32-10, uniform map, Box-Muller).

The generator is pinned to an independent library implementation of
Philox4x32-10 (Salmon et al., SC'11); the derived uniforms and normals are
pinned by their exact lattice and by distribution tests.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_matches_library_implementation(orc):
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2**32, size=(61, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(61, 2), dtype=np.uint64).astype(np.uint32)
    ctr = np.concatenate([ctr, np.zeros((1, 4), np.uint32), np.full((1, 4), 0xFFFFFFFF, np.uint32),
                          np.array([[5, 1000, 17, 3]], np.uint32)])
    key = np.concatenate([key, np.zeros((1, 2), np.uint32), np.full((1, 2), 0xFFFFFFFF, np.uint32),
                          np.array([[20250528, 0]], np.uint32)])
    spec = json.dumps({"ctr": ctr.astype(np.int64).tolist(), "key": key.astype(np.int64).tolist()})
    env = dict(os.environ, TRITON_INTERPRET="1")
    res = subprocess.run([sys.executable, os.path.join(HERE, "_philox_library_ref.py"), spec],
                         capture_output=True, text=True, env=env, timeout=600)
    if res.returncode != 0:
        pytest.skip("library Philox unavailable: " + res.stderr[-300:])
    ref = np.array(json.loads(res.stdout.strip().splitlines()[-1]), dtype=np.uint32)
    mine = np.stack([orc.philox4x32_10(c, k) for c, k in zip(ctr, key)])
    assert np.array_equal(mine, ref)


def test_u01_lattice(orc):
    assert orc.u01(0) == 2.0**-24
    assert orc.u01(0xFFFFFFFF) == 1.0 - 2.0**-24
    rng = np.random.default_rng(1)
    for x in rng.integers(0, 2**32, size=200):
        u = orc.u01(int(x))
        assert 0.0 < u < 1.0
        k = u * 2**24
        assert k == int(k) and int(k) % 2 == 1
        assert np.float32(u) == u  # exact in FP32


def test_init_phases_uniform(orc):
    th = orc.init_phases(300, 40, seed=99, graph=0)
    assert th.min() > 0.0 and th.max() < 1.0
    assert stats.kstest(th.ravel(), "uniform").pvalue > 1e-3
    # lane structure: replicas sharing a quad and nodes are not correlated
    c = np.corrcoef(th[0::4].ravel(), th[1::4].ravel())[0, 1]
    assert abs(c) < 0.05


@pytest.mark.parametrize("lane", [0, 1, 2, 3])
def test_noise_is_standard_normal_per_lane(orc, lane):
    z = np.concatenate([orc.noise_block(200, 16, seed=5, t=t)[lane::4].ravel() for t in range(25)])
    assert abs(z.mean()) < 0.03
    assert abs(z.var() - 1.0) < 0.05
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_box_muller_pairs_independent(orc):
    z = np.stack([orc.noise_block(500, 8, seed=11, t=t) for t in range(20)])  # [t, R, n]
    a, b = z[:, 0::4].ravel(), z[:, 1::4].ravel()
    c, d = z[:, 2::4].ravel(), z[:, 3::4].ravel()
    for x, y in [(a, b), (c, d), (a, c)]:
        assert abs(np.corrcoef(x, y)[0, 1]) < 0.03
    # radius^2 of a Box-Muller pair is exponential with mean 2
    r2 = a**2 + b**2
    assert stats.kstest(r2 / 2.0, "expon").pvalue > 1e-3


def test_streams_graphs_steps_distinct(orc):
    base = orc.noise(3, 0, 10, 4, 2)
    assert base != orc.noise(3, 1, 10, 4, 2)      # graph index
    assert base != orc.noise(3, 0, 10, 5, 2)      # step
    assert base != orc.noise(3, 0, 11, 4, 2)      # node
    assert base != orc.noise(4, 0, 10, 4, 2)      # seed
    assert orc.init_phase(3, 0, 10, 2) != orc.init_phase(3, 0, 10, 6)
