"""Pins for the oracle's dynamics (Eq. 5, Algorithm 1) against closed forms and invariants.

Each test fixes something the paper's equations determine without reference to
the oracle's own code: exact solutions of small systems, first-order
convergence of forward Euler, conservation laws, and the potential whose
negative gradient the flow is.
"""
import numpy as np
import pytest

from workloads import csr_from_edges, erdos_renyi


def circ(x):
    """Signed circular difference in (-1/2, 1/2]."""
    return x - np.round(x)


def two_node(w):
    return csr_from_edges(2, [0], [1], [w])


def isolated(n):
    return csr_from_edges(n, np.zeros(0, int), np.zeros(0, int), np.zeros(0))


@pytest.mark.parametrize("w", [1.0, -1.0])
def test_two_oscillator_lock_closed_form(orc, w):
    # dDelta/dt = 2 K w sin(2 pi Delta)  =>  tan(pi Delta(t)) = tan(pi Delta0) exp(4 pi K w t)
    K, t_end, d0 = 0.25, 0.4, 0.1
    g = two_node(w)
    exact = np.arctan(np.tan(np.pi * d0) * np.exp(4 * np.pi * K * w * t_end)) / np.pi
    errs = []
    for dt in [0.01, 0.005, 0.0025, 0.00125]:
        T = int(round(t_end / dt))
        th, _ = orc.run(g, 2, K, 0.0, 0.0, dt, T, 1, seed=1, theta0=np.array([[0.3 + d0, 0.3]]))
        errs.append(abs(circ((th[0, 0] - th[0, 1]) - exact)))
    errs = np.array(errs)
    assert errs[-1] < 2e-3
    ratios = errs[:-1] / errs[1:]
    assert np.all((ratios > 1.8) & (ratios < 2.2)), ratios  # first order in dt
    # and the long-time lock: anti-phase for w = +1 (a cut edge), in phase for w = -1
    th, _ = orc.run(g, 2, K, 0.0, 0.0, 0.01, 2000, 1, seed=1, theta0=np.array([[0.4, 0.3]]))
    d = circ(th[0, 0] - th[0, 1])
    assert abs(abs(d) - 0.5) < 1e-6 if w > 0 else abs(d) < 1e-6


@pytest.mark.parametrize("q", [2, 3, 5])
def test_injection_locking_closed_form(orc, q):
    # one oscillator, K = 0: dtheta/dt = -Ks sin(2 pi q theta)
    #   => tan(pi q (theta - k/q)) = tan(pi q (theta0 - k/q)) exp(-2 pi q Ks t)
    Ks, t_end = 0.7, 0.3
    offs = np.array([0.35, -0.2, 0.1]) / q
    ks = np.array([0, 1, q - 1])
    th0 = (ks / q + offs) % 1.0
    g = isolated(3)
    exact = np.arctan(np.tan(np.pi * q * offs) * np.exp(-2 * np.pi * q * Ks * t_end)) / (np.pi * q)
    errs = []
    for dt in [0.004, 0.002, 0.001, 0.0005]:
        T = int(round(t_end / dt))
        th, _ = orc.run(g, q, 0.0, Ks, 0.0, dt, T, 1, seed=1, theta0=th0[None])
        errs.append(np.max(np.abs(circ(th[0] - ks / q - exact))))
    errs = np.array(errs)
    ratios = errs[:-1] / errs[1:]
    assert np.all((ratios > 1.8) & (ratios < 2.2)), ratios
    # stable lattice at k/q: a long run lands on it
    th, _ = orc.run(g, q, 0.0, Ks, 0.0, 0.01, 3000, 1, seed=1, theta0=th0[None])
    assert np.max(np.abs(circ(th[0] * q - ks))) < 1e-9


def test_phase_sum_conserved_without_injection_and_noise(orc):
    g = erdos_renyi(30, 0.3, 5, "pm1")
    th0 = np.random.default_rng(0).random((2, 30))
    th, _ = orc.run(g, 2, 0.3, 0.0, 0.0, 0.01, 300, 2, seed=1, theta0=th0)
    moved = np.abs(circ(th - th0)).max()
    assert moved > 1e-2                       # the phases did move
    assert np.all(np.abs(circ(th.sum(1) - th0.sum(1))) < 1e-10)


def test_noise_only_increment_and_variance(orc):
    n, R, T, dt, Kn, seed = 200, 8, 400, 0.01, 0.05, 17
    g = isolated(n)
    th0 = orc.init_phases(n, R, seed)
    th, _ = orc.run(g, 2, 0.0, 0.0, Kn, dt, T, R, seed=seed)
    delta = circ(th - th0)
    ref = Kn * np.sqrt(dt) * sum(orc.noise_block(n, R, seed, t) for t in range(T))
    assert np.max(np.abs(circ(delta - ref))) < 1e-10
    # Algorithm 1 reading: per-step std Kn*sqrt(dt), so Var = Kn^2 * T * dt
    # (the Eq. 5 reading sqrt(Kn*dt) would give Kn * T * dt = 0.2 here)
    var = delta.var()
    assert abs(var / (Kn**2 * T * dt) - 1.0) < 0.12


@pytest.mark.parametrize("q", [2, 3])
def test_derivative_is_negative_gradient_of_potential(orc, q):
    g = erdos_renyi(25, 0.3, 3, "pm1")
    rng = np.random.default_rng(4)
    th = rng.random(25)
    K, Ks = 0.37, 0.81
    f = orc.derivative(g, q, th, K, Ks)
    h = 1e-6
    grad = np.zeros(25)
    for i in range(25):
        e = np.zeros(25)
        e[i] = h
        grad[i] = (orc.lyapunov(g, q, th + e, K, Ks) - orc.lyapunov(g, q, th - e, K, Ks)) / (2 * h)
    assert np.max(np.abs(f + grad)) < 1e-7 * (1 + np.abs(f).max())


@pytest.mark.parametrize("q", [2, 3])
def test_lyapunov_nonincreasing_without_noise(orc, q):
    g = erdos_renyi(40, 0.2, 8, "pm1")
    K, Ks = 0.2, 0.5
    rows = np.repeat(np.arange(40), g.degrees())
    deg_abs = np.bincount(rows, weights=np.abs(g.w.astype(float)), minlength=40)
    # descent lemma: the Hessian of V is bounded by L = 2 pi (2 K max_i sum_j |w_ij| + q Ks)
    L = 2 * np.pi * (2 * K * deg_abs.max() + q * Ks)
    dt = 1.0 / L
    th = orc.init_phases(40, 1, seed=3)
    V = [orc.lyapunov(g, q, th[0], K, Ks)]
    for _ in range(300):
        th, _ = orc.run(g, q, K, Ks, 0.0, dt, 1, 1, seed=3, theta0=th)
        V.append(orc.lyapunov(g, q, th[0], K, Ks))
    V = np.array(V)
    assert np.all(np.diff(V) <= 1e-12), np.diff(V).max()
    assert V[-1] < V[0] - 0.1


def test_single_step_is_synchronous_euler(orc):
    g = erdos_renyi(20, 0.4, 2, "pm1")
    th0 = np.random.default_rng(9).random((1, 20))
    K, Ks, dt = 0.5, 0.3, 0.01
    th, _ = orc.run(g, 3, K, Ks, 0.0, dt, 1, 1, seed=1, theta0=th0)
    expect = (th0[0] + dt * orc.derivative(g, 3, th0[0], K, Ks)) % 1.0
    assert np.max(np.abs(circ(th[0] - expect))) < 1e-15


def test_triangular_waveform_shape(orc):
    # Algorithm 1's Ks waveform: 0 at each period start, Ks_max at mid-period, linear between
    T, kmax, P = 1200, 1.7, 3
    ks = orc.triangular(T, kmax, P)
    period = T // P
    assert np.allclose(ks[::period], 0.0, atol=1e-12)
    assert np.allclose(ks[period // 2::period], kmax, atol=1e-12)
    assert ks.min() >= 0 and ks.max() <= kmax + 1e-12
    d = np.diff(ks[:period // 2])
    assert np.allclose(d, d[0]) and d[0] > 0              # linear rise
    assert np.allclose(ks[:period], ks[period:2 * period])  # periodic
