"""Pins of the oracle's particle dynamics, weights and deposit.

Pins (Sec. 2.1, 2.2, 3.3 of the paper):
* phi = psi = 0: momenta bitwise unchanged, delta-f weights exactly zero;
* free streaming: displacement = q int dtau / eps (adaptive quadrature), and
  n_hat Delta tau for massless particles (closed-form tau);
* uniform potential gradients: the analytic kick of eq:releq_approx, summed
  over the whole run (adaptive quadrature);
* the pre-initial transform eq:transform under uniform fields (closed form);
* time reversibility of the leapfrog and det J = 1 (Sec. 3.3, footnote on
  phase-space density);
* the delta-f weight against its definition 1 - fbar(q)/fbar(p);
* CIC: total mass, a particle on a node, a uniform lattice.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O


def _params(inputs, **over):
    p = inputs.config("c1_32", n_grid=16, n_part=4096, n_steps=40, seed=21)
    p.update(over)
    return p


def _quad_eps(o, m, q, l1, l2, kind):
    def f(s):
        a = math.exp(s)
        e = math.sqrt(q * q + m * m * a * a)
        return (e if kind else 1.0 / e) / (a * o.hubble(a))
    # split at every step boundary so quad sees smooth pieces
    n = 200
    edges = np.linspace(l1, l2, n + 1)
    return math.fsum(integrate.quad(f, a, b, epsrel=1e-13, epsabs=0)[0] for a, b in zip(edges[:-1], edges[1:]))


def test_zero_potentials_exact(inputs, c1_tables):
    p = _params(inputs)
    o = O.Oracle(p, inputs.zero_tables(c1_tables))
    g = np.arange(512)
    r = o.run(g)
    assert np.array_equal(r["q"], r["qs"])
    assert np.array_equal(r["q0"], r["qs"])
    assert np.all(r["w"] == 0.0)


def _periodic_diff(a, b, L):
    d = (a - b) % L
    return np.where(d >= L / 2, d - L, d)


def test_free_streaming_quadrature(inputs, c1_tables):
    p = _params(inputs, m_ev=[0.1])
    o = O.Oracle(p, inputs.zero_tables(c1_tables))
    g = np.arange(64)
    ic = o.initial(g)
    x, q = o.integrate(g, ic["x"], ic["q"], ic["q0"], 0, p["n_steps"])
    l0, l1 = o.lna(0), o.lna(p["n_steps"])
    for i in range(0, 64, 8):
        qm = ic["p"][i]
        I = _quad_eps(o, 0.1, qm, l0, l1, 0)
        disp = ic["q"][:, i] * I
        err = _periodic_diff(x[:, i], ic["x"][:, i] + disp, p["box"])
        assert np.all(np.abs(err) <= 1e-10 * np.linalg.norm(disp) + 1e-9)


def test_free_streaming_massless_closed_form(inputs, c1_tables):
    p = _params(inputs, m_ev=[0.0])
    p["omega_m"] = 1.0 - p["omega_r"]          # no Lambda: tau(a) has a closed form
    o = O.Oracle(p, inputs.zero_tables(c1_tables))
    g = np.arange(32)
    ic = o.initial(g)
    x, q = o.integrate(g, ic["x"], ic["q"], ic["q0"], 0, p["n_steps"])
    H0 = p["h"] / 2997.92458
    aeq = p["omega_r"] / p["omega_m"]

    def tau(a):
        return 2.0 / (H0 * math.sqrt(p["omega_m"])) * a / (math.sqrt(a + aeq) + math.sqrt(aeq))

    dtau = tau(math.exp(o.lna(p["n_steps"]))) - tau(math.exp(o.lna(0)))
    nh = ic["q"] / np.linalg.norm(ic["q"], axis=0)
    err = _periodic_diff(x, ic["x"] + nh * dtau, p["box"])
    assert np.max(np.abs(err)) < 1e-10 * dtau


def test_uniform_gradient_analytic_kick(inputs, c1_tables):
    p = _params(inputs, m_ev=[0.05], n_steps=30)
    N = p["n_grid"]
    gpsi, gphi, cdot = np.array([2e-6, -1e-6, 5e-7]), np.array([-3e-7, 4e-7, 1e-6]), 3e-9
    frozen = inputs.uniform_fields(N, gpsi, gphi, cdot, 0.0)
    o = O.Oracle(p, c1_tables)
    g = np.arange(16)
    ic = o.initial(g, frozen=np.zeros_like(frozen))       # untransformed start: q = q0 = q_sampled
    x, q = o.integrate(g, ic["x"], ic["q"], ic["q0"], 0, p["n_steps"], frozen=frozen)
    l0, l1 = o.lna(0), o.lna(p["n_steps"])
    dtau_tot = math.fsum(integrate.quad(lambda s: 1 / (math.exp(s) * o.hubble(math.exp(s))), a, b,
                                        epsrel=1e-13)[0]
                         for a, b in zip(np.linspace(l0, l1, 201)[:-1], np.linspace(l0, l1, 201)[1:]))
    for i in range(16):
        q0 = ic["q0"][:, i]
        q0m = np.linalg.norm(q0)
        Kpsi = _quad_eps(o, 0.05, q0m, l0, l1, 1)
        Kphi = _quad_eps(o, 0.05, q0m, l0, l1, 0)
        ref = q0 - gpsi * Kpsi - (q0m ** 2 * gphi - q0 * (q0 @ gphi)) * Kphi + q0 * cdot * dtau_tot
        dq_ref = ref - q0
        assert np.linalg.norm(q[:, i] - ref) < 1e-10 * np.linalg.norm(dq_ref)
        # the phi term is perpendicular to q0
        perp = q0m ** 2 * gphi - q0 * (q0 @ gphi)
        assert abs(perp @ q0) < 1e-12 * q0m * np.linalg.norm(perp) * q0m


def test_initial_transform_uniform_fields(inputs, c1_tables):
    p = _params(inputs, m_ev=[0.2])
    p["omega_m"] = 1.0 - p["omega_r"]
    N = p["n_grid"]
    gpsi, psi = np.array([1e-6, 2e-6, -3e-6]), 4e-5
    frozen = inputs.uniform_fields(N, gpsi, [0, 0, 0], 0.0, psi)
    o = O.Oracle(p, c1_tables)
    g = np.arange(8)
    ic = o.initial(g, frozen=frozen)
    H0 = p["h"] / 2997.92458
    aeq = p["omega_r"] / p["omega_m"]
    a0 = math.exp(o.lna(0))
    tau0 = 2.0 / (H0 * math.sqrt(p["omega_m"])) * a0 / (math.sqrt(a0 + aeq) + math.sqrt(aeq))
    eps = np.sqrt(ic["p"] ** 2 + (0.2 * a0) ** 2)
    ref = ic["qs"] * (1 - psi / 2) - (eps * tau0 / 6)[None, :] * gpsi[:, None]
    assert np.allclose(ic["q"], ref, rtol=1e-13, atol=0)
    assert np.array_equal(ic["q0"], ic["q"])


def test_reversibility(inputs, c1_tables):
    p = _params(inputs, m_ev=[0.1], n_steps=60)
    N = p["n_grid"]
    frozen = inputs.cosine_fields(N, p["box"], 3e-4, (1, 2, 3))
    o = O.Oracle(p, c1_tables)
    g = np.arange(128)
    ic = o.initial(g, frozen=np.zeros_like(frozen))
    k0, k1 = 35, 60   # late steps, where particles are slow and kicks are strong
    x1, q1 = o.integrate(g, ic["x"], ic["q"], ic["q0"], k0, k1, frozen=frozen)
    assert np.max(np.linalg.norm(q1 - ic["q"], axis=0) / np.linalg.norm(ic["q"], axis=0)) > 1e-3
    x2, q2 = o.integrate(g, x1, q1, ic["q0"], k1, k0, frozen=frozen)
    assert np.max(np.abs(_periodic_diff(x2, ic["x"], p["box"]))) < 1e-12 * p["box"]
    assert np.max(np.linalg.norm(q2 - ic["q"], axis=0) / np.linalg.norm(ic["q"], axis=0)) < 1e-12


def test_one_step_jacobian_determinant(inputs, c1_tables):
    p = _params(inputs, m_ev=[0.1], n_steps=60)
    N = p["n_grid"]
    frozen = inputs.cosine_fields(N, p["box"], 3e-4, (1, 2, 3))
    o = O.Oracle(p, c1_tables)
    n = 100
    g = np.arange(n)
    ic = o.initial(g, frozen=np.zeros_like(frozen))
    k = 50
    hx, hq = 1e-4, 1e-9
    dets = []
    for i in range(n):
        J = np.zeros((6, 6))
        for c in range(6):
            plus_x, plus_q = ic["x"][:, i:i + 1].copy(), ic["q"][:, i:i + 1].copy()
            minus_x, minus_q = plus_x.copy(), plus_q.copy()
            h = hx if c < 3 else hq
            if c < 3:
                plus_x[c] += h; minus_x[c] -= h
            else:
                plus_q[c - 3] += h; minus_q[c - 3] -= h
            xp, qp = o.integrate(g[i:i + 1], plus_x, plus_q, ic["q0"][:, i:i + 1], k, k + 1, frozen=frozen)
            xm, qm = o.integrate(g[i:i + 1], minus_x, minus_q, ic["q0"][:, i:i + 1], k, k + 1, frozen=frozen)
            dx = _periodic_diff(xp, xm, p["box"])[:, 0] / (2 * h)
            dq = (qp - qm)[:, 0] / (2 * h)
            J[:3, c], J[3:, c] = dx, dq
        dets.append(np.linalg.det(J))
    dets = np.array(dets)
    assert np.max(np.abs(dets - 1)) < 1e-8


def test_gather_nodes_and_linear_reproduction(inputs, c1_tables):
    """Order-1 interpolation: exact at nodes, exact for fields linear within a cell."""
    p = _params(inputs)
    o = O.Oracle(p, c1_tables)
    N, L = p["n_grid"], p["box"]
    h = L / N
    rng = np.random.default_rng(5)
    F = rng.standard_normal((8, N, N, N))
    for ix, iy, iz in ((0, 0, 0), (3, 9, 14), (15, 1, 7)):
        assert np.array_equal(o.gather(F, [ix * h, iy * h, iz * h]), F[:, iz, iy, ix])
    n = np.arange(N, dtype=float)
    z, y, x = np.meshgrid(n, n, n, indexing="ij")
    lin = np.stack([x + 10 * y + 100 * z] * 8)
    for _ in range(50):
        u = rng.uniform(0, N - 1, 3)      # stay clear of the periodic last cell
        v = o.gather(lin, u * h)
        assert np.allclose(v, u[0] + 10 * u[1] + 100 * u[2], rtol=1e-13, atol=1e-11)


def test_weights_definition(inputs, c1_tables):
    p = _params(inputs)
    o = O.Oracle(p, c1_tables)
    T = o.temperature_ev()
    rng = np.random.default_rng(3)
    pm = rng.uniform(0.05, 15, 1000) * T
    nh = rng.standard_normal((3, 1000))
    nh /= np.linalg.norm(nh, axis=0)
    qm = pm * (1 + rng.uniform(-1e-3, 1e-3, 1000))
    q = nh * qm
    w = o.weights(q, pm)
    fbar = lambda v: 1.0 / (1.0 + np.exp(v / T))
    ref = 1.0 - fbar(np.linalg.norm(q, axis=0)) / fbar(pm)
    assert np.max(np.abs(w - ref)) < 1e-13
    # far tail (q/T ~ 40): the stable form neither overflows nor cancels
    w2 = o.weights(nh[:, :1] * 40 * T * 1.001, np.array([40 * T]))
    assert np.isfinite(w2[0]) and abs(w2[0] - (1 - math.exp(-0.04))) < 1e-12


def test_deposit_mass_delta_and_lattice(inputs, c1_tables):
    p = _params(inputs)
    o = O.Oracle(p, c1_tables)
    N, L = p["n_grid"], p["box"]
    rng = np.random.default_rng(2)
    n = 3000
    x = rng.uniform(0, L, (3, n))
    q = rng.standard_normal((3, n)) * 5e-4
    w = rng.standard_normal(n) * 1e-3
    a = 1 / 32
    grid = o.deposit(np.zeros(n, np.int64), x, q, w, a, 0)
    eps = np.sqrt((q ** 2).sum(0) + (0.1 * a) ** 2)
    assert abs(grid.sum() - (w * eps).sum()) < 1e-12 * np.abs(w * eps).sum()
    # on a node: all weight on that node
    h = L / N
    xs = np.array([[3 * h], [5 * h], [7 * h]])
    gd = o.deposit(np.zeros(1, np.int64), xs, q[:, :1], w[:1], a, 1)
    assert gd[7, 5, 3] == w[0] and np.count_nonzero(gd) == 1
    # a uniform lattice offset by a fraction of a cell gives a uniform grid
    idx = (np.arange(N) + 0.3) * h
    z, y, xg = np.meshgrid(idx, idx, idx, indexing="ij")
    xl = np.stack([xg.ravel(), y.ravel(), z.ravel()])
    gl = o.deposit(np.zeros(N ** 3, np.int64), xl, np.zeros_like(xl), np.ones(N ** 3), a, 1)
    assert np.allclose(gl, 1.0, rtol=1e-13, atol=0)
