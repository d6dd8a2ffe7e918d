"""Pins of the oracle's pre-initial sampler (Sec. 2.1) and of its Philox generator.

Pins: published Philox4x32-10 known-answer vectors; closed-form Fermi-Dirac
moments <q>/T = 7 pi^4 / (180 zeta(3)) and <q^2>/T^2 = 15 zeta(5) / zeta(3);
a Kolmogorov-Smirnov test against the Fermi-Dirac CDF computed by scipy; the
CDF table against the oracle's own adaptive integral and scipy.integrate.quad;
uniformity of positions and isotropy of directions.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_fd_cdf_table_against_independent_integrals(inputs):
    t, F = inputs.fd_cdf_table()
    assert len(t) == 4001 and t[0] == 0.0 and F[0] == 0.0
    assert np.all(np.diff(F) >= 0.0)
    norm = 1.5 * special.zeta(3.0)
    for j in (1, 7, 50, 100, 222, 400, 1000, 2000, 3999, 4000):
        own = O.fd_cdf(t[j])
        ref = integrate.quad(lambda x: x * x / (1.0 + math.exp(x)), 0.0, t[j], epsabs=1e-15, epsrel=1e-14,
                             limit=200)[0] / norm
        assert abs(F[j] - own) < 1e-12
        assert abs(F[j] - ref) < 1e-12
    # the tail beyond q/T = 40 is 40^2 e^-40 / (1.5 zeta 3) ~ 4e-15
    assert abs(F[-1] - 1.0) < 1e-13


@pytest.fixture(scope="module")
def big_sample(inputs, c1_tables):
    p = inputs.config("c1_32", seed=11)
    o = O.Oracle(p, c1_tables)
    X, qs, pm = o.sample(np.arange(400_000))
    return o, X, qs, pm


def test_fermi_dirac_moments(big_sample):
    o, X, qs, pm = big_sample
    T = o.temperature_ev()
    assert T == 1.95 * 8.617333262e-5
    x = pm / T
    n = len(x)
    m1 = 7 * math.pi ** 4 / (180 * special.zeta(3.0))
    m2 = 15 * special.zeta(5.0) / special.zeta(3.0)
    assert abs(m1 - 3.15137) < 1e-5 and abs(m2 - 12.9394) < 1e-4
    assert abs(x.mean() - m1) < 4 * x.std() / math.sqrt(n)
    assert abs((x * x).mean() - m2) < 4 * (x * x).std() / math.sqrt(n)


def test_fermi_dirac_ks(big_sample):
    o, X, qs, pm = big_sample
    x = np.sort(pm / o.temperature_ev())[::40]
    norm = 1.5 * special.zeta(3.0)
    grid = np.linspace(0, 40, 8001)
    vals = np.array([0.0] + [integrate.quad(lambda s: s * s / (1 + math.exp(s)), a, b)[0]
                             for a, b in zip(grid[:-1], grid[1:])])
    cdf = np.cumsum(vals) / norm
    res = stats.kstest(x, lambda v: np.interp(v, grid, cdf))
    assert res.pvalue > 1e-3


def test_positions_uniform_and_directions_isotropic(big_sample):
    o, X, qs, pm = big_sample
    u = X.astype(np.float64) / 2 ** 32
    n = u.shape[1]
    for d in range(3):
        assert abs(u[d].mean() - 0.5) < 4 * math.sqrt(1 / 12 / n)
        assert stats.kstest(u[d][::20], "uniform").pvalue > 1e-3
    nh = qs / pm
    assert np.allclose(np.linalg.norm(nh, axis=0), 1.0, atol=4e-16)
    assert np.all(np.abs(nh.mean(axis=1)) < 4 * math.sqrt(1 / 3 / n))
    M = nh @ nh.T / n
    assert np.allclose(M, np.eye(3) / 3, atol=4 * math.sqrt(2 / 15 / n) * 3)


def test_pmag_is_the_sampled_vector_norm(big_sample):
    o, X, qs, pm = big_sample
    q0, q1, q2 = qs[:, :1000]
    assert np.array_equal(pm[:1000], np.sqrt(q0 * q0 + q1 * q1 + q2 * q2))


def test_sampler_is_deterministic_and_index_addressed(inputs, c1_tables):
    p = inputs.config("c1_32", seed=5)
    o = O.Oracle(p, c1_tables)
    a = o.sample(np.arange(100))
    b = o.sample(np.arange(50, 150))
    assert np.array_equal(a[0][:, 50:], b[0][:, :50])
    assert np.array_equal(a[1][:, 50:], b[1][:, :50])
    p2 = inputs.config("c1_32", seed=6)
    c = O.Oracle(p2, c1_tables).sample(np.arange(100))
    assert not np.array_equal(a[0], c[0])


def test_inverse_cdf(inputs, c1_tables):
    """Inversion of the tabulated CDF: exact at nodes, linear between, clamped at the end."""
    o = O.Oracle(inputs.config("c1_32"), c1_tables)
    t, F = c1_tables["cdf_t"], c1_tables["cdf_F"]
    for j in (3, 100, 1234, 3000):
        assert o.fd_inverse(F[j]) == t[j]
    rng = np.random.default_rng(0)
    for u in rng.random(200):
        assert abs(o.fd_inverse(u) - np.interp(u, F, t)) < 1e-13
    assert o.fd_inverse(0.0) == 0.0
    assert o.fd_inverse(1.0 - 2 ** -53) == 40.0
