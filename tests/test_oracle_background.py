"""Pins of the oracle's background and step integrals (Sec. 3.3, conformal-time steps).

Pins: Gauss-Legendre nodes against numpy's leggauss; tau(a) and Delta tau against
the closed form of a radiation + matter universe; the eps integrals against the
closed forms of a massless particle and of a particle at rest in pure matter
domination; and every integral against scipy.integrate.quad in LCDM.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O


def test_gauss_legendre_matches_numpy():
    for n in (1, 2, 3, 4, 5, 8, 16):
        x, w = O.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.allclose(x, xr, atol=1e-15, rtol=0)
        assert np.allclose(w, wr, atol=1e-15, rtol=0)


def _rm_params(inputs):
    # Omega_Lambda = 0: radiation + matter only
    p = inputs.config("c1_32")
    p["omega_m"] = 1.0 - p["omega_r"]
    return p


def _tau_closed(p, a):
    H0 = p["h"] / 2997.92458
    om, orad = p["omega_m"], p["omega_r"]
    aeq = orad / om
    # sqrt(a + aeq) - sqrt(aeq), written without cancellation
    return 2.0 / (H0 * math.sqrt(om)) * a / (math.sqrt(a + aeq) + math.sqrt(aeq))


def test_tau_closed_form_radiation_matter(inputs, c1_tables):
    p = _rm_params(inputs)
    o = O.Oracle(p, c1_tables)
    for a in (1e-10, 1e-9, 1e-6, 3e-4, 1e-2, 1 / 32, 0.5, 1.0):
        assert abs(o.tau(a) / _tau_closed(p, a) - 1) < 1e-12


def test_dtau_closed_form_and_quad(inputs, c1_tables):
    p = _rm_params(inputs)
    o = O.Oracle(p, c1_tables)
    for k in range(0, 100, 7):
        l1, l2 = o.lna(k), o.lna(k + 1)
        ref = _tau_closed(p, math.exp(l2)) - _tau_closed(p, math.exp(l1))
        assert abs(o.dtau(l1, l2) / ref - 1) < 1e-12
        assert abs(o.dtau(l2, l1) / -ref - 1) < 1e-12
    # LCDM: against adaptive quadrature
    pl = inputs.config("c1_32")
    ol = O.Oracle(pl, c1_tables)
    for k in (0, 40, 80, 99):
        l1, l2 = ol.lna(k), ol.lna(k + 1)
        ref = integrate.quad(lambda s: 1.0 / (math.exp(s) * ol.hubble(math.exp(s))), l1, l2, epsrel=1e-14)[0]
        assert abs(ol.dtau(l1, l2) / ref - 1) < 1e-12


def test_eps_integrals_closed_forms(inputs, c1_tables):
    p = inputs.config("c1_32")
    o = O.Oracle(p, c1_tables)
    # massless: int dtau / q = Delta tau / q and int q dtau = q Delta tau
    for k in (0, 50, 99):
        l1, l2 = o.lna(k), o.lna(k + 1)
        dt = o.dtau(l1, l2)
        assert abs(o.eps_integral(0.0, 3e-4, l1, l2, 0) / (dt / 3e-4) - 1) < 1e-14
        assert abs(o.eps_integral(0.0, 3e-4, l1, l2, 1) / (dt * 3e-4) - 1) < 1e-14
    # at rest in pure matter domination: H = H0 a^-3/2
    pm = dict(p, omega_m=1.0, omega_r=0.0)
    om = O.Oracle(pm, c1_tables)
    H0 = p["h"] / 2997.92458
    m = 0.1
    for a1, a2 in ((1e-3, 1.2e-3), (0.02, 0.03125)):
        l1, l2 = math.log(a1), math.log(a2)
        ref0 = 2.0 / (m * H0) * (a1 ** -0.5 - a2 ** -0.5)
        ref1 = m / H0 * (2.0 / 3.0) * (a2 ** 1.5 - a1 ** 1.5)
        assert abs(om.eps_integral(m, 0.0, l1, l2, 0) / ref0 - 1) < 1e-13
        assert abs(om.eps_integral(m, 0.0, l1, l2, 1) / ref1 - 1) < 1e-13


@pytest.mark.parametrize("q", [1e-5, 5e-4, 3e-3])
def test_eps_integrals_against_quad(inputs, c1_tables, q):
    p = inputs.config("c1_32")
    o = O.Oracle(p, c1_tables)
    m = 0.1
    for k in (0, 60, 85, 99):
        l1, l2 = o.lna(k), o.lna(k + 0.5)
        for kind in (0, 1):
            def f(s):
                a = math.exp(s)
                e = math.sqrt(q * q + m * m * a * a)
                return (e if kind else 1.0 / e) / (a * o.hubble(a))
            ref = integrate.quad(f, l1, l2, epsrel=2e-14, epsabs=0)[0]
            assert abs(o.eps_integral(m, q, l1, l2, kind) / ref - 1) < 1e-12


def test_time_grid(inputs, c1_tables):
    p = inputs.config("c1_32")
    o = O.Oracle(p, c1_tables)
    assert abs(o.lna(0) + math.log(1 + 1e9)) < 1e-14
    assert abs(o.lna(100) + math.log(32.0)) < 1e-13
    assert abs((o.lna(100) - o.lna(0)) / 100 - 0.172576) < 1e-6
