"""Pins of the oracle's pre-initial momentum transform (eq:transform, Sec. 2.1)
by the moments it must produce, computed from sampled particles.

Sec. 2.1 takes the super-horizon moments delta = -2 psi and theta = k^2 tau psi / 2
(with nu = dlog rho/dlog T = 4 and omega = 1 + w = 4/3 for relativistic
particles), writes the perturbed distribution as a rescaling of fbar (eq:pre_int)
and applies it to particles drawn from fbar (eq:transform).  The delta-f weights
w = 1 - fbar(|q|)/fbar(p) of Sec. 2.2 then carry the perturbation, so the moments
follow from the ensemble (eq:empirical_rho and its momentum analogue):

* energy density:  delta = sum_k w_k eps_k / sum_k eps(p_k);
* energy flux:     (rho + P) theta = div J, J = (1/n) sum_k w_k q_k, i.e. for one
  Fourier mode  i k . J_k = (4/3) rho theta_k.

The monopole reproduces delta = -2 psi exactly as printed.  For the dipole the
paper's Legendre convention (eq:def2, with the factor 2l+1) and eq:theta give
(rho + P) theta as the flux of Psi_1's term; eq:pre_int and eq:transform print
the dipole without that factor 3, so the printed transform carries one third of
theta's flux.  The oracle's default follows the printed formula; flag bit 1
(FDF_FLAG_LEGENDRE_DIPOLE in the library) multiplies the dipole by 3 and then
carries theta in full.  Both readings are pinned here: a flipped sign, a lost
factor 1/2 on psi or on theta, or a wrong factor on the dipole fails one test.

Sampling noise: the estimators below average ~1e6 independent particles, so
their relative noise is a few 1e-3; the tolerances are a few per cent.
"""
import math

import numpy as np
import pytest

import oracle as O

FLAG_LEGENDRE_DIPOLE = 2


def _massless(inputs, **over):
    # m = 0: eps = |q| exactly, so nu = 4 and omega = 4/3 hold without corrections
    p = inputs.config("c1_32", n_grid=32, n_part=1 << 20, m_ev=[0.0], seed=404)
    p.update(over)
    return p


def _eps(ic, o, m):
    a0 = math.exp(o.lna(0))
    eps_q = np.sqrt(np.sum(ic["q"] ** 2, axis=0) + (m * a0) ** 2)
    eps_p = np.sqrt(ic["p"] ** 2 + (m * a0) ** 2)
    return eps_q, eps_p


@pytest.mark.parametrize("psi", [3e-4, -1e-3])
def test_energy_contrast_uniform_psi_is_minus_two_psi(inputs, c1_tables, psi):
    """Uniform psi, no gradient: the delta-f energy contrast is delta = -2 psi."""
    p = _massless(inputs)
    N = p["n_grid"]
    o = O.Oracle(p, c1_tables)
    g = np.arange(p["n_part"])
    ic = o.initial(g, frozen=inputs.uniform_fields(N, [0, 0, 0], [0, 0, 0], 0.0, psi))
    w = o.weights(ic["q"], ic["p"])
    eps_q, eps_p = _eps(ic, o, 0.0)
    delta = np.sum(w * eps_q) / np.sum(eps_p)
    print("delta / (-2 psi) = %.5f" % (delta / (-2 * psi)))
    assert abs(delta / (-2 * psi) - 1) < 0.02


def _flux_ratio(inputs, c1_tables, flags):
    """i k . J_k / ((4/3) rho theta_k) for one cosine mode of psi along x; only grad psi
    is injected (slot 7, psi itself, is zero), so the monopole adds no noise."""
    p = _massless(inputs, flags=flags)
    N, L = p["n_grid"], p["box"]
    o = O.Oracle(p, c1_tables)
    tau0 = o.tau(math.exp(o.lna(0)))
    k = 2 * math.pi / L
    # grad psi amplitude: a fractional momentum change (eps tau0/6)|grad psi|/q of 1e-6,
    # deep in the linear regime
    A = 6e-6 / tau0 / k
    x_nodes = np.arange(N) * (L / N)
    F = np.zeros((8, N, N, N))
    F[0] = (-A * k * np.sin(k * x_nodes))[None, None, :]
    g = np.arange(p["n_part"])
    ic = o.initial(g, frozen=F)
    w = o.weights(ic["q"], ic["p"])
    _, eps_p = _eps(ic, o, 0.0)
    x = ic["x"][0]
    J = np.mean(w * ic["q"][0] * np.exp(-1j * k * x))
    rho = np.mean(eps_p)
    theta_k = 0.5 * k * k * tau0 * (A / 2)
    # the trilinear read of the sampled mode scales it by sinc^2(k h / 2)
    kh = k * L / N
    interp = (math.sin(kh / 2) / (kh / 2)) ** 2
    return 1j * k * J / ((4.0 / 3.0) * rho * theta_k * interp)


def test_flux_of_the_printed_transform_is_one_third_of_theta(inputs, c1_tables):
    r = _flux_ratio(inputs, c1_tables, 0)
    print("printed eq:transform: div J / ((rho + P) theta) = %.5f %+.5fi" % (r.real, r.imag))
    assert abs(r.real - 1.0 / 3.0) < 0.01 and abs(r.imag) < 0.01


def test_flux_of_the_legendre_dipole_reading_is_theta(inputs, c1_tables):
    r = _flux_ratio(inputs, c1_tables, FLAG_LEGENDRE_DIPOLE)
    print("2l+1 reading: div J / ((rho + P) theta) = %.5f %+.5fi" % (r.real, r.imag))
    assert abs(r.real - 1.0) < 0.03 and abs(r.imag) < 0.03


def test_legendre_dipole_flag_scales_only_the_dipole(inputs, c1_tables):
    """With psi and grad psi both present, the flag triples q - q_s (1 - psi/2) and leaves
    the monopole's rescaling alone."""
    p = _massless(inputs, n_part=256, m_ev=[0.1])
    N = p["n_grid"]
    F = inputs.uniform_fields(N, [10.0, -20.0, 30.0], [0, 0, 0], 0.0, 5e-5)
    g = np.arange(p["n_part"])
    a = O.Oracle(p, c1_tables).initial(g, frozen=F)
    b = O.Oracle(dict(p, flags=FLAG_LEGENDRE_DIPOLE), c1_tables).initial(g, frozen=F)
    da = a["q"] - a["qs"] * (1 - 5e-5 / 2)
    db = b["q"] - b["qs"] * (1 - 5e-5 / 2)
    assert np.max(np.abs(db - 3 * da)) < 1e-9 * np.max(np.abs(db))
