"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds no arithmetic of the method itself.  It produces the data a
user of the method brings along:

* run parameters for the workloads the library is measured on (particle count,
  grid size, box, mass, redshift range, step count, seed, cosmology);
* smooth transfer-function tables T_psi(k, a), T_phi(k, a) and
  dT_phi/dln a on a uniform (ln k, ln a) grid.  In the paper these come from
  CLASS (Sec. 2.1); here a closed-form stand-in with the same qualitative shape
  replaces them: a radiation-era decay 3 (sin x - x cos x) / x^3 at horizon
  entry and a matter-era plateau with a smooth small-scale cut-off;
* the cumulative distribution of q^2 fbar(q) for the Fermi-Dirac function
  fbar(q) = 1 / (1 + exp(q/T)) of Sec. 2, tabulated in q/T so that momenta can
  be drawn by inversion with exactly rounded arithmetic on every device.

Both the product path and the oracle receive these arrays unchanged.
"""
import math

import numpy as np

C_OVER_H100 = 2997.92458  # c / (100 km/s/Mpc) in Mpc


def omega_radiation(h: float) -> float:
    """Photons (T_cmb = 2.7255 K) plus 3.046 massless neutrino species."""
    return 2.4728e-5 * (1.0 + 3.046 * (7.0 / 8.0) * (4.0 / 11.0) ** (4.0 / 3.0)) / (h * h)


def base_params(**over) -> dict:
    h = 0.67
    p = dict(box=1000.0, n_part=32 ** 3, n_grid=32, n_species=1, m_ev=[0.1], T_K=1.95, z_start=1e9, z_end=31.0,
             n_steps=100, flags=0, seed=1, h=h, omega_m=0.31, omega_r=omega_radiation(h), A_s=2.1e-9, n_s=0.965,
             k_pivot=0.05, precision=0, n_gl=0, sort_every=0)
    p.update(over)
    return p


#: Precision settings (include/fdf.h FDF_PREC_*): FP64 everywhere; FP32 or BF16 grids with
#: an FP64 phase-space state; FP32 or BF16 grids with the split (fixed-point) state.
PREC_F64, PREC_F32, PREC_BF16, PREC_F32_FIXED, PREC_BF16_FIXED = 0, 1, 2, 3, 4

#: The four measured workloads.  The first is small enough for the oracle to
#: run in full in seconds; the third (three species of 256^3 particles on a
#: 256^3 grid) is the throughput workload.
CONFIGS = {
    "c1_32": base_params(box=1000.0, n_part=32 ** 3, n_grid=32, m_ev=[0.1], seed=1, n_steps=100,
                         precision=PREC_F64),
    "c2_128": base_params(box=1000.0, n_part=128 ** 3, n_grid=128, m_ev=[0.06], seed=2, n_steps=200,
                          precision=PREC_F32),
    "c3_3x256": base_params(box=2000.0, n_part=256 ** 3, n_grid=256, n_species=3, m_ev=[0.1, 0.1, 0.1], seed=3,
                            n_steps=200, precision=PREC_F32),
    "c4_512_bf16": base_params(box=1000.0, n_part=512 ** 3, n_grid=256, m_ev=[0.05], seed=2, n_steps=300,
                               precision=PREC_BF16),
}


def config(name: str, **over) -> dict:
    p = dict(CONFIGS[name])
    p["m_ev"] = list(p["m_ev"])
    p.update(over)
    return p


# ----------------------------------------------------------------------------------------
# Fermi-Dirac CDF table
# ----------------------------------------------------------------------------------------
def fd_cdf_table(n: int = 4001, t_max: float = 40.0):
    """Nodes t_j = j * t_max/(n-1) and F_j = int_0^t_j x^2/(1+e^x) dx / (3 zeta(3)/2).

    Each interval is integrated with a 12-point Gauss-Legendre rule (the
    integrand is entire, so this is exact to rounding on intervals of 0.01) and
    the partial sums are accumulated with Neumaier compensation.
    """
    from scipy.special import zeta

    t = np.arange(n, dtype=np.float64) * (t_max / (n - 1))
    gx, gw = np.polynomial.legendre.leggauss(12)
    a, b = t[:-1], t[1:]
    mid, half = 0.5 * (a + b), 0.5 * (b - a)
    xs = mid[:, None] + half[:, None] * gx[None, :]
    f = xs * xs / (1.0 + np.exp(xs))
    pieces = (f * gw[None, :]).sum(axis=1) * half
    F = np.zeros(n)
    s = c = 0.0  # Neumaier-compensated running sum
    for j in range(1, n):
        v = float(pieces[j - 1])
        t_ = s + v
        c += (s - t_) + v if abs(s) >= abs(v) else (v - t_) + s
        s = t_
        F[j] = s + c
    F /= 1.5 * float(zeta(3.0))
    return t, F


# ----------------------------------------------------------------------------------------
# Synthetic transfer tables
# ----------------------------------------------------------------------------------------
def _tau_rm(a, h, om, orad):
    """Closed-form conformal time of a radiation + matter universe (shape only)."""
    H0 = h / C_OVER_H100
    aeq = orad / om
    return 2.0 / (H0 * math.sqrt(om)) * (np.sqrt(a + aeq) - math.sqrt(aeq))


def _T_shapes(lnk, lna, h, om, orad):
    k = np.exp(lnk)[None, :]
    a = np.exp(lna)[:, None]
    aeq = orad / om
    H0 = h / C_OVER_H100
    keq = aeq * H0 * math.sqrt(orad / aeq ** 4 + om / aeq ** 3 + (1.0 - om - orad))
    r = 1.0 / (1.0 + a / aeq)
    x = k * _tau_rm(a, h, om, orad) / math.sqrt(3.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        J = np.where(x < 1e-3, 1.0 - x * x / 10.0, 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3)
    B = 1.0 / (1.0 + (k / keq) ** 2)
    T_psi = (2.0 / 3.0) * r * J + (3.0 / 5.0) * (1.0 - r) * B
    T_phi = T_psi * (1.0 + 0.4 * 0.405 * r)
    return T_psi, T_phi


def transfer_tables(params: dict, nk: int = 256, na: int = 64, k_min: float = 1e-4, k_max: float = 10.0,
                    a_min: float = 1e-10, a_max: float = 1.0) -> dict:
    """Tables on a uniform (ln k, ln a) grid, arrays [na][nk] in float64."""
    h, om, orad = params["h"], params["omega_m"], params["omega_r"]
    lnk = np.linspace(math.log(k_min), math.log(k_max), nk)
    lna = np.linspace(math.log(a_min), math.log(a_max), na)
    T_psi, T_phi = _T_shapes(lnk, lna, h, om, orad)
    # d T_phi / d ln a by a Richardson-extrapolated central difference
    e = 1e-3
    d1 = (_T_shapes(lnk, lna + e, h, om, orad)[1] - _T_shapes(lnk, lna - e, h, om, orad)[1]) / (2 * e)
    d2 = (_T_shapes(lnk, lna + e / 2, h, om, orad)[1] - _T_shapes(lnk, lna - e / 2, h, om, orad)[1]) / e
    dT = (4.0 * d2 - d1) / 3.0
    t, F = fd_cdf_table()
    return dict(lnk=lnk, lna=lna, T_psi=np.ascontiguousarray(T_psi), T_phi=np.ascontiguousarray(T_phi),
                dTphi_dlna=np.ascontiguousarray(dT), cdf_t=t, cdf_F=F)


def zero_tables(tables: dict) -> dict:
    """The same tables with every transfer function set to zero (phi = psi = 0)."""
    z = dict(tables)
    for k in ("T_psi", "T_phi", "dTphi_dlna"):
        z[k] = np.zeros_like(tables[k])
    return z


def uniform_fields(N: int, grad_psi, grad_phi, phi_dot, psi=0.0) -> np.ndarray:
    """Constant fields [8][N][N][N] (d psi, d phi, phi_dot, psi) for injection tests."""
    v = list(grad_psi) + list(grad_phi) + [phi_dot, psi]
    return np.broadcast_to(np.asarray(v, np.float64)[:, None, None, None], (8, N, N, N)).copy()


def cosine_fields(N: int, box: float, amp: float, n_mode=(1, 0, 0)) -> np.ndarray:
    """Smooth single-mode fields: psi = phi = amp cos(k.x) on the node grid."""
    k = 2 * math.pi / box * np.asarray(n_mode, np.float64)
    idx = np.arange(N) * (box / N)
    z, y, x = np.meshgrid(idx, idx, idx, indexing="ij")
    ph = k[0] * x + k[1] * y + k[2] * z
    c, s = np.cos(ph), np.sin(ph)
    F = np.zeros((8, N, N, N))
    for d in range(3):
        F[d] = -amp * k[d] * s
        F[3 + d] = -amp * k[d] * s
    F[7] = amp * c
    return F
