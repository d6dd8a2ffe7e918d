"""Pins of the oracle's potential grids (Sec. 2.1: potentials from transfer functions).

Pins: the radix-2 FFT against the DFT written out (brute force) and against
numpy.fft; the Hermitian noise (R_-n = conj R_n, zero mean mode and Nyquist
planes, |R| = sqrt(P/V) for fixed amplitudes); a single canonical mode against
the analytic cosine and sine fields, which fixes the sign of i k and the
normalisation; Parseval's identity for the grid variance; bilinear table
interpolation against a table that is itself bilinear.
"""
import math

import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("N", [2, 4, 8])
def test_fft_against_naive_dft(N):
    rng = np.random.default_rng(N)
    a = rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))
    f = O.fft3d_inverse(a)
    d = O.dft3d_inverse_naive(a)
    assert np.max(np.abs(f - d)) < 1e-12 * np.max(np.abs(d))


@pytest.mark.parametrize("N", [16, 32])
def test_fft_against_numpy(N):
    rng = np.random.default_rng(N)
    a = rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))
    f = O.fft3d_inverse(a)
    ref = np.fft.ifftn(a) * N ** 3
    assert np.max(np.abs(f - ref)) < 1e-12 * np.max(np.abs(ref))


def _sidx(N):
    j = np.arange(N)
    return np.where(j < N // 2, j, j - N)


def test_noise_hermitian_and_amplitude(inputs, c1_tables):
    for flags in (0, 1):
        p = inputs.config("c1_32", n_grid=16, flags=flags, seed=9)
        o = O.Oracle(p, c1_tables)
        R = o.noise()
        N = 16
        n = _sidx(N)
        nz, ny, nx = np.meshgrid(n, n, n, indexing="ij")
        neg = (-np.arange(N)) % N
        Rm = R[np.ix_(neg, neg, neg)]
        assert np.array_equal(R, np.conj(Rm))
        assert R[0, 0, 0] == 0
        assert np.all(R[N // 2, :, :] == 0) and np.all(R[:, N // 2, :] == 0) and np.all(R[:, :, N // 2] == 0)
        L = p["box"]
        k = 2 * math.pi / L * np.sqrt(nx ** 2 + ny ** 2 + nz ** 2)
        nyq = (nx == -N // 2) | (ny == -N // 2) | (nz == -N // 2)
        ok = (k > 0) & ~nyq
        PR = 2 * math.pi ** 2 * p["A_s"] / k[ok] ** 3 * (k[ok] / p["k_pivot"]) ** (p["n_s"] - 1)
        ratio = np.abs(R[ok]) ** 2 / (PR / L ** 3)
        if flags:
            assert np.allclose(ratio, 1.0, rtol=1e-13)
        else:
            # |R|^2 / (P/V) is exponential with mean 1 (two Gaussian components of variance 1/2)
            assert abs(ratio.mean() - 1) < 4 / math.sqrt(ratio.size)


def test_single_mode_fields_analytic(inputs, c1_tables):
    N, L = 16, 1000.0
    p = inputs.config("c1_32", n_grid=N, box=L)
    o = O.Oracle(p, c1_tables)
    A = 1e-5 * (0.6 - 0.8j)
    mode = (2, 1, 3)   # (n_x, n_y, n_z), canonical since n_z > 0
    R = np.zeros((N, N, N), complex)
    R[mode[2], mode[1], mode[0]] = A
    R[(-mode[2]) % N, (-mode[1]) % N, (-mode[0]) % N] = np.conj(A)
    lna = o.lna(40)
    F, mi = o.fields(lna, 0xFF, R)
    kvec = 2 * math.pi / L * np.asarray(mode, float)
    kmag = np.linalg.norm(kvec)
    Tpsi = o.interp_table("T_psi", math.log(kmag), lna)
    Tphi = o.interp_table("T_phi", math.log(kmag), lna)
    dT = o.interp_table("dTphi_dlna", math.log(kmag), lna)
    aH = math.exp(lna) * o.hubble(math.exp(lna))
    xs = np.arange(N) * (L / N)
    z, y, x = np.meshgrid(xs, xs, xs, indexing="ij")
    ph = kvec[0] * x + kvec[1] * y + kvec[2] * z + np.angle(A)
    S, Cc = np.sin(ph), np.cos(ph)
    scale = 2 * abs(A)
    for d in range(3):
        assert np.allclose(F[d], -scale * Tpsi * kvec[d] * S, atol=1e-12 * scale * kmag, rtol=0)
        assert np.allclose(F[3 + d], -scale * Tphi * kvec[d] * S, atol=1e-12 * scale * kmag, rtol=0)
    assert np.allclose(F[6], scale * aH * dT * Cc, atol=1e-12 * scale * abs(aH * dT) + 1e-300, rtol=0)
    assert np.allclose(F[7], scale * Tpsi * Cc, atol=1e-12 * scale, rtol=0)
    assert mi < 1e-12 * scale * kmag


def test_fields_parseval_and_real(inputs, c1_tables):
    N = 16
    p = inputs.config("c1_32", n_grid=N, seed=4)
    o = O.Oracle(p, c1_tables)
    R = o.noise()
    lna = o.lna(70)
    F, mi = o.fields(lna, 0xFF, R)
    assert mi < 1e-12 * np.abs(F).max()
    n = _sidx(N)
    nz, ny, nx = np.meshgrid(n, n, n, indexing="ij")
    k = 2 * math.pi / p["box"] * np.sqrt(nx ** 2 + ny ** 2 + nz ** 2)
    T = np.zeros_like(k)
    for idx in zip(*np.nonzero(k)):
        T[idx] = o.interp_table("T_psi", math.log(k[idx]), lna)
    # (1/N^3) sum_x psi^2 = sum_n |T R_n|^2
    assert abs(np.mean(F[7] ** 2) / np.sum(np.abs(T * R) ** 2) - 1) < 1e-12
    kx = 2 * math.pi / p["box"] * nx
    assert abs(np.mean(F[0] ** 2) / np.sum(np.abs(kx * T * R) ** 2) - 1) < 1e-12


def test_bilinear_table_interpolation(inputs, c1_tables):
    t = dict(c1_tables)
    lnk, lna = t["lnk"], t["lna"]
    bil = (0.3 + 0.2 * lnk[None, :]) * (1.5 - 0.05 * lna[:, None])
    t["T_psi"] = bil
    o = O.Oracle(inputs.config("c1_32"), t)
    rng = np.random.default_rng(1)
    for _ in range(50):
        x = rng.uniform(lnk[0], lnk[-1])
        y = rng.uniform(lna[0], lna[-1])
        assert abs(o.interp_table("T_psi", x, y) - (0.3 + 0.2 * x) * (1.5 - 0.05 * y)) < 1e-13
    # clamped outside the table
    assert abs(o.interp_table("T_psi", lnk[0] - 5, lna[-1] + 3) - bil[-1, 0]) < 1e-15
