/*
 * fdf_oracle.h -- interface of the plain scalar FP64 CPU oracle of the fastdf
 * hot path (Elbers 2022, "Geodesic motion and phase-space evolution of massive
 * neutrinos", arXiv:2207.14256).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and oracle/fdf_oracle.c are loaded by
 * the test-suite, by the smoke check and by the benchmark's CPU-baseline leg,
 * and by nothing else.  The product library (libfdf.so) neither includes this
 * header nor links the oracle; the two share no code, no header and no table.
 *
 * Units: Mpc for lengths and conformal time (c = 1), eV for momenta, masses
 * and temperature.  Arrays of 3-vectors are SoA: v[c*n + i], c = 0,1,2.
 * Field grids are [8][N^3] with the cell index (iz*N + iy)*N + ix and the slot
 * order (d_x psi, d_y psi, d_z psi, d_x phi, d_y phi, d_z phi, phi_dot, psi).
 */
#ifndef FDF_ORACLE_H
#define FDF_ORACLE_H
#include <stdint.h>

typedef struct {
    double   box;          /* L, Mpc */
    int64_t  n_part;       /* particles per species */
    int32_t  n_grid;       /* N, a power of two */
    int32_t  n_species;
    double   m_ev[4];      /* neutrino mass per species, eV */
    double   T_K;          /* present-day neutrino temperature, K (paper: 1.95) */
    double   z_start, z_end;
    int32_t  n_steps;
    int32_t  flags;        /* bit 0: fixed amplitudes (|R| = sqrt(P/V)); bit 1: the dipole term of
                              eq:transform with the factor 2l+1 = 3 of eq:def2 */
    uint64_t seed;
    double   h, omega_m, omega_r;   /* Omega_Lambda = 1 - omega_m - omega_r */
    double   A_s, n_s, k_pivot;
    int32_t  interp_order; /* interpolation order r of Sec. 4: 1 (or 0) cloud-in-cell, 2 TSC */
    double   superstep_tol; /* super-steps of Sec. 2.1: > 0 builds the fields only where the
                               transfer functions changed by more than this fraction (paper:
                               0.01) and interpolates linearly in ln a in between; 0 = off */
    int32_t  eom;           /* equation of motion of the kick, each with the momentum frozen at
                               its z = 1e9 value (separable, symplectic):
                               0 eq:releq_approx (Sec. 3.3, the method's), 1 eq:releq_lag
                               (canonical P), 2 eq:p_eq (special-relativistic, Newtonian
                               gravity), 3 eq:q_eq (Sec. 5's simpler form), 4 Newtonian
                               acceleration -m a grad psi (Sec. 5); or
                               5 the exact eq:releq and eq:geodesic in the non-symplectic
                               leapfrog of Sec. 3.3 (or_integrate says how) */
} or_params;

/* or_fields mask bit: slot 7 holds phi + psi (the drift factor of eq:geodesic)
 * instead of psi. */
#define OR_SLOT7_PHI_PLUS_PSI 0x100u

typedef struct {
    int32_t nk, na;
    const double *lnk, *lna;                    /* ascending node positions */
    const double *T_psi, *T_phi, *dTphi_dlna;   /* [na][nk] */
    int32_t ncdf;
    const double *cdf_t, *cdf_F;                /* q/T nodes, normalised CDF */
} or_tables;

#define OR_FLAG_FIXED_AMPLITUDE 1
#define OR_FLAG_LEGENDRE_DIPOLE 2

#endif
