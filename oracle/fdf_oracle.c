/*
 * fdf_oracle.c -- plain, slow, scalar FP64 CPU oracle of the fastdf hot path
 * (Elbers 2022, "Geodesic motion and phase-space evolution of massive
 * neutrinos", arXiv:2207.14256).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  The product path never
 * links, imports or calls it and shares no code with it.
 *
 * The oracle takes the method's steps in the paper's order:
 *   pre-initial sampling (Sec. 2.1), the momentum transform (eq:transform),
 *   the potential grids from transfer functions (Sec. 2.1), the leapfrog of the
 *   separable equations of motion (eq:releq_approx, eq:geodesic_approx) in
 *   Sec. 3.3 with constant d log a and conformal-time steps, the delta-f
 *   weight (Sec. 2.2) and the weighted density estimate (eq:empirical_rho)
 *   with a cloud-in-cell kernel.
 * Where the paper is silent the oracle follows one stated reading:
 *   R1  each kick integrates eps_0(a) and 1/eps_0(a) over its half-step with
 *       the potentials frozen at the half-step's end point, and each drift
 *       integrates 1/sqrt(q^2 + m^2 a^2) over the step with q frozen;
 *   the grid is a node grid x_n = n L/N, read and deposited with trilinear
 *   (cloud-in-cell) weights; p_k is the magnitude of the sampled vector.
 *
 * All arithmetic is IEEE FP64; build with -ffp-contract=off so no FMA forms.
 * OpenMP, when enabled, only splits loops over independent particles, modes or
 * FFT lines; the result does not depend on the thread count.
 *
 * Parity status: every function below is pinned by the CPU tests (closed
 * forms, brute force, library routines, invariants) except or_fields' choice
 * of synthetic physics, which is an input recipe, not a result.
 */
#include "fdf_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_KB_EV_PER_K 8.617333262e-5   /* Boltzmann constant in eV/K (SI 2019, exact) */
#define OR_C_OVER_H100 2997.92458       /* c / (100 km/s/Mpc) in Mpc */
#define OR_ZETA3 1.2020569031595942854  /* Apery's constant zeta(3) */
#define OR_PI 3.14159265358979323846
#define OR_NGL 16                       /* Gauss-Legendre nodes per step integral */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator, from its published definition      */
/* (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random numbers: as easy as  */
/* 1, 2, 3"): ten rounds of two 32x32->64 multiplies with a Weyl key bump.   */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* A uniform double in [0, 1) with 53 random bits from two 32-bit words. */
static double u53(uint32_t w0, uint32_t w1)
{
    return ((double)(w0 >> 5) * 67108864.0 + (double)(w1 >> 6)) * (1.0 / 9007199254740992.0);
}

static void philox_for(const or_params* p, uint64_t g, uint32_t stream, uint32_t attempt, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)g, (uint32_t)(g >> 32), stream, attempt};
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Background (the paper takes it from CLASS; reading: a flat radiation +    */
/* matter + Lambda stand-in).  Conformal-time steps of Sec. 3.3.            */
/* ------------------------------------------------------------------------ */
double or_hubble(const or_params* p, double a)
{
    double H0 = p->h / OR_C_OVER_H100;
    double ol = 1.0 - p->omega_m - p->omega_r;
    return H0 * sqrt(p->omega_r / (a * a * a * a) + p->omega_m / (a * a * a) + ol);
}

/* Nodes and weights of the n-point Gauss-Legendre rule on [-1, 1], by Newton
 * iteration on the three-term recurrence of the Legendre polynomials. */
void or_gauss_legendre(int n, double* x, double* w)
{
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            double dp = n * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        double p1 = 1.0, p2 = 0.0;
        for (int j = 1; j <= n; ++j) {
            double p3 = p2;
            p2 = p1;
            p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        double dp = n * (z * p1 - p2) / (z * z - 1.0);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

/* Quadrature nodes of one interval [l1, l2] in ln a: the integral of g(a)
 * d ln a / (a H(a)) equals sum_j wdt[j] g(a_j).  For l2 < l1 the weights are
 * negative, so a backward step integrates with the opposite sign. */
typedef struct {
    double wdt[OR_NGL];
    double a2[OR_NGL];
} or_quad;

static void quad_nodes(const or_params* p, double l1, double l2, or_quad* Q)
{
    double gx[OR_NGL], gw[OR_NGL];
    or_gauss_legendre(OR_NGL, gx, gw);
    double half = 0.5 * (l2 - l1), mid = 0.5 * (l1 + l2);
    for (int j = 0; j < OR_NGL; ++j) {
        double a = exp(mid + half * gx[j]);
        Q->wdt[j] = gw[j] * half / (a * or_hubble(p, a));
        Q->a2[j] = a * a;
    }
}

/* Delta tau between ln a = l1 and l2 (Sec. 3.3). */
double or_dtau(const or_params* p, double l1, double l2)
{
    or_quad Q;
    quad_nodes(p, l1, l2, &Q);
    double s = 0.0;
    for (int j = 0; j < OR_NGL; ++j) s += Q.wdt[j];
    return s;
}

/* Integrals over [l1, l2] of d tau / sqrt(q^2 + m^2 a^2) (kind 0) and of
 * sqrt(q^2 + m^2 a^2) d tau (kind 1).  Kind 0 with the current q is the drift
 * (eq:discrete_drift) integrated exactly for frozen q; with q_0 it is the
 * factor of the phi terms of eq:releq_approx; kind 1 with q_0 is the factor
 * of -grad psi. */
double or_eps_integral(const or_params* p, double m, double q, double l1, double l2, int kind)
{
    or_quad Q;
    quad_nodes(p, l1, l2, &Q);
    double s = 0.0;
    for (int j = 0; j < OR_NGL; ++j) {
        double e = sqrt(q * q + m * m * Q.a2[j]);
        s += kind ? Q.wdt[j] * e : Q.wdt[j] / e;
    }
    return s;
}

/* Adaptive Simpson quadrature (textbook, with the Richardson correction). */
typedef double (*or_fn)(const void* ctx, double x);

static double simpson_rec(or_fn f, const void* c, double a, double b, double fa, double fm, double fb,
                          double whole, double eps, int depth)
{
    double m = 0.5 * (a + b), lm = 0.5 * (a + m), rm = 0.5 * (m + b);
    double flm = f(c, lm), frm = f(c, rm);
    double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm);
    double right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
    double delta = left + right - whole;
    if (depth <= 0 || fabs(delta) <= 15.0 * eps) return left + right + delta / 15.0;
    return simpson_rec(f, c, a, m, fa, flm, fm, left, 0.5 * eps, depth - 1) +
           simpson_rec(f, c, m, b, fm, frm, fb, right, 0.5 * eps, depth - 1);
}

static double simpson(or_fn f, const void* c, double a, double b, double eps)
{
    double fa = f(c, a), fb = f(c, b), fm = f(c, 0.5 * (a + b));
    double whole = (b - a) / 6.0 * (fa + 4.0 * fm + fb);
    return simpson_rec(f, c, a, b, fa, fm, fb, whole, eps, 40);
}

static double tau_integrand(const void* c, double a)
{
    const or_params* p = (const or_params*)c;
    double H0 = p->h / OR_C_OVER_H100;
    double ol = 1.0 - p->omega_m - p->omega_r;
    return 1.0 / (H0 * sqrt(p->omega_r + p->omega_m * a + ol * a * a * a * a));
}

/* Conformal time tau(a) = int_0^a da' / (a'^2 H(a')). */
double or_tau(const or_params* p, double a)
{
    double guess = a * tau_integrand(p, 0.0);
    return simpson(tau_integrand, p, 0.0, a, 1e-15 * guess);
}

/* ------------------------------------------------------------------------ */
/* Homogeneous Fermi-Dirac distribution (Sec. 2, T = 1.95 K).                */
/* ------------------------------------------------------------------------ */
double or_temperature_ev(const or_params* p) { return p->T_K * OR_KB_EV_PER_K; }

static double fd_integrand(const void* c, double x)
{
    (void)c;
    return x * x / (1.0 + exp(x));
}

/* CDF of q^2 fbar(q) in x = q/T:  int_0^t x^2/(1+e^x) dx / (3 zeta(3)/2). */
double or_fd_cdf(double t)
{
    if (t <= 0.0) return 0.0;
    double s = 0.0, step = 0.25;
    for (double a = 0.0; a < t; a += step) {
        double b = a + step < t ? a + step : t;
        s += simpson(fd_integrand, NULL, a, b, 1e-16);
    }
    return s / (1.5 * OR_ZETA3);
}

/* ------------------------------------------------------------------------ */
/* Pre-initial sampling (Sec. 2.1): uniform positions in the periodic box,   */
/* |q| from fbar by inversion of the tabulated CDF, isotropic direction.     */
/* Only correctly rounded IEEE operations are used, so the result is exact.  */
/* ------------------------------------------------------------------------ */
static double fd_inverse(const or_tables* t, double u)
{
    int last = t->ncdf - 1;
    if (u >= t->cdf_F[last]) return t->cdf_t[last];
    int lo = 0, hi = last;          /* cdf_F[lo] <= u < cdf_F[hi] */
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (t->cdf_F[mid] <= u) lo = mid; else hi = mid;
    }
    double du = u - t->cdf_F[lo];
    double dt = t->cdf_t[lo + 1] - t->cdf_t[lo];
    double dF = t->cdf_F[lo + 1] - t->cdf_F[lo];
    return t->cdf_t[lo] + (du * dt) / dF;
}

double or_fd_inverse(const or_tables* t, double u) { return fd_inverse(t, u); }

/* Returns 0, or -1 if a direction could not be drawn in 64 attempts. */
int or_sample(const or_params* p, const or_tables* t, const int64_t* gidx, int64_t n,
              uint32_t* X, double* qs, double* pmag)
{
    const double T = or_temperature_ev(p);
    int fail = 0;
#pragma omp parallel for schedule(static) reduction(| : fail)
    for (int64_t i = 0; i < n; ++i) {
        uint64_t g = (uint64_t)gidx[i];
        uint32_t w[4], w2[4];
        /* stream 0: position, one 32-bit word per axis: x = L * X / 2^32 */
        philox_for(p, g, 0u, 0u, w);
        X[0 * n + i] = w[0];
        X[1 * n + i] = w[1];
        X[2 * n + i] = w[2];
        /* stream 1: momentum magnitude by inversion of the Fermi-Dirac CDF */
        philox_for(p, g, 1u, 0u, w);
        double qmag = T * fd_inverse(t, u53(w[0], w[1]));
        /* streams 2 and 3: direction by rejection from the cube [-1, 1)^3 */
        double v0 = 0, v1 = 0, v2 = 0, r2 = 0;
        int ok = 0;
        for (uint32_t att = 0; att < 64 && !ok; ++att) {
            philox_for(p, g, 2u, att, w);
            philox_for(p, g, 3u, att, w2);
            v0 = 2.0 * u53(w[0], w[1]) - 1.0;
            v1 = 2.0 * u53(w[2], w[3]) - 1.0;
            v2 = 2.0 * u53(w2[0], w2[1]) - 1.0;
            r2 = v0 * v0 + v1 * v1 + v2 * v2;
            ok = (r2 > 1e-300 && r2 <= 1.0);
        }
        if (!ok) { fail |= 1; continue; }
        double s = sqrt(r2);
        double q0 = qmag * (v0 / s), q1 = qmag * (v1 / s), q2 = qmag * (v2 / s);
        qs[0 * n + i] = q0;
        qs[1 * n + i] = q1;
        qs[2 * n + i] = q2;
        pmag[i] = sqrt(q0 * q0 + q1 * q1 + q2 * q2);
    }
    return fail ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Potential grids from transfer functions (Sec. 2.1).                       */
/* Field convention: f(x) = sum_n fhat_n exp(i k.x), k = 2 pi n / L.         */
/* ------------------------------------------------------------------------ */
static int signed_index(int j, int N) { return j < N / 2 ? j : j - N; }

/* Gaussian amplitude of one canonical mode n (no Hermitian bookkeeping). */
static double complex noise_mode(const or_params* p, int nx, int ny, int nz)
{
    const double L = p->box;
    uint64_t pack = (uint64_t)(nx + (1 << 20)) | ((uint64_t)(ny + (1 << 20)) << 21) |
                    ((uint64_t)(nz + (1 << 20)) << 42);
    uint32_t w[4];
    philox_for(p, pack, 16u, 0u, w);
    double u1 = ((double)(w[0] >> 8) + 1.0) * (1.0 / 16777216.0);   /* (0, 1] */
    double u2 = (double)(w[1] >> 8) * (1.0 / 16777216.0);           /* [0, 1) */
    double kf = 2.0 * OR_PI / L;
    double k = kf * sqrt((double)nx * nx + (double)ny * ny + (double)nz * nz);
    /* primordial curvature power P_R(k) = 2 pi^2 A_s k^-3 (k/k_pivot)^(n_s-1) */
    double PR = 2.0 * OR_PI * OR_PI * p->A_s / (k * k * k) * pow(k / p->k_pivot, p->n_s - 1.0);
    double amp = sqrt(PR / (L * L * L));
    if (p->flags & OR_FLAG_FIXED_AMPLITUDE)
        return amp * (cos(2.0 * OR_PI * u2) + I * sin(2.0 * OR_PI * u2));
    double r = sqrt(-2.0 * log(u1));
    return amp * (r * cos(2.0 * OR_PI * u2) + I * r * sin(2.0 * OR_PI * u2)) / sqrt(2.0);
}

static int is_canonical(int nx, int ny, int nz)
{
    return nz > 0 || (nz == 0 && (ny > 0 || (ny == 0 && nx > 0)));
}

/* The Hermitian Gaussian field R_n on the full N^3 mode array. */
void or_noise(const or_params* p, double complex* R)
{
    const int N = p->n_grid;
#pragma omp parallel for schedule(static)
    for (int jz = 0; jz < N; ++jz)
        for (int jy = 0; jy < N; ++jy)
            for (int jx = 0; jx < N; ++jx) {
                int nx = signed_index(jx, N), ny = signed_index(jy, N), nz = signed_index(jz, N);
                double complex v = 0.0;
                int nyq = (nx == -N / 2) || (ny == -N / 2) || (nz == -N / 2);
                if (!nyq && (nx || ny || nz)) {
                    if (is_canonical(nx, ny, nz)) v = noise_mode(p, nx, ny, nz);
                    else v = conj(noise_mode(p, -nx, -ny, -nz));
                }
                R[((size_t)jz * N + jy) * N + jx] = v;
            }
}

/* Bilinear interpolation in (ln k, ln a), clamped at the table edges. */
static int bracket(const double* x, int n, double v, double* f)
{
    if (v <= x[0]) { *f = 0.0; return 0; }
    if (v >= x[n - 1]) { *f = 1.0; return n - 2; }
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (x[mid] <= v) lo = mid; else hi = mid;
    }
    *f = (v - x[lo]) / (x[lo + 1] - x[lo]);
    return lo;
}

double or_interp_table(const or_tables* t, const double* T, double lnk, double lna)
{
    double fk, fa;
    int ik = bracket(t->lnk, t->nk, lnk, &fk);
    int ia = bracket(t->lna, t->na, lna, &fa);
    const double* r0 = T + (size_t)ia * t->nk;
    const double* r1 = T + (size_t)(ia + 1) * t->nk;
    double v0 = (1.0 - fk) * r0[ik] + fk * r0[ik + 1];
    double v1 = (1.0 - fk) * r1[ik] + fk * r1[ik + 1];
    return (1.0 - fa) * v0 + fa * v1;
}

/* In-place inverse DFT of one line, x_m = sum_n X_n exp(+2 pi i n m / N):
 * iterative radix-2 Cooley-Tukey with bit reversal; tw[j] = exp(2 pi i j/N). */
static void fft_line_inverse(int N, double complex* a, const double complex* tw)
{
    for (int i = 1, j = 0; i < N; ++i) {
        int bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { double complex t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (int len = 2; len <= N; len <<= 1) {
        int half = len / 2, stride = N / len;
        for (int i = 0; i < N; i += len)
            for (int k = 0; k < half; ++k) {
                double complex u = a[i + k], v = a[i + k + half] * tw[k * stride];
                a[i + k] = u + v;
                a[i + k + half] = u - v;
            }
    }
}

/* In-place unnormalised 3D inverse DFT of an N^3 array (x fastest). */
void or_fft3d_inverse(int N, double complex* d)
{
    double complex* tw = (double complex*)malloc(sizeof(double complex) * N);
    for (int j = 0; j < N; ++j) tw[j] = cos(2.0 * OR_PI * j / N) + I * sin(2.0 * OR_PI * j / N);
    for (int axis = 0; axis < 3; ++axis) {
        size_t stride = axis == 0 ? 1 : (axis == 1 ? (size_t)N : (size_t)N * N);
#pragma omp parallel
        {
            double complex* line = (double complex*)malloc(sizeof(double complex) * N);
#pragma omp for schedule(static)
            for (int l = 0; l < N * N; ++l) {
                int o1 = l % N, o2 = l / N;
                size_t base;
                if (axis == 0) base = (size_t)l * N;
                else if (axis == 1) base = (size_t)o2 * N * N + o1;
                else base = (size_t)o2 * N + o1;
                for (int m = 0; m < N; ++m) line[m] = d[base + m * stride];
                fft_line_inverse(N, line, tw);
                for (int m = 0; m < N; ++m) d[base + m * stride] = line[m];
            }
            free(line);
        }
    }
    free(tw);
}

/* The definition written out, for tiny N: out_m = sum_n in_n e^{2 pi i n.m/N}. */
void or_dft3d_inverse_naive(int N, const double complex* in, double complex* out)
{
    for (int mz = 0; mz < N; ++mz)
        for (int my = 0; my < N; ++my)
            for (int mx = 0; mx < N; ++mx) {
                double complex s = 0.0;
                for (int nz = 0; nz < N; ++nz)
                    for (int ny = 0; ny < N; ++ny)
                        for (int nx = 0; nx < N; ++nx) {
                            double ph = 2.0 * OR_PI * (double)((nx * mx + ny * my + nz * mz) % N) / N;
                            s += in[((size_t)nz * N + ny) * N + nx] * (cos(ph) + I * sin(ph));
                        }
                out[((size_t)mz * N + my) * N + mx] = s;
            }
}

/* Real-space fields at ln a: slots 0-2 grad psi, 3-5 grad phi, 6 phi_dot =
 * a H dphi/dln a, 7 psi (phi + psi if mask has OR_SLOT7_PHI_PLUS_PSI); only
 * slots set in mask are computed.  Each slot is
 * the inverse transform of its own Hermitian spectrum; max_imag returns the
 * largest |Im| met (zero up to round-off). */
void or_fields(const or_params* p, const or_tables* t, const double complex* R, double lna,
               unsigned mask, double* out, double* max_imag)
{
    const int N = p->n_grid;
    const size_t N3 = (size_t)N * N * N;
    const double kf = 2.0 * OR_PI / p->box;
    const double a = exp(lna);
    const double aH = a * or_hubble(p, a);
    double complex* s = (double complex*)malloc(sizeof(double complex) * N3);
    double mi = 0.0;
    for (int slot = 0; slot < 8; ++slot) {
        if (!(mask & (1u << slot))) continue;
#pragma omp parallel for schedule(static)
        for (size_t c = 0; c < N3; ++c) {
            int jx = (int)(c % N), jy = (int)((c / N) % N), jz = (int)(c / ((size_t)N * N));
            int n[3] = {signed_index(jx, N), signed_index(jy, N), signed_index(jz, N)};
            double complex v = 0.0;
            if (R[c] != 0.0) {
                double k = kf * sqrt((double)n[0] * n[0] + (double)n[1] * n[1] + (double)n[2] * n[2]);
                double lnk = log(k);
                if (slot < 3) v = I * (kf * n[slot]) * or_interp_table(t, t->T_psi, lnk, lna) * R[c];
                else if (slot < 6) v = I * (kf * n[slot - 3]) * or_interp_table(t, t->T_phi, lnk, lna) * R[c];
                else if (slot == 6) v = aH * or_interp_table(t, t->dTphi_dlna, lnk, lna) * R[c];
                else if (mask & OR_SLOT7_PHI_PLUS_PSI)
                    v = (or_interp_table(t, t->T_psi, lnk, lna) + or_interp_table(t, t->T_phi, lnk, lna)) * R[c];
                else v = or_interp_table(t, t->T_psi, lnk, lna) * R[c];
            }
            s[c] = v;
        }
        or_fft3d_inverse(N, s);
        for (size_t c = 0; c < N3; ++c) {
            out[(size_t)slot * N3 + c] = creal(s[c]);
            if (fabs(cimag(s[c])) > mi) mi = fabs(cimag(s[c]));
        }
    }
    if (max_imag) *max_imag = mi;
    free(s);
}

/* ------------------------------------------------------------------------ */
/* Interpolation from the node grid x_n = n L/N with the kernel of order r    */
/* (Sec. 4 offers r = 1 and r = 2): the B-spline of degree r, a product of    */
/* one-dimensional weights.                                                   */
/*   r = 1 (cloud-in-cell): nodes i, i+1 around u = x/h, weights 1-f, f.      */
/*   r = 2 (triangular-shaped cloud): the nearest node c and its neighbours,  */
/*        d = u - c in [-1/2, 1/2): (1/2 - d)^2/2, 3/4 - d^2, (1/2 + d)^2/2.  */
/* ------------------------------------------------------------------------ */
static int order_of(const or_params* p) { return p->interp_order == 2 ? 2 : 1; }

static int kernel1d(int order, int N, double u, int idx[3], double w[3])
{
    if (order == 2) {
        double c = floor(u + 0.5);
        double d = u - c;
        int i = (int)c % N;
        if (i < 0) i += N;
        idx[0] = (i + N - 1) % N;
        idx[1] = i;
        idx[2] = (i + 1) % N;
        w[0] = 0.5 * (0.5 - d) * (0.5 - d);
        w[1] = 0.75 - d * d;
        w[2] = 0.5 * (0.5 + d) * (0.5 + d);
        return 3;
    }
    double fl = floor(u);
    double f = u - fl;
    int i = (int)fl % N;
    if (i < 0) i += N;
    idx[0] = i;
    idx[1] = (i + 1) % N;
    w[0] = 1.0 - f;
    w[1] = f;
    return 2;
}

static void gather(int N, double L, int order, const double* F, unsigned mask, const double x[3], double out[8])
{
    const size_t N3 = (size_t)N * N * N;
    const double h = L / N;
    int idx[3][3];
    double w[3][3];
    int m = 0;
    for (int d = 0; d < 3; ++d) m = kernel1d(order, N, x[d] / h, idx[d], w[d]);
    for (int s = 0; s < 8; ++s) out[s] = 0.0;
    for (int cz = 0; cz < m; ++cz)
        for (int cy = 0; cy < m; ++cy)
            for (int cx = 0; cx < m; ++cx) {
                double wgt = w[0][cx] * w[1][cy] * w[2][cz];
                size_t c = ((size_t)idx[2][cz] * N + idx[1][cy]) * N + idx[0][cx];
                for (int s = 0; s < 8; ++s)
                    if (mask & (1u << s)) out[s] += wgt * F[(size_t)s * N3 + c];
            }
}

void or_gather(const or_params* p, const double* F, const double* x, double* out)
{
    gather(p->n_grid, p->box, order_of(p), F, 0xFFu, x, out);
}

/* Periodic wrap into [0, L). */
static double wrap(double x, double L)
{
    double y = x - L * floor(x / L);
    if (y < 0.0) y += L;
    if (y >= L) y = 0.0;
    return y;
}

/* ------------------------------------------------------------------------ */
/* Time grid: constant step in log a from z_start to z_end (Sec. 3.3).       */
/* ------------------------------------------------------------------------ */
double or_lna(const or_params* p, double k)
{
    double l0 = -log(1.0 + p->z_start), l1 = -log(1.0 + p->z_end);
    return l0 + k * ((l1 - l0) / p->n_steps);
}

static double mass_of(const or_params* p, int64_t g) { return p->m_ev[g / p->n_part]; }

/* One half-kick of eq:releq_approx (Sec. 3.3) with the potentials frozen at the half-step's
 * end point (reading R1): grad psi * int eps0 dtau, grad phi * q0^2 int
 * dtau/eps0, q0 (q0.grad phi) int dtau/eps0 and q0 phi_dot * int dtau. */
/*
 * The other equations of motion (eom), each with the momentum (q or the canonical
 * P) frozen at its z = 1e9 value so that the kick stays separable:
 *   1 eq:releq_lag (Sec. 3.2):  dP/dtau = -eps0 grad psi - (P0^2/eps0) grad phi
 *   2 eq:p_eq (Sec. 5):         dP/dtau = -((2 P0^2 + m^2 a^2)/eps0) grad psi
 *   3 eq:q_eq (Sec. 5):         dq/dtau = -eps0 grad psi
 *   4 Newtonian (Sec. 5):       dq/dtau = -m a grad psi  (reading: the paper's
 *                               dq/dt = -m grad psi per cosmic time, dtau = dt/a)
 * with eps0 = sqrt(P0^2 + m^2 a^2); the drift is eq:geodesic_approx for all.
 */
static void kick(const double g[8], const double q0[3], double m, const or_quad* Q, int eom, double q[3])
{
    double q02 = q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2];
    double Kpsi = 0.0, Kphi = 0.0, dtau = 0.0, Ka = 0.0;
    for (int j = 0; j < OR_NGL; ++j) {
        double e0 = sqrt(q02 + m * m * Q->a2[j]);
        Kpsi += Q->wdt[j] * e0;
        Kphi += Q->wdt[j] / e0;
        dtau += Q->wdt[j];
        Ka += Q->wdt[j] * m * sqrt(Q->a2[j]);
    }
    double qdphi = q0[0] * g[3] + q0[1] * g[4] + q0[2] * g[5];
    if (eom == 0) {
        for (int d = 0; d < 3; ++d)
            q[d] += -g[d] * Kpsi - g[3 + d] * (q02 * Kphi) + q0[d] * (qdphi * Kphi) + q0[d] * (g[6] * dtau);
        return;
    }
    for (int d = 0; d < 3; ++d) {
        if (eom == 1) q[d] += -g[d] * Kpsi - g[3 + d] * (q02 * Kphi);
        else if (eom == 2) q[d] += -g[d] * (Kpsi + q02 * Kphi);
        else if (eom == 3) q[d] += -g[d] * Kpsi;
        else q[d] += -g[d] * Ka;
    }
}

/* The fields used at step index k: the frozen set if given, else built. */
/* ------------------------------------------------------------------------ */
/* Super-steps (Sec. 2.1): the potential fields are computed only when the    */
/* transfer functions have changed by more than a fraction tol (the paper     */
/* uses 1%) since the last computed ones, and interpolated linearly between   */
/* these super-steps.  Reading: the change between steps j0 and j1 is, for    */
/* Q = T_psi and T_phi, the largest |Q(k, a_j1) - Q(k, a_j0)| over 64 ln k    */
/* points spanning the mesh's modes (2 pi/L to sqrt(3) pi N/L), relative to  */
/* the largest |Q(k, a_j0)| there; the larger of the two.  A step becomes a   */
/* super-step when its change from the last super-step exceeds tol; steps 0   */
/* and n_steps always are; interpolation is linear in ln a.                   */
/* ------------------------------------------------------------------------ */
double or_tf_change(const or_params* p, const or_tables* t, int j0, int j1)
{
    const double lk0 = log(2.0 * OR_PI / p->box), lk1 = log(sqrt(3.0) * OR_PI * p->n_grid / p->box);
    const double la0 = or_lna(p, j0), la1 = or_lna(p, j1);
    double worst = 0.0;
    for (int which = 0; which < 2; ++which) {
        const double* T = which ? t->T_phi : t->T_psi;
        double dmax = 0.0, qmax = 0.0;
        for (int i = 0; i < 64; ++i) {
            double lk = lk0 + (lk1 - lk0) * i / 63.0;
            double q0 = or_interp_table(t, T, lk, la0), q1 = or_interp_table(t, T, lk, la1);
            if (fabs(q1 - q0) > dmax) dmax = fabs(q1 - q0);
            if (fabs(q0) > qmax) qmax = fabs(q0);
        }
        if (qmax > 0.0 && dmax / qmax > worst) worst = dmax / qmax;
    }
    return worst;
}

void or_supersteps(const or_params* p, const or_tables* t, int* is_super)
{
    const int n = p->n_steps;
    for (int j = 0; j <= n; ++j) is_super[j] = !(p->superstep_tol > 0.0);
    is_super[0] = is_super[n] = 1;
    if (!(p->superstep_tol > 0.0)) return;
    int s = 0;
    for (int j = 1; j < n; ++j)
        if (or_tf_change(p, t, s, j) > p->superstep_tol) {
            is_super[j] = 1;
            s = j;
        }
}

typedef struct {
    const or_params* p;
    const or_tables* t;
    const double* frozen;
    double complex* R;
    int* is_super;          /* the super-step schedule, or NULL (every step computed) */
} field_src;

static void field_src_schedule(field_src* fs)
{
    fs->is_super = NULL;
    if (fs->frozen || !(fs->p->superstep_tol > 0.0)) return;
    fs->is_super = (int*)malloc(sizeof(int) * (fs->p->n_steps + 1));
    or_supersteps(fs->p, fs->t, fs->is_super);
}

static const double* fields_at(field_src* fs, double k, unsigned mask)
{
    if (fs->frozen) return fs->frozen;
    size_t N3 = (size_t)fs->p->n_grid * fs->p->n_grid * fs->p->n_grid;
    double* F = (double*)calloc(8 * N3, sizeof(double));
    const int kk = (int)k;
    if (!fs->is_super || fs->is_super[kk]) {
        or_fields(fs->p, fs->t, fs->R, or_lna(fs->p, k), mask, F, NULL);
        return F;
    }
    /* between the super-steps s < k < e: linear in ln a */
    int s = kk, e = kk;
    while (!fs->is_super[s]) --s;
    while (!fs->is_super[e]) ++e;
    double* Fs = (double*)calloc(8 * N3, sizeof(double));
    double* Fe = (double*)calloc(8 * N3, sizeof(double));
    or_fields(fs->p, fs->t, fs->R, or_lna(fs->p, s), mask, Fs, NULL);
    or_fields(fs->p, fs->t, fs->R, or_lna(fs->p, e), mask, Fe, NULL);
    const double w = (or_lna(fs->p, k) - or_lna(fs->p, s)) / (or_lna(fs->p, e) - or_lna(fs->p, s));
    for (size_t i = 0; i < 8 * N3; ++i) F[i] = (1.0 - w) * Fs[i] + w * Fe[i];
    free(Fs);
    free(Fe);
    return F;
}

static void fields_done(field_src* fs, const double* F)
{
    if (F != fs->frozen) free((void*)F);
}

/* ------------------------------------------------------------------------ */
/* Pre-initial transform (eq:transform, Sec. 2.1) with delta = -2 psi and   */
/* theta = k^2 tau psi / 2 (Sec. 2.1), nu = 4, omega = 4/3:                  */
/*   q_i <- q_i (1 - psi/2) - (eps tau_0 / 6) d_i psi.                       */
/* ------------------------------------------------------------------------ */
int or_initial(const or_params* p, const or_tables* t, const double* frozen, const int64_t* gidx,
               int64_t n, uint32_t* X, double* qs, double* pmag, double* x, double* q, double* q0)
{
    if (or_sample(p, t, gidx, n, X, qs, pmag) != 0) return -1;
    const int N = p->n_grid;
    const size_t N3 = (size_t)N * N * N;
    field_src fs = {p, t, frozen, NULL, NULL};
    if (!frozen) {
        fs.R = (double complex*)malloc(sizeof(double complex) * N3);
        or_noise(p, fs.R);
    }
    field_src_schedule(&fs);
    const double* F = fields_at(&fs, 0.0, 0xFFu);
    const double a0 = exp(or_lna(p, 0.0));
    const double tau0 = or_tau(p, a0);
    const double L = p->box;
    /* eq:transform with nu = 4, omega = 4/3: 1 + delta/nu = 1 - psi/2 and
     * (omega eps/nu) grad(nabla^-2 theta) = (eps/3)(-tau0/2) grad psi = -(eps tau0/6) grad psi.
     * The paper expands Psi in Legendre terms with the factor 2l+1 (eq:def2), which
     * puts a factor 3 on the dipole that eq:pre_int and eq:transform do not print;
     * flag bit 1 takes that reading (the dipole then carries the flux theta). */
    const double dip = (p->flags & OR_FLAG_LEGENDRE_DIPOLE) ? 3.0 : 1.0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double xi[3], g[8];
        for (int d = 0; d < 3; ++d) xi[d] = L * ((double)X[d * n + i] * (1.0 / 4294967296.0));
        gather(N, L, order_of(p), F, 0xFFu, xi, g);
        double m = mass_of(p, gidx[i]);
        double eps = sqrt(pmag[i] * pmag[i] + m * m * a0 * a0);
        for (int d = 0; d < 3; ++d) {
            double qd = qs[d * n + i] * (1.0 - g[7] / 2.0) - dip * (eps * tau0 / 6.0) * g[d];
            x[d * n + i] = xi[d];
            q[d * n + i] = qd;
            q0[d * n + i] = qd;
        }
    }
    fields_done(&fs, F);
    free(fs.R);
    free(fs.is_super);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Leapfrog (Sec. 3.3) from step index k_from to k_to (backward if smaller): */
/*   q_{k+1/2} = q_k + kick(x_k, a_k; [a_k, a_{k+1/2}])                      */
/*   x_{k+1}   = x_k + q_{k+1/2} int_{a_k}^{a_{k+1}} dtau / eps              */
/*   q_{k+1}   = q_{k+1/2} + kick(x_{k+1}, a_{k+1}; [a_{k+1/2}, a_{k+1}])    */
/*                                                                          */
/* eom 5, the non-symplectic leapfrog on the exact eq:releq and             */
/* eq:geodesic that Sec. 3.3 uses as a check (reading: the same three       */
/* stages, each explicit in what it does not advance):                      */
/*   each half kick is eq:releq with q, eps = sqrt(q^2 + m^2 a^2) and the   */
/*   products q (q.grad phi), q phi_dot held at the kick's starting q (the  */
/*   kick of eom 0 with that q in place of q0);                             */
/*   the drift is eq:geodesic, x_{k+1} = x_k + (1 + phi + psi)_k q_{k+1/2}  */
/*   int dtau / eps, with phi + psi read at x_k from the fields of a_k.     */
/* ------------------------------------------------------------------------ */
int or_integrate(const or_params* p, const or_tables* t, const double* frozen, const int64_t* gidx,
                 int64_t n, int k_from, int k_to, double* x, double* q, const double* q0)
{
    if (k_from == k_to) return 0;
    const int N = p->n_grid;
    const size_t N3 = (size_t)N * N * N;
    const int dir = k_to > k_from ? 1 : -1;
    const double L = p->box;
    field_src fs = {p, t, frozen, NULL, NULL};
    if (!frozen) {
        fs.R = (double complex*)malloc(sizeof(double complex) * N3);
        or_noise(p, fs.R);
    }
    field_src_schedule(&fs);
    const int exact = p->eom == 5;
    const unsigned gmask = exact ? 0xFFu : 0x7Fu;
    const unsigned fmask = exact ? (0xFFu | OR_SLOT7_PHI_PLUS_PSI) : 0x7Fu;
    const double* Fk = fields_at(&fs, (double)k_from, fmask);
    for (int k = k_from; k != k_to; k += dir) {
        const double* Fn = fields_at(&fs, (double)(k + dir), fmask);
        double lk = or_lna(p, k), lh = or_lna(p, k + 0.5 * dir), ln = or_lna(p, k + dir);
        or_quad Qopen, Qdrift, Qclose;
        quad_nodes(p, lk, lh, &Qopen);
        quad_nodes(p, lk, ln, &Qdrift);
        quad_nodes(p, lh, ln, &Qclose);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double m = mass_of(p, gidx[i]);
            double xi[3], qi[3], q0i[3], g[8];
            for (int d = 0; d < 3; ++d) {
                xi[d] = x[d * n + i];
                qi[d] = q[d * n + i];
                q0i[d] = q0[d * n + i];
            }
            gather(N, L, order_of(p), Fk, gmask, xi, g);
            const double metric = exact ? 1.0 + g[7] : 1.0;   /* (1 + phi + psi) at x_k, a_k */
            if (exact) {
                double qstart[3] = {qi[0], qi[1], qi[2]};
                kick(g, qstart, m, &Qopen, 0, qi);
            } else {
                kick(g, q0i, m, &Qopen, p->eom, qi);
            }
            double qq = qi[0] * qi[0] + qi[1] * qi[1] + qi[2] * qi[2];
            double D = 0.0;
            for (int j = 0; j < OR_NGL; ++j) D += Qdrift.wdt[j] / sqrt(qq + m * m * Qdrift.a2[j]);
            for (int d = 0; d < 3; ++d) xi[d] = wrap(xi[d] + metric * D * qi[d], L);
            gather(N, L, order_of(p), Fn, gmask, xi, g);
            if (exact) {
                double qstart[3] = {qi[0], qi[1], qi[2]};
                kick(g, qstart, m, &Qclose, 0, qi);
            } else {
                kick(g, q0i, m, &Qclose, p->eom, qi);
            }
            for (int d = 0; d < 3; ++d) {
                x[d * n + i] = xi[d];
                q[d * n + i] = qi[d];
            }
        }
        fields_done(&fs, Fk);
        Fk = Fn;
    }
    fields_done(&fs, Fk);
    free(fs.R);
    free(fs.is_super);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The four terms of eq:releq (Sec. 3.2), whose root mean square over the     */
/* particles Fig. 2 plots from z = 1e9 to 0:                                 */
/*   T1 = -eps grad psi,  T2 = -(q^2/eps) grad phi,  T3 = q (q.grad phi)/eps, */
/*   T4 = q phi_dot,      eps = sqrt(q^2 + m^2 a^2),                         */
/* at each particle's x and q with the fields of step k.  out[i] = sqrt of   */
/* the mean of |T_{i+1}|^2 over the n particles; out[4] the same for the     */
/* sum T1 + T2 + T3 + T4 (the whole acceleration).                            */
/* ------------------------------------------------------------------------ */
int or_accel_terms(const or_params* p, const or_tables* t, const double* frozen, const int64_t* gidx, int64_t n,
                   int k, const double* x, const double* q, double* out)
{
    const int N = p->n_grid;
    const size_t N3 = (size_t)N * N * N;
    field_src fs = {p, t, frozen, NULL, NULL};
    if (!frozen) {
        fs.R = (double complex*)malloc(sizeof(double complex) * N3);
        or_noise(p, fs.R);
    }
    field_src_schedule(&fs);
    const double* F = fields_at(&fs, (double)k, 0x7Fu);
    const double a = exp(or_lna(p, k));
    double sum[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) {
        double xi[3], qi[3], g[8];
        for (int d = 0; d < 3; ++d) {
            xi[d] = x[d * n + i];
            qi[d] = q[d * n + i];
        }
        gather(N, p->box, order_of(p), F, 0x7Fu, xi, g);
        const double m = mass_of(p, gidx[i]);
        const double qq = qi[0] * qi[0] + qi[1] * qi[1] + qi[2] * qi[2];
        const double eps = sqrt(qq + m * m * a * a);
        const double qdphi = qi[0] * g[3] + qi[1] * g[4] + qi[2] * g[5];
        for (int d = 0; d < 3; ++d) {
            const double T[4] = {-eps * g[d], -(qq / eps) * g[3 + d], qi[d] * qdphi / eps, qi[d] * g[6]};
            for (int j = 0; j < 4; ++j) sum[j] += T[j] * T[j];
            const double tot = T[0] + T[1] + T[2] + T[3];
            sum[4] += tot * tot;
        }
    }
    for (int j = 0; j < 5; ++j) out[j] = n > 0 ? sqrt(sum[j] / (double)n) : 0.0;
    fields_done(&fs, F);
    free(fs.R);
    free(fs.is_super);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* delta-f weight (Sec. 2.2): w = 1 - fbar(|q|)/fbar(p), written as          */
/*   w = -expm1((p - |q|)/T) / (1 + exp(-|q|/T)),                            */
/* which is the same quantity without cancellation or overflow.              */
/* ------------------------------------------------------------------------ */
void or_weights(const or_params* p, int64_t n, const double* q, const double* pmag, double* w)
{
    const double T = or_temperature_ev(p);
    for (int64_t i = 0; i < n; ++i) {
        double qm = sqrt(q[i] * q[i] + q[n + i] * q[n + i] + q[2 * n + i] * q[2 * n + i]);
        w[i] = -expm1((pmag[i] - qm) / T) / (1.0 + exp(-qm / T));
    }
}

/* ------------------------------------------------------------------------ */
/* Density estimate (eq:empirical_rho, Sec. 2.2) on the node grid, CIC:     */
/*   grid[n] += v_k W(x_n - x_k), v_k = w_k eps_k (quantity 0), w_k (1),     */
/*   eps_k (2) or 1 (3); eps_k = sqrt(|q_k|^2 + m^2 a^2).  The raw sum is    */
/*   returned; the paper's M/N normalisation is left to the caller.          */
/* ------------------------------------------------------------------------ */
void or_deposit(const or_params* p, const int64_t* gidx, int64_t n, const double* x, const double* q,
                const double* w, double a, int quantity, double* grid)
{
    const int N = p->n_grid, order = order_of(p);
    const double L = p->box, h = L / N;
    for (int64_t i = 0; i < n; ++i) {
        double m = mass_of(p, gidx[i]);
        double qq = q[i] * q[i] + q[n + i] * q[n + i] + q[2 * n + i] * q[2 * n + i];
        double eps = sqrt(qq + m * m * a * a);
        /* 0: w eps (eq:empirical_rho), 1: w, 2: eps, 3: 1, 4-6: w q_x, w q_y, w q_z
         * (the delta-f momentum density, whose divergence gives (1 + delta) theta) */
        double v = quantity == 0 ? w[i] * eps
                 : quantity == 1 ? w[i]
                 : quantity == 2 ? eps
                 : quantity == 3 ? 1.0
                 : w[i] * q[(size_t)(quantity - 4) * n + i];
        int idx[3][3];
        double wt[3][3];
        int mm = 0;
        for (int d = 0; d < 3; ++d) {
            double xd = x[d * n + i];
            mm = kernel1d(order, N, xd / h, idx[d], wt[d]);
        }
        for (int cz = 0; cz < mm; ++cz)
            for (int cy = 0; cy < mm; ++cy)
                for (int cx = 0; cx < mm; ++cx) {
                    double wgt = wt[0][cx] * wt[1][cy] * wt[2][cz];
                    size_t c = ((size_t)idx[2][cz] * N + idx[1][cy]) * N + idx[0][cx];
                    grid[c] += wgt * v;
                }
    }
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
