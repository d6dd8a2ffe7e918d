/*
 * fdf.h -- C-ABI of libfdf.so: GB300 (sm_103a) integration of massive-neutrino
 * particles along geodesics of a linearly perturbed spacetime, the fastdf
 * method of Elbers 2022, "Geodesic motion and phase-space evolution of massive
 * neutrinos" (arXiv:2207.14256).
 *
 * The calls follow the paper's statement of the problem.  Inputs are the
 * transfer functions of the potentials phi and psi, the box, the mesh, the
 * step in log a, the redshift range, the neutrino masses and the particle
 * count (Sec. 2.1 and Sec. 4).  Outputs are particle positions, momenta and
 * delta-f weights (Sec. 2.2) and the weighted density estimate
 * (eq:empirical_rho).
 *
 * Conventions.
 *  - Units: Mpc for lengths and conformal time (c = 1); eV for momenta, masses
 *    and temperatures; k in 1/Mpc.
 *  - Every call returns FDF_OK (0) or a negative FDF_E* code; no exception or
 *    C++ type crosses this boundary.  fdf_error_string() names a code and
 *    fdf_last_error() returns the last detailed message of this thread.
 *  - The context owns the device memory it allocated.  A caller-provided
 *    arena stays owned by the caller and must outlive the context.
 *  - All device work is enqueued on the CUDA stream given to fdf_create (NULL
 *    = the legacy default stream).  Calls that return data to the host
 *    (fdf_get, fdf_get_initial, fdf_deposit, fdf_build_fields with host
 *    output) synchronise that stream before returning.
 *  - Arrays of 3-vectors are structure-of-arrays: v[c * n + i], c = 0, 1, 2.
 *    Grids are N^3 with cell index (iz * N + iy) * N + ix, node positions
 *    x = (ix, iy, iz) * L / N.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef FDF_H
#define FDF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FDF_API __attribute__((visibility("default")))
#else
#define FDF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------- */
#define FDF_OK        0
#define FDF_EINVAL   (-1)  /* invalid argument or parameter set */
#define FDF_ENOMEM   (-2)  /* device allocation failed, or the arena is too small */
#define FDF_ECUDA    (-3)  /* a CUDA runtime call or kernel launch failed */
#define FDF_ESTATE   (-4)  /* call out of order (e.g. fdf_step before fdf_sample) */
#define FDF_ETIMEOUT (-5)  /* a bounded device-side wait gave up */
#define FDF_ENAN     (-6)  /* a non-finite value was produced */
#define FDF_ENOSYS   (-7)  /* configuration not supported by this build */

/* ---- precision forms (fdf_params.precision) ------------------------------ */
/* FDF_PREC_F64: the plain form.  Grids, FFTs, positions, momenta and all
 *   arithmetic in FP64 (positions as FP64 Mpc, wrapped with floor).
 * FDF_PREC_F32: FP32 grid build, FFT and gradient storage with FP32
 *   interpolation, and an FP64 phase-space state: positions (Mpc) and momenta
 *   (eV) are stored and accumulated in FP64, and the step integrals are
 *   evaluated in FP64 -- the drift's int dtau / eps and the kick's
 *   int eps_0 dtau and int dtau / eps_0 (eq:discrete_drift, eq:releq_approx).
 *   Each integral is r_c sum_k C_k t^k, a series about the interval's centre in
 *   t = m^2 a_c^2 r_c^2 with r_c = (|q|^2 + m^2 a_c^2)^(-1/2) and FP64
 *   coefficients from the host; r_c, t and the leading terms (five for the
 *   drift, one for a kick, whose integrals only scale a kick of ~1e-3 of |q|) are
 *   FP64, and the terms beyond them (below 1e-7 of the drift integral, 3e-3 of
 *   a kick's, at the workloads' step sizes) are FP32.  The kick
 *   itself (a change of at most ~1e-3 of |q| per step) is formed in FP32 from
 *   the FP32 gradients and q_0 (stored in FP32) and added to q in FP64.
 * FDF_PREC_BF16: FDF_PREC_F32 with BF16 gradient-grid storage (FP32
 *   interpolation, the same FP64 state and integrals).
 * FDF_PREC_F32_FIXED: the split-state form.  FP32 grids as FDF_PREC_F32;
 *   positions as 32-bit fixed-point fractions of the box (resolution L / 2^32,
 *   periodic wrap exact by integer overflow); momenta as q = q_0 + dq with q_0
 *   and dq in FP32 (|dq| << |q|); the drift integral in float-float (about
 *   44-bit mantissa) on the FP32 pipe; kick integrals in FP32.  No FP64
 *   instruction runs in its particle pass.
 * FDF_PREC_BF16_FIXED: the split-state form with BF16 gradient-grid storage. */
#define FDF_PREC_F64        0
#define FDF_PREC_F32        1
#define FDF_PREC_BF16       2
#define FDF_PREC_F32_FIXED  3
#define FDF_PREC_BF16_FIXED 4

/* ---- flags (fdf_params.flags) -------------------------------------------- */
#define FDF_FLAG_FIXED_AMPLITUDE 1  /* |R_k| = sqrt(P(k)/V), random phase ("fixed" ICs, Sec. 4) */
/* The dipole term of eq:transform times 3, the factor 2l+1 of the paper's Legendre
 * convention (eq:def2) that eq:pre_int and eq:transform do not print.  As printed
 * (the default) the transform's delta-f energy flux is (rho + P) theta / 3 with
 * theta = k^2 tau psi / 2; with this flag it is (rho + P) theta. */
#define FDF_FLAG_LEGENDRE_DIPOLE 2

/* ---- deposit quantities (fdf_deposit) ------------------------------------ */
#define FDF_Q_W_EPS 0  /* w_k eps_k: the delta-f energy density of eq:empirical_rho */
#define FDF_Q_W     1  /* w_k */
#define FDF_Q_EPS   2  /* eps_k (no delta-f weight) */
#define FDF_Q_COUNT 3  /* 1 */
#define FDF_Q_W_QX  4  /* w_k q_k,x: the delta-f momentum density, whose divergence */
#define FDF_Q_W_QY  5  /*   gives the (1 + delta) theta spectrum of Sec. 4 */
#define FDF_Q_W_QZ  6

/* ---- timed kernel classes (fdf_kernel_time) ------------------------------ */
#define FDF_K_PUSH     0  /* fused drift + wrap + gather + kick */
#define FDF_K_FIELDS_Z 1  /* spectrum generation + inverse DFT along z */
#define FDF_K_FIELDS_Y 2  /* inverse DFT along y */
#define FDF_K_FIELDS_X 3  /* inverse DFT along x + interleave into the gather grid */
#define FDF_K_OTHER    4  /* sampling, initial transform, weights, deposit, export */
#define FDF_K_SORT     5  /* re-bucketing of particles by position */
#define FDF_K_COUNT    6

typedef struct fdf_ctx fdf_ctx;

/* Run parameters (Sec. 4 lists the paper's: 800^3 particles, L = 3.2 Gpc,
 * M = 800, d log a = 0.01, z = 1e9 to 0).  Species share the potential grids
 * and the time grid; they differ in mass.  The background is a flat
 * radiation + matter + Lambda model, H = H0 sqrt(omega_r a^-4 + omega_m a^-3 +
 * 1 - omega_m - omega_r), H0 = h / 2997.92458 Mpc^-1. */
typedef struct fdf_params {
    double   box_mpc;          /* L > 0 */
    int64_t  n_part;           /* particles per species, >= 0 */
    int32_t  n_grid;           /* N, power of two in [8, 512] */
    int32_t  n_species;        /* 1..4 */
    double   m_ev[4];          /* neutrino mass per species, >= 0 */
    double   T_nu_K;           /* present-day neutrino temperature (1.95 K in Sec. 2) */
    double   z_start, z_end;   /* z_start > z_end > -1 (paper: 1e9 and the N-body start) */
    int32_t  n_steps;          /* >= 1, constant step in log a (Sec. 3.3) */
    int32_t  precision;        /* FDF_PREC_* */
    uint64_t seed;             /* Philox key of the sampler and of the Gaussian field */
    double   h, omega_m, omega_r;
    double   A_s, n_s, k_pivot; /* primordial curvature spectrum, k_pivot in 1/Mpc */
    int32_t  flags;            /* FDF_FLAG_* */
    int32_t  n_gl;             /* Gauss-Legendre nodes per step integral, 2..8; 0 = the
                                  smallest count whose error bound is below 1e-13 for
                                  this step size (4 at d ln a = 0.17) */
    int32_t  sort_every;       /* re-bucket particles by position (gather locality): 0 = after
                                  sampling and whenever the typical displacement since the last
                                  sort exceeds sort_cells cells; k > 0 = every k steps; -1 = never
                                  (always after sampling unless -1) */
    int32_t  steps_per_pass;   /* leapfrog steps per particle pass, 1..8: the particle state is
                                  read and written once per pass, and 2 steps_per_pass + 1 grids
                                  are held (0 = 4 for the FP32/BF16-grid forms, 1 for the plain
                                  FP64 form) */
    int32_t  sort_tile;        /* sort buckets are cubes of 2^sort_tile cells per axis, 0..3
                                  (0 = single cells) */
    int32_t  sort_cells;       /* with sort_every = 0: re-bucket when the typical particle has
                                  moved this many cells since the last sort (0 = 4) */
    int32_t  interp_order;     /* interpolation order r of the force read and the deposit
                                  (Sec. 4): 1 (or 0) cloud-in-cell, 2 triangular-shaped cloud */
    double   superstep_tol;    /* super-steps (Sec. 2.1): > 0 builds the fields by transform only
                                  at steps where the transfer functions of phi and psi changed
                                  by more than this fraction (the paper uses 0.01) since the last
                                  built step, and interpolates them linearly in ln a in between;
                                  0 builds every step.  The change between steps j0 and j1 is,
                                  for T = T_psi and T_phi, max |T(k, a_j1) - T(k, a_j0)| over 64
                                  ln k points from 2 pi/L to sqrt(3) pi N/L, relative to
                                  max |T(k, a_j0)| there; the larger of the two. */
    int32_t  eom;              /* the kick's equation of motion, each with the momentum frozen at
                                  its z = 1e9 value so that the leapfrog stays symplectic:
                                  FDF_EOM_GEODESIC (0, eq:releq_approx, the method's), or, in the
                                  plain FP64 form only (FDF_ENOSYS otherwise), the comparison
                                  forms FDF_EOM_CANONICAL (eq:releq_lag), FDF_EOM_SR_NEWTON
                                  (eq:p_eq), FDF_EOM_Q_SIMPLE (eq:q_eq), FDF_EOM_NEWTONIAN, and
                                  FDF_EOM_EXACT (eq:releq and eq:geodesic themselves, not
                                  symplectic; steps_per_pass 0, 1 or 2) */
    int32_t  pass_blocks;      /* the FP32/BF16-grid forms with the FP64 state: the launch shape
                                  of the particle pass, a persistent grid of this many blocks
                                  of 256 threads per SM: 2 = two particles per thread (128
                                  registers), 1 or 3 = one particle per thread (80 registers);
                                  0 = automatic (2: measured fastest on the 3 x 256^3
                                  workload, 714 ms per run against 736 ms with 3).  The
                                  results are the same bit for bit.  Ignored by the other
                                  forms. */
    int32_t  gather_tile;      /* the split-state forms: 1 = each block's kicks read the grid from a
                                  shared-memory tile of the cells its particles occupy (loaded once
                                  per kick; order-1 reads only), -1 = every read from the grid in
                                  device memory, 0 = automatic (-1: the tile measured slower on
                                  the 3 x 256^3 workload).  Ignored by the other forms. */
    int32_t  deposit_presum;   /* the weighted deposit (eq:empirical_rho): 1 = the lanes of a warp
                                  whose particles share a base cell first add their
                                  contributions to each node by warp shuffles, and one lane
                                  per such set issues the atomic additions; -1 = one atomic
                                  addition per particle and node; 0 = automatic (-1: the
                                  pre-sum measured slower on the 3 x 256^3 workload, 5.7 ms
                                  against 4.7 ms).  Either way the sums are FP64 in an
                                  unspecified order. */
} fdf_params;

/* ---- equations of motion (fdf_params.eom) -------------------------------- */
#define FDF_EOM_GEODESIC  0  /* dq/dtau = -eps0 grad psi - (q0^2/eps0) grad phi + q0 (q0.grad phi)/eps0 + q0 phi_dot */
#define FDF_EOM_CANONICAL 1  /* dP/dtau = -eps0 grad psi - (P0^2/eps0) grad phi (Sec. 3.2) */
#define FDF_EOM_SR_NEWTON 2  /* dP/dtau = -((2 P0^2 + m^2 a^2)/eps0) grad psi (Sec. 5) */
#define FDF_EOM_Q_SIMPLE  3  /* dq/dtau = -eps0 grad psi (Sec. 5) */
#define FDF_EOM_NEWTONIAN 4  /* dq/dtau = -m a grad psi (Sec. 5: dq/dt = -m grad psi, dtau = dt/a) */
/* The exact eq:releq, dq/dtau = -eps grad psi - (q^2/eps) grad phi + q (q.grad phi)/eps
 * + q phi_dot, and eq:geodesic, dx/dtau = (q/eps)(1 + phi + psi), in the non-symplectic
 * leapfrog Sec. 3.3 uses as a check: each half kick holds q (and eps) at its start;
 * the drift takes 1 + phi + psi at its starting point from the fields of that step.
 * The steps' grids then carry phi + psi in slot 7 (psi otherwise); the initial
 * transform and fdf_build_fields still see psi there.  Frozen fields
 * (fdf_set_fields) are used as given: slot 7 is read as phi + psi by the drift. */
#define FDF_EOM_EXACT     5

/* Input tables, host memory, copied by fdf_create.
 *  T_psi, T_phi, dTphi_dlna: [na][nk] row-major, the transfer functions of
 *  psi and phi relative to the primordial curvature R, and d T_phi / d ln a,
 *  on uniform ascending grids lnk[nk] (ln(k Mpc)) and lna[na]; read with
 *  bilinear interpolation in (ln k, ln a), clamped at the edges (Sec. 2.1:
 *  CLASS supplies these in the paper).
 *  cdf_t[ncdf], cdf_F[ncdf]: the normalised CDF F(t) of t^2 / (1 + e^t),
 *  t = q/T, ascending, F[0] = 0; momenta are drawn by piecewise-linear
 *  inversion (Sec. 2.1, Fermi-Dirac fbar). */
typedef struct fdf_tables {
    int32_t nk, na;
    const double *lnk, *lna;
    const double *T_psi, *T_phi, *dTphi_dlna;
    int32_t ncdf;
    const double *cdf_t, *cdf_F;
} fdf_tables;

/* Device bytes fdf_create would need for these parameters (admission
 * control).  Returns FDF_EINVAL for an invalid parameter set. */
FDF_API int fdf_footprint(const fdf_params* p, size_t* bytes);

/* Validate p and t, copy the tables to the device, allocate (or carve from
 * arena, a device pointer with arena_bytes >= fdf_footprint) every buffer,
 * and precompute the background.  stream is a cudaStream_t (may be NULL).
 * On success *out holds a new context; on failure *out is NULL. */
FDF_API int fdf_create(const fdf_params* p, const fdf_tables* t, void* stream, void* arena, size_t arena_bytes,
               fdf_ctx** out);

/* Pre-initial conditions at z_start (Sec. 2.1): draw every particle of every
 * species (uniform position, Fermi-Dirac |q|, isotropic direction, from
 * Philox4x32-10 keyed by seed and addressed by the global particle index),
 * build the fields at a_0 and apply the momentum transform eq:transform with
 * delta = -2 psi and theta = k^2 tau psi / 2; set q_0 = q and p = |q_sampled|.
 * Leaves the state at step 0. */
FDF_API int fdf_sample(fdf_ctx* c);

/* Advance n steps of the kick-drift-kick leapfrog of Sec. 3.3
 * (eq:releq_approx, eq:geodesic_approx, eq:discrete_drift) with constant
 * d log a; n < 0 steps backward.  Each step builds the potential-gradient
 * grids at the new scale factor (spectrum times transfer functions times i k,
 * inverse FFT) and makes one fused particle pass (drift, periodic wrap,
 * trilinear gather, kick).  Positions and momenta are synchronised when the
 * call returns.  FDF_EINVAL if the step index would leave [0, n_steps];
 * FDF_ESTATE before fdf_sample. */
FDF_API int fdf_step(fdf_ctx* c, int32_t n);

/* fdf_sample(c) followed by fdf_step(c, n), 0 <= n <= n_steps, replayed as one
 * CUDA graph.  The paper has no counterpart: this is the launch form of a run
 * (Sec. 2.1's particles are independent once the metric is known, so a run's
 * launches and their order are fixed by fdf_params and n alone).  The first call
 * for a given n records every launch of the run (field builds on the context's
 * second stream, particle passes, sorts) into a graph held by the context; each
 * later call with the same n replays it with one launch, without re-issuing the
 * kernels from the host, and leaves the context in the state the sequential
 * calls would (step n, the same buffers; the results are bitwise the same).
 * A call with another n records anew.  Queued on the context's stream (a context
 * on the legacy default stream, which cannot be recorded, runs its graph on a
 * private blocking stream that the legacy stream orders); returns
 * after the run, like fdf_sample, so that the sampler's failure is reported
 * (FDF_EINVAL).  FDF_ESTATE while fdf_timing is on (per-kernel events are not
 * recorded inside a graph) or with fdf_set_fields in force. */
FDF_API int fdf_run_graph(fdf_ctx* c, int32_t n);

/* The four terms of the exact acceleration eq:releq at the current step, as
 * Fig. 2 of the paper plots them: with the potentials of the current scale factor
 * a read at each particle's position (the kernel of order interp_order) and its
 * momentum q, eps = sqrt(q^2 + m^2 a^2),
 *   T1 = -eps grad psi,  T2 = -(q^2/eps) grad phi,  T3 = q (q.grad phi)/eps,
 *   T4 = q phi_dot;
 * rms[i] = sqrt(mean over the particles of |T_{i+1}|^2), i = 0..3, and rms[4] the
 * same for T1 + T2 + T3 + T4.  species: 0..n_species-1, or -1 for all.  rms: 5
 * host doubles.  Sums in FP64 on the device; synchronises the stream.  FDF_ESTATE
 * before fdf_sample; all zero for an empty species. */
FDF_API int fdf_accel_terms(fdf_ctx* c, int32_t species, double* rms);

/* Weighted CIC density estimate of eq:empirical_rho at the current scale
 * factor: out[n] = sum_k v_k W(x_n - x_k) over the grid nodes n, with v_k
 * chosen by quantity (FDF_Q_*), over one species (0..n_species-1) or all (-1);
 * W is the kernel of order interp_order.
 * w_k = 1 - fbar(|q_k|)/fbar(p_k) (Sec. 2.2).  The raw sum is returned; the
 * M/N normalisation is the caller's.  out is N^3 doubles, device memory if
 * out_on_device else host memory. */
FDF_API int fdf_deposit(fdf_ctx* c, int32_t species, int32_t quantity, double* out, int32_t out_on_device);

/* fdf_deposit over one half of the ensemble: parity 0 deposits the particles
 * with even ids, 1 those with odd ids, -1 all.  The cross-spectrum of the two
 * halves removes the shot-noise plateau (Sec. 4 computes power spectra so). */
FDF_API int fdf_deposit_subset(fdf_ctx* c, int32_t species, int32_t quantity, int32_t parity, double* out,
                               int32_t out_on_device);

/* Current state of one species in particle-index order: x[3][n_part] (Mpc,
 * in [0, L)), q[3][n_part] (eV), w[n_part] (delta-f weight, Sec. 2.2:
 * w = -expm1((p - |q|)/T) / (1 + exp(-|q|/T)); the FP32/BF16-grid forms take
 * p - |q| in FP64 and the rest in FP32, as their deposit does).  Any output pointer may be
 * NULL.  Device or host memory per out_on_device; synchronises the stream.  Host buffers
 * that are page-locked and mapped (cudaHostAlloc, cudaHostRegister) are written by the
 * device directly; other host memory through a device staging buffer and copies. */
FDF_API int fdf_get(fdf_ctx* c, int32_t species, double* x, double* q, double* w, int32_t out_on_device);

/* The pre-initial draw of one species before the momentum transform:
 * X[3][n_part] (x = L * X / 2^32), q_sampled[3][n_part] (eV) and
 * p[n_part] = |q_sampled|.  Exact: every operation is a correctly rounded IEEE
 * operation.  Any pointer may be NULL. */
FDF_API int fdf_get_initial(fdf_ctx* c, int32_t species, uint32_t* X, double* q_sampled, double* p, int32_t out_on_device);

/* Test and inspection hook: the eight real fields at ln a, as built on the
 * device, converted to FP64: out[8][N^3] in the slot order (d_x psi, d_y psi,
 * d_z psi, d_x phi, d_y phi, d_z phi, phi_dot, psi), phi_dot = a H d phi / d ln a.
 * Field convention f(x) = sum_n f_n e^{i k.x}.  Slots 0-6 come from a build as the
 * steps' particle passes read it (phi_dot, packed with slot 7 in one complex
 * transform, is transformed alone there); slot 7 (psi, which the initial transform
 * reads) from a second build. */
FDF_API int fdf_build_fields(fdf_ctx* c, double lna, double* out, int32_t out_on_device);

/* fdf_build_fields without a context and without allocating: for callers that
 * must not allocate device memory, such as a simulation code embedding this
 * library whose own allocator owns the device budget, or a serving loop that
 * forbids cudaMalloc/cudaFree after start-up because those calls synchronise
 * the device and fragment its memory.  The paper has no counterpart; this is
 * an interface convenience.
 *  p, t: as for fdf_create (host memory; cdf_t and cdf_F are not used).  lna:
 *  ln a of the fields.  out: DEVICE memory of 8 N^3 doubles on the current
 *  device, written as by fdf_build_fields.  stream: a cudaStream_t or NULL.
 *  Every call copies t's transfer tables and the FFT twiddles from host memory
 *  into the array, and synchronises stream before returning.
 *  Work arrays live in one static device array of FDF_NOALLOC_SCRATCH_BYTES
 *  that every GPU loading the library holds until the process exits; the call
 *  performs no cudaMalloc or cudaFree.  FDF_EINVAL, with a message naming both
 *  sizes, when the grid needs more scratch than that (n_grid <= 64 in FP32,
 *  <= 32 in FP64).  The first call on each device looks up the array's device
 *  address with that device current; make that first call before any stream
 *  capture.  All calls share the one array and overwrite it: calls that
 *  overlap on the GPU (other host threads, other streams) race. */
#define FDF_NOALLOC_SCRATCH_BYTES (20u << 20)
FDF_API int fdf_build_fields_noalloc(const fdf_params* p, const fdf_tables* t, double lna, double* out,
                                     void* stream);

/* Test hook: freeze the fields.  fields[8][N^3] (same layout as
 * fdf_build_fields) replace the per-step grid build for every later call;
 * fields = NULL returns to building them. */
FDF_API int fdf_set_fields(fdf_ctx* c, const double* fields, int32_t on_device);

/* The super-step schedule: is_super[j] = 1 where the fields of step j are built
 * by transform (every step when superstep_tol = 0), for j = 0..min(len, n_steps+1)-1;
 * *count = the number of such steps.  Either pointer may be NULL. */
FDF_API int fdf_supersteps(fdf_ctx* c, int32_t* is_super, int32_t len, int32_t* count);

/* Which particle-pass kernel the last fdf_step (or the run of fdf_run_graph) used:
 * info[0] the state form (0 plain FP64, 1 FP64 state with FP32/BF16 grids, 2 split
 * state), info[1] 1 if every pass evaluated its step integrals as series or fitted
 * polynomials (FDF_PREC_F32/BF16: the polynomials of include/fdf.h's precision notes;
 * split state: the drift's power series) and 0 if any pass summed them node by node,
 * info[2] the number of passes, info[3] the most leapfrog steps in one pass.  info:
 * 4 host int32.  The paper has no counterpart (an inspection hook for tests). */
FDF_API int fdf_pass_info(fdf_ctx* c, int32_t* info);

/* Current step index (0..n_steps) and its ln a. */
FDF_API int fdf_state(fdf_ctx* c, int32_t* step, double* lna);

/* Kernel timing with CUDA events recorded on the context's stream around
 * each launch of the classes FDF_K_*.  fdf_timing(c, 1) clears and starts,
 * fdf_timing(c, 0) stops; fdf_kernel_time synchronises and returns the summed
 * milliseconds and the launch count of one class. */
FDF_API int fdf_timing(fdf_ctx* c, int32_t enable);
FDF_API int fdf_kernel_time(fdf_ctx* c, int32_t which, double* ms, int64_t* launches);

/* Issue rates of the arithmetic pipes the particle pass uses, measured on the
 * current device (the denominators of the passes' FP64-pipe roofline): dependent
 * FP64 fused multiply-adds per second (*dfma_per_s; 2 flops each), FP32 fused
 * multiply-adds per second (*ffma_per_s), and FP64 -> FP32 -> FP64 conversion
 * round trips per second (*cvt_per_s, two conversions each).  Each is the best of
 * five timed launches (CUDA events on stream, a cudaStream_t or NULL) of every SM
 * holding 64 warps with 8 independent chains per thread.  The paper has no
 * counterpart.  Any pointer may be NULL; changes no device setting. */
FDF_API int fdf_pipe_rates(void* stream, double* dfma_per_s, double* ffma_per_s, double* cvt_per_s);

/* Number of kernels this context has launched since creation. */
FDF_API int64_t fdf_launch_count(const fdf_ctx* c);

FDF_API const char* fdf_error_string(int code);
FDF_API const char* fdf_last_error(void);

/* Free everything the context allocated.  NULL is allowed. */
FDF_API void fdf_destroy(fdf_ctx* c);

/* Autotuner of the schedule knobs that change speed only (no result beyond the
 * stated tolerances): sort_cells, sort_tile, steps_per_pass and (FP64-state forms)
 * pass_blocks.  It times whole runs (fdf_sample + fdf_step(n_steps)) of p on the
 * device, one knob at a time (coordinate descent over sort_cells in {2, 4, 8, 16, 32, 64},
 * sort_tile in {0, 1, 2, 3}, steps_per_pass in {2, 3, 4, 6, 8}, pass_blocks in {2, 3} (FP64-state
 * forms) or gather_tile in {-1, 1} (split-state forms), then sort_cells again in
 * {3, 5, 6, 12, 24, 48}), starting from the automatic choices, and writes
 * the fastest parameter set to *out (p with the knobs set).  The paper
 * has no counterpart.  stream: a cudaStream_t or NULL; every trial allocates
 * and frees its own context.  ms (may be NULL) receives the best run time;
 * trials (may be NULL) the number of timed runs.  Only the FP32/BF16-grid forms are tuned;
 * for FDF_PREC_F64 *out = *p. */
FDF_API int fdf_tune(const fdf_params* p, const fdf_tables* t, void* stream, fdf_params* out, double* ms,
                     int32_t* trials);

/* ---- request server (continuous batching) --------------------------------
 * Runs many independent runs ("requests": one fdf_params + fdf_tables each,
 * of any grid size, particle count, species count, masses and step count) on
 * one GPU at once.  The paper has no counterpart: each of its runs is one job
 * (Sec. 2.1 notes that every neutrino is independent once the metric is known,
 * so independent runs can share a GPU without interacting).
 *
 * The server allocates one device arena of hbm_budget bytes at creation and
 * never calls cudaMalloc or cudaFree afterwards.  A worker thread:
 *  - admits queued requests first-come-first-served while a slot is free
 *    (at most max_active running) and the arena has a free range of the
 *    request's fdf_footprint; a request that would never fit is refused at
 *    submission (FDF_ENOMEM);
 *  - runs every admitted request on its own CUDA streams (fdf_create on the
 *    arena range, fdf_sample, then fdf_step in slices of slice_steps steps,
 *    at most two slices in flight per request), so the kernels of different
 *    requests overlap on the device;
 *  - after the last step, deposits the weighted density of all species
 *    (FDF_Q_W_EPS) on the device and marks the request done.
 * A done request keeps its state (particles, deposit) resident until
 * fdf_server_release returns its arena range; only then can a waiting request
 * use that memory.  Each request's results do not depend on what else runs:
 * positions, momenta and weights are bitwise those of the same request run
 * alone; the deposit differs by the order of its FP64 atomic additions only.
 *
 * Times are seconds on the server's steady clock (fdf_server_clock).
 * t_done is taken on the GPU timeline (a host function enqueued after the
 * deposit), so a request's latency is t_done - t_submit. */
typedef struct fdf_server fdf_server;

#define FDF_REQ_QUEUED  0
#define FDF_REQ_RUNNING 1
#define FDF_REQ_DONE    2
#define FDF_REQ_FAILED  3

typedef struct fdf_request_info {
    int64_t id;
    int32_t status;            /* FDF_REQ_* */
    int32_t error;             /* FDF_E* code when FAILED, else 0 */
    double  t_submit, t_admit, t_done;
    size_t  footprint;         /* device bytes held while admitted */
    int64_t particle_steps;    /* n_species * n_part * n_steps */
    char    message[160];      /* error detail when FAILED */
} fdf_request_info;

/* hbm_budget: bytes of the device arena (allocated on the current device);
 * max_active: running requests at most (>= 1); slice_steps: steps per
 * fdf_step call of the worker (>= 1).  FDF_ENOMEM if the arena cannot be
 * allocated. */
FDF_API int fdf_server_create(size_t hbm_budget, int32_t max_active, int32_t slice_steps, fdf_server** out);

/* fdf_server_create with options: FDF_SERVER_MERGE_PASSES steps the running requests
 * of the FP32/BF16-grid forms with the FP64 state (per grid precision, at most 16 at a
 * time) in merged launches, one kernel issuing the next pass of every such request
 * (the other forms keep their own launches).  Each request's particles run the same
 * arithmetic alone and in a merge, so its results are bitwise the same either way
 * within this mode; against the default mode they differ by rounding only. */
#define FDF_SERVER_MERGE_PASSES 1
FDF_API int fdf_server_create_opts(size_t hbm_budget, int32_t max_active, int32_t slice_steps, int32_t options,
                                   fdf_server** out);

/* The number of merged launches the server made so far (0 without FDF_SERVER_MERGE_PASSES). */
FDF_API int fdf_server_merged_launches(const fdf_server* s, int64_t* launches);

/* Queue a run.  p and t are copied (host memory; the caller may free them on
 * return).  *id receives the request's id.  FDF_EINVAL for invalid
 * parameters; FDF_ENOMEM if fdf_footprint exceeds the whole budget. */
FDF_API int fdf_server_submit(fdf_server* s, const fdf_params* p, const fdf_tables* t, int64_t* id);

/* Wait up to timeout_ms (< 0: forever) for the next request to finish (done or
 * failed) and return its id; each finished request is reported once.
 * FDF_ETIMEOUT if none finished in time. */
FDF_API int fdf_server_wait(fdf_server* s, int32_t timeout_ms, int64_t* id);

/* Status and timestamps of a request that has not been released. */
FDF_API int fdf_server_info(fdf_server* s, int64_t id, fdf_request_info* info);

/* Results of a done request: as fdf_get for one species, and the all-species
 * FDF_Q_W_EPS deposit at z_end (N^3 doubles).  Host or device memory per
 * on_device; both synchronise the request's stream only.  FDF_ESTATE if the
 * request is not done. */
FDF_API int fdf_server_get(fdf_server* s, int64_t id, int32_t species, double* x, double* q, double* w,
                           int32_t on_device);
FDF_API int fdf_server_deposit(fdf_server* s, int64_t id, double* out, int32_t on_device);

/* Drop a finished request and return its memory to the arena.  FDF_ESTATE
 * if it is still queued or running. */
FDF_API int fdf_server_release(fdf_server* s, int64_t id);

/* Seconds since fdf_server_create on the server's steady clock. */
FDF_API double fdf_server_clock(const fdf_server* s);

/* Queued and running request counts and arena bytes in use. */
FDF_API int fdf_server_load(fdf_server* s, int32_t* queued, int32_t* running, size_t* bytes_in_use);

/* Stop the worker, wait for the work already enqueued for running requests,
 * drop every request (queued, running or finished) and free the arena.  NULL
 * is allowed. */
FDF_API void fdf_server_destroy(fdf_server* s);

#ifdef __cplusplus
}
#endif
#endif /* FDF_H */
