// fdf_internal.cuh -- shared declarations of libfdf.so (device kernels and the
// host context).  Nothing here is part of the C-ABI; include/fdf.h is.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/fdf.h"

namespace fdf {

// The three state forms of the precision settings (FDF_PREC_*): the plain FP64 form,
// the FP64-state form with FP32 or BF16 grids, and the split-state form with
// fixed-point positions.
enum Form { kPlain = 0, kWide = 1, kFixed = 2 };
__host__ __device__ constexpr int form_of(int prec)
{
    return prec == FDF_PREC_F64 ? kPlain : (prec == FDF_PREC_F32 || prec == FDF_PREC_BF16) ? kWide : kFixed;
}
// The grid storage of a precision setting: FDF_PREC_F64, FDF_PREC_F32 or FDF_PREC_BF16.
__host__ __device__ constexpr int grid_prec(int prec)
{
    return prec == FDF_PREC_F32_FIXED ? FDF_PREC_F32 : prec == FDF_PREC_BF16_FIXED ? FDF_PREC_BF16 : prec;
}

constexpr int kMaxGL = 8;       // Gauss-Legendre nodes per step integral
constexpr int kMaxSpecies = 4;
constexpr int kSlots = 8;       // d psi (3), d phi (3), phi_dot, psi

struct FF {                     // float-float: value = hi + lo, |lo| <= ulp(hi)/2
    float hi, lo;
};

// Coefficients of one particle pass for one species.  Every integral is a sum
// over Gauss-Legendre nodes a_j of the pass's interval in ln a:
//   int g(a) dtau = sum_j W_j g(a_j),  W_j = w_j (dlna/2) / (a_j H(a_j)).
constexpr int kTaylor = 12;     // terms of the drift correction series

struct SpeciesCoef {
    // drift over [ln a_k, ln a_k+1]: D(q) = sum_j Wd_j / sqrt(q^2 + mud_j)
    double Wd[kMaxGL];
    double mud[kMaxGL];
    FF Wd_sum;                  // sum_j Wd_j, times 2^32/L (position quanta)
    FF mud_c;                   // mud at the centre node jc
    float Wd_f[kMaxGL];         // Wd_j times 2^32/L
    float dmud_f[kMaxGL];       // mud_j - mud_c
    // the same correction as a series: sum_j Wd_j g(delta_j) = sum_k Cd_k t^k with
    // t = mud_c / (q^2 + mud_c) (see k_push_split)
    float Cd[kTaylor];          // c_k sum_j Wd_j e_j^k, e_j = (mud_j - mud_c) / mud_c, times 2^32/L
    float mud_c_f;
    // kick over [lo, hi]: K_psi = sum Wk sqrt(q0^2 + muk), K_phi = sum Wk / sqrt(..)
    double Wk[kMaxGL];
    double muk[kMaxGL];
    double dtau_k;
    double Ka;                  // m sum_j Wk_j a_j (the Newtonian kick's integral)
    float Wk_f[kMaxGL];
    float muk_f[kMaxGL];
    float dtau_k_f;
};

// The FP64-state form's step integrals as polynomials.  Over an interval with
// Gauss-Legendre nodes a_j and weights W_j, centre a_c (the midpoint in ln a) and
// e_j = a_j^2 / a_c^2 - 1,
//   sum_j W_j (s + m^2 a_j^2)^(-1/2) = r gm(t),   sum_j W_j (s + m^2 a_j^2)^(1/2) = (u r) gp(t),
// with u = s + m^2 a_c^2, r = u^(-1/2), t = m^2 a_c^2 / u in [0, 1] and
// gm(t) = sum_j W_j (1 + e_j t)^(-1/2), gp(t) = sum_j W_j (1 + e_j t)^(1/2).  gm and gp
// depend on the interval only (not on the mass); the host fits each by a polynomial
// in t (Chebyshev interpolation on [0, 1], turned into monomial coefficients) and
// checks it against the sum.  The device takes the first kWideD64 (drift) or
// kWideK64 (kick) coefficients in FP64 and the rest in FP32.
constexpr int kWideDeg = 10;    // highest degree of a fitted polynomial
constexpr int kWideD64 = 5;     // drift terms evaluated in FP64
constexpr int kWideK64 = 1;     // kick terms evaluated in FP64 (the kick needs ~1e-9)

struct WidePoly {
    double c64[kWideD64];       // coefficients 0..kWideD64-1 (FP64)
    float c32[kWideDeg + 1];    // coefficients kWideD64.. (kick: kWideK64..), FP32, zero-padded
};

struct WideCoef {
    // The drift in the variable v = 1 + |q|^2 / (m^2 a_c^2) (per species, m > 0): then
    // t = 1/v = r_v^2 with r_v = v^(-1/2), and D = r gm(t) = r_v gm(t) / (m a_c), the
    // factor 1/(m a_c) folded into the species' copy of the polynomial.  A massless
    // species (inv_muc = 0) takes D = |q|^-1 sum_j W_j.
    double inv_muc[kMaxSpecies];    // 1 / (m^2 a_c^2) of the drift interval, or 0 for m = 0
    int massless[kMaxSpecies];      // m = 0 (tested as an integer: an FP64 comparison costs an FP64 slot)
    double wsum[kMaxSpecies];       // sum_j W_j (the massless drift)
    WidePoly drift[kMaxSpecies];    // gm of the drift interval / (m a_c), per species
    double muk[kMaxSpecies];    // m^2 a_c^2 of the kick interval, per species
    WidePoly kphi;              // gm of the kick interval: K_phi = r gm(t)
    WidePoly kpsi;              // gp of the kick interval: K_psi = u r gp(t)
    float dtau_k;               // conformal time of the kick interval
};

// One sub-step of a particle pass: an optional drift over [ln a_k, ln a_k+1] and an
// optional kick with the grid of the sub-step's end point.
struct SubStep {
    int do_drift;
    int do_kick;
    double emax;                // largest |e_j| of any species (the series converges for <= 1/4)
    int wide_ok;                // the FP64-state form's fits of this sub-step passed
    SpeciesCoef sp[kMaxSpecies];
    WideCoef wide;              // the FP64-state form
};

constexpr double kSeriesMaxE = 0.25;

constexpr int kMaxSub = 9;      // sub-steps per particle pass (an open kick and 8 steps)

struct PushArgs {
    int64_t n;                  // particles in all species
    int64_t n_part;             // particles per species
    int64_t sp_begin[kMaxSpecies];  // first particle of species 1, 2, 3 (n beyond the last species)
    int n_gl;                   // Gauss-Legendre nodes of the drift integral
    int n_kick;                 // nodes of the kick integrals
    int uniform_species;        // every species has the same mass: use sp[0]
    int drift_series;           // the drift corrections of this pass converge as a series
    int order;                  // interpolation order r: 1 cloud-in-cell, 2 TSC
    int eom;                    // FDF_EOM_* (the plain FP64 form)
    int grid_blocks;            // the FP64-state form: blocks of its persistent pass grid
    unsigned long long* ctr;    // the FP64-state form: two work counters, zero at launch
    int pair;                   // the FP64-state form: two particles per thread (two blocks per SM)
    int tile_gather;            // the split-state form: kicks gather from shared-memory tiles
    int wide_series;            // the FP64-state form: every fitted polynomial of this pass passed
                                // its check (else the integrals loop over the nodes)
    double m2[kMaxSpecies];     // m^2 per species (eV^2)
    int N;                      // grid side
    int nsub;                   // sub-steps in this pass, 1..kMaxSub
    double L, invL, invh;
    FF fx_scale;                // 2^32 / L
    SubStep sub[kMaxSub];
    const void* G[kMaxSub];     // the grid each sub-step's kick reads
};
// a kernel's parameters may take up to 32764 bytes
static_assert(sizeof(PushArgs) <= 32000, "PushArgs must fit the kernel parameter space");

// What slot 7 of a gather grid holds.  It shares its packed transform with phi_dot
// (phi_dot + i slot 7), and an FFT's rounding is relative to the larger of the two, so
// the steps' grids of the separable forms, whose passes never read slot 7, carry zero
// there and phi_dot is transformed alone.
constexpr int kSlot7Psi = 0;    // psi: the initial transform (eq:transform) reads it
constexpr int kSlot7Sum = 1;    // phi + psi: the drift factor of the exact equations of motion
constexpr int kSlot7Zero = 2;   // nothing

// Field-build arguments for one scale factor.
struct FieldArgs {
    int N, logN;
    int nk, na;
    double kf;                  // 2 pi / L
    double lnk0, inv_dlnk;      // uniform ln k grid
    int ia;                     // a-row of the tables below ln a (clamped)
    double fa;                  // fraction between rows ia and ia+1
    double aH;                  // a H(a) (multiplies dT_phi/dln a into phi_dot)
    double amp0;                // sqrt(2 pi^2 A_s / V)
    double half_nsm1;           // (n_s - 1) / 2
    double lnkp;                // ln k_pivot
    uint32_t key0, key1;        // Philox key (seed)
    int fixed_amp;
    int slot7;                  // slot 7: kSlot7Psi, kSlot7Sum (phi + psi) or kSlot7Zero
};

inline int ilog2_host(int v)
{
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

// ----- host helpers shared by the entry points (fdf_api.cu) ----------------
int set_error(int code, const char* msg);       // records the message fdf_last_error() returns
int validate_params(const fdf_params* p);       // FDF_OK or FDF_EINVAL with a message
bool uniform_grid(const double* v, int n, double* v0, double* dv);
// The FFT twiddles tw[j] = exp(2 pi i j / N), j < N, as (cos, sin) pairs in FP64 on the
// host; both field-build entry points upload this one table (FP32 copies for FP32 grids).
void twiddle_table(int N, double* cs);
FieldArgs make_field_args(const fdf_params& p, int nk, int na, double lnk0, double dlnk, double lnat0,
                          double dlnat, double lna);

// ----- kernel launchers (each returns cudaGetLastError()) -----------------

// Pre-initial sampling of particles [0, n): X, q_sampled, |q_sampled|, id.
cudaError_t launch_sample(cudaStream_t s, int64_t n, uint32_t key0, uint32_t key1, double T_ev, const double* cdf_t,
                          const double* cdf_F, int ncdf, uint32_t* X, double* qs, double* pmag, uint32_t* id,
                          int* flag);

// Field build: three passes.  precision: FDF_PREC_*.  W0/W1 are two complex
// work arrays of 4 N^3 elements (float2 or double2), G the gather grid.
// Per-step amplitude table A[4 M] (M = mode_table_size(N)) from the FP64
// tables [3][na][nk]; read by the z pass.
int mode_table_size(int N);
cudaError_t launch_mode_table(cudaStream_t s, int precision, const FieldArgs& a, const double* tabs64, void* A);
// The unit Gaussian field R_n / sqrt(P_R/V) on the N^3 mode array (drawn once per run).
cudaError_t launch_noise(cudaStream_t s, int precision, const FieldArgs& a, void* R);
cudaError_t launch_fields_z(cudaStream_t s, int precision, const FieldArgs& a, const void* A, const void* R,
                            const void* tw, void* W0);
cudaError_t launch_fields_y(cudaStream_t s, int precision, const FieldArgs& a, const void* tw, const void* W0,
                            void* W1);
cudaError_t launch_fields_x(cudaStream_t s, int precision, const FieldArgs& a, const void* tw, const void* W1,
                            void* G);
// G (any precision) <-> [8][N^3] FP64; to_f64 writes the slots whose bit is set in mask.
cudaError_t launch_fields_to_f64(cudaStream_t s, int precision, int N, const void* G, double* out,
                                 unsigned mask = 0xFFu);
// G = (1 - w) A + w B over whole gather grids (super-steps, Sec. 2.1)
cudaError_t launch_interp_grid(cudaStream_t s, int precision, int N, const void* A, const void* B, double w,
                               void* G);
cudaError_t launch_fields_from_f64(cudaStream_t s, int precision, int N, const double* in, void* G);

// Particle passes.
struct ParticleState {
    uint32_t* X;        // [3][n] fixed-point positions (split-state form; sampler output in all forms)
    float* q0f;         // [3][n] (split-state and FP64-state forms)
    float* dqf;         // [3][n] (split-state form)
    double* xd;         // [3][n] (plain and FP64-state forms)
    double* qd;         // [3][n] (plain and FP64-state forms)
    double* q0d;        // [3][n] (plain form)
    double* sd;         // [n] phi + psi from the last kick (the exact equations of motion), or NULL
    double* qs;         // [3][n] sampled momenta (one array for both halves: id order in the plain form;
                        // the FP32/BF16-grid forms carry it through their sort before the transform only)
    double* pmag;       // [n]
    uint32_t* id;       // [n]
};

cudaError_t launch_initial(cudaStream_t s, int precision, const ParticleState& st, int64_t n, int64_t n_part,
                           const double* m_ev, double a0, double tau0, int order, int N, double L, const void* G);
cudaError_t launch_push(cudaStream_t s, int precision, const ParticleState& st, const PushArgs& a);

// The passes of up to kMaxMerge contexts of the FP64-state form with one grid precision,
// in one launch: segment k covers global particle indices [begin, begin + args->n).
constexpr int kMaxMerge = 16;
struct MultiPass {
    struct Seg {
        int64_t begin;
        const PushArgs* args;   // device memory
        double* xd;
        double* qd;
        const float* q0f;
    };
    int nseg;
    int64_t total;
    Seg seg[kMaxMerge];
};
cudaError_t launch_push_multi(cudaStream_t s, int grid_precision, const MultiPass& m, int grid_blocks);

// Counting sort of the particle state a into b by (species, Morton index of
// the particle's tile of 2^tile_shift cells per axis, tile_shift = sort_tile).  key: n words; hist:
// n_species * tiles words; bsum: scan_scratch_words(bins) words; recs: n records
// of sort_record_bytes(precision).
// The FP32/BF16-grid forms bucket particles by where they will be halfway through the
// next pass: X + q dtau / sqrt(q^2 + m^2 a^2) (a free-streaming estimate), so that
// neighbours in memory stay neighbours in space for longer.
struct SortLead {
    int on;
    float dtau_q32[kMaxSpecies];  // conformal time of the lead, times 2^32 / L
    float m2a2[kMaxSpecies];      // m^2 a^2 at the middle of the lead
    // FP32/BF16-grid forms, before the momentum transform: the momenta do not exist yet; the keys
    // use the positions alone and the sampled momenta qs travel with the particles
    int pre_transform;
};
inline int sort_tile_shift(const fdf_params& p) { return p.sort_tile; }
size_t sort_record_bytes(int precision);
cudaError_t launch_sort(cudaStream_t s, int precision, const ParticleState& a, const ParticleState& b, int64_t n,
                        int64_t n_part, int n_species, int N, int tile_shift, double L, const SortLead& lead,
                        uint32_t* key, uint32_t* hist, uint32_t* bsum, void* recs);
// Particles [begin, begin + count) of an array of n; outputs in id order
// (out index = id - begin).
cudaError_t launch_export(cudaStream_t s, int precision, const ParticleState& st, int64_t n, int64_t begin,
                          int64_t count, double L, double T_ev, double* x, double* q, double* w);
cudaError_t launch_export_initial(cudaStream_t s, int precision, const ParticleState& st, int64_t n, int64_t begin,
                                  int64_t count, uint32_t* X, double* p, double* qs);
// launch_export's outputs for a permuted (sorted) state, through recs (the sort's
// record buffer, >= count records): one whole record per particle scattered to its
// id slot, then a streaming pass that writes x, q, w.
cudaError_t launch_export_records(cudaStream_t s, int precision, const ParticleState& st, int64_t n, int64_t begin,
                                  int64_t count, double L, double T_ev, void* recs, double* x, double* q, double* w);
// The four terms of eq:releq at particles [begin, begin + count) with the grid G:
// sums[0..3] += |T_i|^2, sums[4] += |T1 + T2 + T3 + T4|^2 (sums: 5 device doubles).
cudaError_t launch_accel_terms(cudaStream_t s, int precision, const ParticleState& st, int64_t n, int64_t begin,
                               int64_t count, int64_t n_part, const double* m_ev, double a, int order, int N,
                               double L, const void* G, double* sums);
// parity: -1 every particle, 0 or 1 the particles whose id has that parity (the
// two halves of the ensemble); order: the kernel order r (1 or 2).
cudaError_t launch_deposit(cudaStream_t s, int precision, const ParticleState& st, int64_t n, int64_t begin,
                           int64_t count, int64_t n_part, const double* m_ev, double a, double T_ev, int quantity,
                           int parity, int order, int N, double L, bool presum, double* grid);

// Asynchronous forms of two entry points, for the request server: the work is
// enqueued on the context's streams and nothing waits for it.
//   sample_enqueue: fdf_sample minus its final check; a failed direction draw
//     leaves a nonzero word at ctx_error_flag(c) (device memory).
//   deposit_enqueue: fdf_deposit into device memory out_dev (N^3 doubles).
int sample_enqueue(fdf_ctx* c);
int deposit_enqueue(fdf_ctx* c, int32_t species, int32_t quantity, int32_t parity, double* out_dev);
int* ctx_error_flag(fdf_ctx* c);
// fdf_step(c, n) pass by pass: slice_begin(c, n), then while slice_active(c):
// slice_next (the pass's arguments; c's stream then waits for the pass's grids), a
// launch of the pass on c's stream (or one that c's stream waits for), slice_done (the
// grids' release and a re-sort, on c's stream).
int slice_begin(fdf_ctx* c, int32_t n);
bool slice_active(const fdf_ctx* c);
int slice_next(fdf_ctx* c, PushArgs& a);
int slice_done(fdf_ctx* c);
const ParticleState& ctx_state(const fdf_ctx* c);
int ctx_precision(const fdf_ctx* c);
cudaStream_t ctx_stream(fdf_ctx* c);
double* ctx_deposit_grid(fdf_ctx* c);

}  // namespace fdf
