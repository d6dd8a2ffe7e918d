// fdf_api.cu -- host side of libfdf.so: the C-ABI of include/fdf.h.
//
// The context validates the run, owns one device block carved into every
// buffer, computes the background quantities and the per-pass quadrature
// coefficients on the host in FP64, and enqueues the kernels on the caller's
// stream in the order of the method (Elbers 2022):
//   fdf_sample: sampling (Sec. 2.1), fields at a_0, pre-initial transform
//               (eq:transform);
//   fdf_step:   per step, the fields at a_{k+1} and one fused particle pass
//               of the kick-drift-kick leapfrog of Sec. 3.3; consecutive half
//               kicks that read the same grid at the same position are merged
//               into one kick over [a_{k+1/2}, a_{k+3/2}].
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <climits>
#include <map>
#include <tuple>
#include <new>
#include <string>
#include <vector>

#include "fdf_internal.cuh"

using namespace fdf;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) { return fdf::set_error(code, msg.c_str()); }

constexpr double kC_over_H100 = 2997.92458;  // c / (100 km/s/Mpc) in Mpc
constexpr double kBoltzmann_eV = 8.617333262e-5;
constexpr double kPi = 3.14159265358979323846;
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(int v)
{
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

// storage of the grids by precision setting (the FP64-state and split-state forms
// share their grids' storage)
size_t grid_bytes_per_cell(int prec)
{
    const int g = grid_prec(prec);
    return g == FDF_PREC_F64 ? 64 : (g == FDF_PREC_F32 ? 32 : 16);
}
size_t complex_bytes(int prec) { return grid_prec(prec) == FDF_PREC_F64 ? 16 : 8; }
size_t real_bytes(int prec) { return grid_prec(prec) == FDF_PREC_F64 ? 8 : 4; }

// Gauss-Legendre rule on [-1, 1] by Newton's method on P_n, with
// P_n' = n (x P_n - P_{n-1}) / (x^2 - 1).
void gauss_legendre(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double z = -std::cos(kPi * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 60; ++it) {
            double pm = 1.0, pn = z;
            for (int k = 2; k <= n; ++k) {
                const double pk = ((2 * k - 1) * z * pn - (k - 1) * pm) / k;
                pm = pn;
                pn = pk;
            }
            const double dz = pn / (n * (z * pn - pm) / (z * z - 1.0));
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double pm = 1.0, pn = z;
        for (int k = 2; k <= n; ++k) {
            const double pk = ((2 * k - 1) * z * pn - (k - 1) * pm) / k;
            pm = pn;
            pn = pk;
        }
        const double d = n * (z * pn - pm) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * d * d);
    }
}

// Nodes per step integral.  The integrands 1/(a H sqrt(q^2 + m^2 a^2)) and
// their kin are analytic in ln a within |Im ln a| < pi/2 (the branch points of
// sqrt(q^2 + m^2 a^2) sit at a = +-i q/m), so an n-point Gauss-Legendre rule
// on a step of half-width h converges like rho^(-2n) with rho = b + sqrt(b^2 + 1),
// b = (pi/2)/h.  Take the smallest n (2..8) with rho^(-2n) < 1e-13.
int auto_nodes(double dlna)
{
    const double h = 0.5 * std::fabs(dlna);
    const double b = 0.5 * kPi / h;
    const double rho = b + std::sqrt(b * b + 1.0);
    int n = 2;
    while (n < kMaxGL && std::pow(rho, -2.0 * n) > 1e-13) ++n;
    return n;
}

// ---- the FP64-state form's step integrals as polynomials (WideCoef) ---------------
// g(t) = sum_j W_j (1 + e_j t)^power on t in [0, 1] (power -1/2 or +1/2), interpolated at
// the Chebyshev points of [0, 1] and written as monomial coefficients in t.  The degree
// is the smallest in [max(nf64, 3), kWideDeg] for which the polynomial agrees with the sum
// within `tol` of max |g| at 65 points of [0, 1] after the device's split (the first
// nf64 coefficients in FP64, the rest rounded to FP32), with the FP32 Horner sum's
// rounding bounded by sum_{k >= nf64} |a_k| 4 2^-24 added.  Returns false (the pass
// then integrates node by node) if no degree does.
bool fit_wide_poly(const double* W, const double* e, int n, double power, int nf64, double tol, WidePoly& P)
{
    std::memset(&P, 0, sizeof(P));
    auto g = [&](long double t) {
        long double v = 0;
        for (int j = 0; j < n; ++j) {
            const double b = std::sqrt(1.0 + e[j] * (double)t);
            v += (long double)W[j] * (power < 0 ? 1.0L / b : (long double)b);
        }
        return v;
    };
    constexpr int kCheck = 64;   // check points t = i / kCheck
    long double gmax = 0;
    for (int i = 0; i <= kCheck; ++i) gmax = std::max(gmax, std::fabs(g((long double)i / kCheck)));
    if (gmax == 0) return true;
    for (int K = std::max(nf64, 3); K <= kWideDeg; ++K) {
        // Chebyshev coefficients of g(t(s)), s = 2t - 1, from its values at the K + 1 points
        long double cc[kWideDeg + 1] = {};
        long double gv[kWideDeg + 1];
        for (int i = 0; i <= K; ++i) {
            const long double th = 3.14159265358979323846264338327950288L * (i + 0.5L) / (K + 1);
            gv[i] = g((1.0L + std::cos(th)) / 2);
        }
        for (int m = 0; m <= K; ++m) {
            long double acc = 0;
            for (int i = 0; i <= K; ++i)
                acc += gv[i] * std::cos(3.14159265358979323846264338327950288L * m * (i + 0.5L) / (K + 1));
            cc[m] = acc * 2 / (K + 1);
        }
        cc[0] /= 2;
        // T_m(2t - 1) as polynomials in t: T_0 = 1, T_1 = 2t - 1, T_{m+1} = 2 (2t - 1) T_m - T_{m-1}
        long double Tm1[kWideDeg + 2] = {}, Tm[kWideDeg + 2] = {}, a[kWideDeg + 1] = {};
        Tm1[0] = 1;
        Tm[0] = -1;
        Tm[1] = 2;
        a[0] += cc[0];
        for (int m = 1; m <= K; ++m) {
            for (int k = 0; k <= m; ++k) a[k] += cc[m] * Tm[k];
            long double Tn[kWideDeg + 2] = {};
            for (int k = 0; k <= m; ++k) {
                Tn[k + 1] += 4 * Tm[k];
                Tn[k] -= 2 * Tm[k];
            }
            for (int k = 0; k <= m + 1; ++k) Tn[k] -= Tm1[k];
            std::memcpy(Tm1, Tm, sizeof(Tm));
            std::memcpy(Tm, Tn, sizeof(Tn));
        }
        // the device's evaluation: FP64 coefficients below nf64, FP32 ones above
        long double tail = 0;
        for (int k = nf64; k <= K; ++k) tail += std::fabs(a[k]);
        const long double tail_bound = tail * 4 * 5.9604644775390625e-8L;
        long double err = 0;
        for (int i = 0; i <= kCheck; ++i) {
            const long double t = (long double)i / kCheck;
            long double pt = 0;
            for (int k = K; k >= 0; --k) pt = pt * t + (k < nf64 ? (long double)(double)a[k] : (long double)(float)a[k]);
            err = std::max(err, std::fabs(pt - g(t)));
        }
        if ((err + tail_bound) <= tol * gmax) {
            for (int k = 0; k < nf64; ++k) P.c64[k] = (double)a[k];
            for (int k = nf64; k <= K; ++k) P.c32[k - nf64] = (float)a[k];
            return true;
        }
    }
    return false;
}

FF split_ff(double v)
{
    FF r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
}

struct StateLayout {
    size_t X, q0f, dqf, xd, qd, q0d, sd, pmag, id;
};

// Steps per particle pass: the caller's choice, else 4 for the FP32/BF16-grid forms (the
// particle state is read and written once per 4 steps) and 1 for the plain form.
int steps_per_pass(const fdf_params& p)
{
    if (p.steps_per_pass > 0) return p.steps_per_pass;
    return form_of(p.precision) == kPlain ? 1 : 4;
}

// Grids held at once: the current pass's (its steps plus the opening kick's) and
// the next pass's, which are built on a second stream while the current pass runs.
constexpr int kMaxBuf = 2 * (kMaxSub - 1) + 1;
int grid_buffers(const fdf_params& p) { return std::min(kMaxBuf, 2 * steps_per_pass(p) + 1); }

struct Layout {
    size_t tabs, modeA, noise, cdf_t, cdf_F, tw, W0, W1, G[kMaxBuf], Gss[2], qs, stage, dep, flag, ctr, key, hist, bsum,
        recs, total;
    int nbuf;
    StateLayout s[2];
};

int64_t sort_bins(const fdf_params& p)
{
    const int64_t tpa = p.n_grid >> sort_tile_shift(p);
    return tpa * tpa * tpa * p.n_species;
}

Layout make_layout(const fdf_params& p, int nk, int na, int ncdf)
{
    Layout L{};
    const int prec = p.precision;
    const size_t N = (size_t)p.n_grid, N3 = N * N * N;
    const size_t n = (size_t)p.n_part * (size_t)p.n_species;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes ? bytes : 1);
        return o;
    };
    L.tabs = take(3 * (size_t)na * nk * 8);
    L.modeA = take(4 * (size_t)mode_table_size(p.n_grid) * real_bytes(prec));
    L.noise = take(N3 * complex_bytes(prec));
    L.cdf_t = take((size_t)ncdf * 8);
    L.cdf_F = take((size_t)ncdf * 8);
    L.tw = take(N * complex_bytes(prec));
    L.W0 = take(4 * N3 * complex_bytes(prec));
    L.W1 = take(4 * N3 * complex_bytes(prec));
    L.nbuf = grid_buffers(p);
    for (int b = 0; b < L.nbuf; ++b) L.G[b] = take(N3 * grid_bytes_per_cell(prec));
    // the two super-step grids an interpolated step reads (super-steps only)
    for (int b = 0; b < 2; ++b) L.Gss[b] = take(p.superstep_tol > 0 ? N3 * grid_bytes_per_cell(prec) : 0);
    const int form = form_of(prec);
    const bool split = form != kPlain;     // sorts the sampler's output before the transform
    const bool sorts = p.sort_every >= 0;
    for (int h = 0; h < (sorts ? 2 : 1); ++h) {
        StateLayout& S = L.s[h];
        // the plain form's live positions are FP64; its sampled fixed-point
        // positions are written once and never permuted, so they are not doubled
        S.X = (h == 0 || split) ? take(3 * n * 4) : L.s[0].X;
        S.q0f = take(split ? 3 * n * 4 : 0);
        S.dqf = take(form == kFixed ? 3 * n * 4 : 0);
        S.xd = take(form != kFixed ? 3 * n * 8 : 0);
        S.qd = take(form != kFixed ? 3 * n * 8 : 0);
        S.q0d = take(form == kPlain ? 3 * n * 8 : 0);
        // 1 + phi + psi's phi + psi at each particle, carried from a kick to the next
        // drift (the exact equations of motion only)
        S.sd = take(p.eom == FDF_EOM_EXACT ? n * 8 : 0);
        S.pmag = take(n * 8);
        S.id = take(n * 4);
    }
    if (!sorts) L.s[1] = L.s[0];
    L.qs = take(3 * n * 8);
    L.key = take(sorts ? n * 4 : 0);
    L.hist = take(sorts ? (size_t)sort_bins(p) * 4 : 0);
    // scan totals of every level: bins/1024 + bins/1024^2 + ... < bins/1000 + 3
    L.bsum = take(sorts ? ((size_t)sort_bins(p) / 1000 + 64) * 4 : 0);
    L.recs = take(sorts ? n * sort_record_bytes(prec) : 0);
    L.stage = take(7 * (size_t)p.n_part * 8);
    L.dep = take(N3 * 8);
    L.flag = take(64);
    L.ctr = take(64);
    L.total = off;
    return L;
}

}  // namespace

int fdf::set_error(int code, const char* msg)
{
    g_last_error = msg;
    return code;
}

int fdf::validate_params(const fdf_params* p)
{
    if (!p) return fail(FDF_EINVAL, "params is NULL");
    if (!(p->box_mpc > 0) || !std::isfinite(p->box_mpc)) return fail(FDF_EINVAL, "box_mpc must be > 0");
    if (p->n_part < 0) return fail(FDF_EINVAL, "n_part must be >= 0");
    if (!is_pow2(p->n_grid) || p->n_grid < 8 || p->n_grid > 512)
        return fail(FDF_EINVAL, "n_grid must be a power of two in [8, 512]");
    if (p->n_species < 1 || p->n_species > kMaxSpecies) return fail(FDF_EINVAL, "n_species must be in 1..4");
    if ((double)p->n_part * p->n_species >= 4294967296.0) return fail(FDF_EINVAL, "more than 2^32 - 1 particles");
    for (int s = 0; s < p->n_species; ++s)
        if (!(p->m_ev[s] >= 0) || !std::isfinite(p->m_ev[s])) return fail(FDF_EINVAL, "masses must be >= 0");
    if (!(p->T_nu_K > 0)) return fail(FDF_EINVAL, "T_nu_K must be > 0");
    if (!(p->z_start > p->z_end) || !(p->z_end > -1.0) || !std::isfinite(p->z_start))
        return fail(FDF_EINVAL, "need z_start > z_end > -1");
    if (p->n_steps < 1) return fail(FDF_EINVAL, "n_steps must be >= 1");
    if (p->precision < FDF_PREC_F64 || p->precision > FDF_PREC_BF16_FIXED) return fail(FDF_EINVAL, "unknown precision");
    if (p->n_gl != 0 && (p->n_gl < 2 || p->n_gl > kMaxGL)) return fail(FDF_EINVAL, "n_gl must be 0 or 2..8");
    if (!(p->h > 0) || !(p->omega_m >= 0) || !(p->omega_r >= 0) || !(p->A_s > 0) || !(p->k_pivot > 0) ||
        !std::isfinite(p->n_s))
        return fail(FDF_EINVAL, "invalid cosmology");
    const double ol = 1.0 - p->omega_m - p->omega_r;
    const double a0 = 1.0 / (1.0 + p->z_start);
    if (!(p->omega_r / (a0 * a0 * a0 * a0) + p->omega_m / (a0 * a0 * a0) + ol > 0))
        return fail(FDF_EINVAL, "H^2 <= 0 at z_start");
    if (p->flags & ~(FDF_FLAG_FIXED_AMPLITUDE | FDF_FLAG_LEGENDRE_DIPOLE)) return fail(FDF_EINVAL, "unknown flags");
    if (p->sort_every < -1) return fail(FDF_EINVAL, "sort_every must be -1, 0 or a step count");
    if (p->steps_per_pass < 0 || p->steps_per_pass > kMaxSub - 1)
        return fail(FDF_EINVAL, "steps_per_pass must be 0 (automatic) or 1..8");
    if (p->sort_tile < 0 || p->sort_tile > 3 || (p->n_grid >> p->sort_tile) < 1)
        return fail(FDF_EINVAL, "sort_tile must be 0..3 and at most log2(n_grid)");
    if (p->sort_cells < 0) return fail(FDF_EINVAL, "sort_cells must be >= 0");
    if (p->interp_order < 0 || p->interp_order > 2) return fail(FDF_EINVAL, "interp_order must be 0, 1 or 2");
    if (p->pass_blocks < 0 || p->pass_blocks > 3) return fail(FDF_EINVAL, "pass_blocks must be 0 (automatic) or 1..3");
    if (p->gather_tile < -1 || p->gather_tile > 1) return fail(FDF_EINVAL, "gather_tile must be -1, 0 or 1");
    if (p->deposit_presum < -1 || p->deposit_presum > 1)
        return fail(FDF_EINVAL, "deposit_presum must be -1, 0 or 1");
    if (!(p->superstep_tol >= 0.0) || !std::isfinite(p->superstep_tol))
        return fail(FDF_EINVAL, "superstep_tol must be finite and >= 0");
    if (p->eom < FDF_EOM_GEODESIC || p->eom > FDF_EOM_EXACT) return fail(FDF_EINVAL, "unknown eom");
    if (p->eom != FDF_EOM_GEODESIC && p->precision != FDF_PREC_F64)
        return fail(FDF_ENOSYS, "the comparison equations of motion run in the plain FP64 form only");
    // the exact form splits every kick in two sub-steps: an opening kick and two
    // sub-steps per leapfrog step must fit in one pass
    if (p->eom == FDF_EOM_EXACT && p->steps_per_pass > 2)
        return fail(FDF_EINVAL, "steps_per_pass must be 0, 1 or 2 with FDF_EOM_EXACT");
    return FDF_OK;
}

void fdf::twiddle_table(int N, double* cs)
{
    for (int j = 0; j < N; ++j) {
        cs[2 * j] = std::cos(2.0 * kPi * j / N);
        cs[2 * j + 1] = std::sin(2.0 * kPi * j / N);
    }
}

bool fdf::uniform_grid(const double* v, int n, double* v0, double* dv)
{
    if (n < 2) return false;
    const double d = (v[n - 1] - v[0]) / (n - 1);
    if (!(d > 0)) return false;
    for (int i = 0; i < n; ++i)
        if (std::fabs(v[i] - (v[0] + i * d)) > 1e-9 * std::fabs(d) + 1e-12 * std::fabs(v[i])) return false;
    *v0 = v[0];
    *dv = d;
    return true;
}

namespace {
int validate(const fdf_params* p) { return fdf::validate_params(p); }
}  // namespace

struct fdf_ctx {
    fdf_params p{};
    cudaStream_t stream = nullptr;
    int64_t n = 0;
    int ngl = 4, nkick = 4;
    int sm_count = 152;                     // SMs of the context's device
    double glx[kMaxGL]{}, glw[kMaxGL]{};    // drift rule
    double glxk[kMaxGL]{}, glwk[kMaxGL]{};  // kick rule
    int uniform = 0;                        // all species share one mass
    double T_ev = 0, H0 = 0, ol = 0, lna0 = 0, lnaN = 0, dlna = 0, a0 = 0, tau0 = 0;
    int nk = 0, na = 0, ncdf = 0;
    std::vector<double> tab_host;     // T_psi, T_phi, dT_phi/dln a on the host (super-step schedule)
    std::vector<int> is_super;        // super-step schedule, n_steps + 1 entries
    bool supersteps = false;
    int slot7 = kSlot7Psi;               // what the grids built next carry in slot 7
    void* Gss[2] = {nullptr, nullptr};
    int ssk[2] = {-1, -1};            // the step each super-step grid holds
    double lnk0 = 0, dlnk = 0, lnat0 = 0, dlnat = 0;
    // fitted integral polynomials of the FP64-state form by interval (ln a ends) and
    // kind (0 drift, 1 kick 1/eps, 2 kick eps), with whether the fit passed
    std::map<std::tuple<double, double, int>, std::pair<bool, WidePoly>> wide_fits;
    Layout lay{};
    char* block = nullptr;
    bool own_block = false;
    double* tabs = nullptr;   // FP64 [3][na][nk]
    void* modeA = nullptr;    // per-step amplitude table
    void* noise = nullptr;    // unit Gaussian field of the run
    bool noise_ready = false;
    double* cdf_t = nullptr;
    double* cdf_F = nullptr;
    void* tw = nullptr;
    void* W0 = nullptr;
    void* W1 = nullptr;
    int nbuf = 0;
    void* G[kMaxBuf] = {};
    int gk[kMaxBuf];                     // step index whose fields each buffer holds (-1: none)
    cudaEvent_t built[kMaxBuf] = {};     // recorded on the fields stream after a build
    cudaEvent_t released[kMaxBuf] = {};  // recorded on the main stream after the last read
    bool has_release[kMaxBuf] = {};
    cudaStream_t sf = nullptr;           // the fields stream
    cudaEvent_t joined = nullptr;
    int spp = 1;                         // steps per particle pass
    void* Gfrozen = nullptr;
    bool frozen = false;
    ParticleState st{};       // the live state
    ParticleState st_alt{};   // the other half of the double buffer (sort target)
    uint32_t* key = nullptr;
    uint32_t* hist = nullptr;
    uint32_t* bsum = nullptr;
    void* recs = nullptr;
    double disp = 0;          // typical displacement (Mpc) since the last sort
    int64_t sorts = 0;
    double* stage = nullptr;
    double* dep = nullptr;
    int* dflag = nullptr;
    unsigned long long* pass_ctr = nullptr;   // the FP64-state pass's work counters (zero between passes)
    bool sampled = false;
    bool stepped = false;
    int k = 0;
    int64_t launches = 0;
    // the passes of the last fdf_step: all with series integrals, count, most steps in one
    int pass_series = 1, pass_count = 0, pass_steps = 0;
    // the call of fdf_step being issued (slice_begin .. slice_done)
    struct Slice {
        bool active = false;
        int dir = 1, steps = 0, k_start = 0, passes = 0, j = 0;
        std::vector<int> bufs_cur, bufs_next;
        std::vector<const void*> grids_cur, grids_next;
    } slice;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
    // the recorded run of fdf_run_graph, and the host state it leaves behind
    struct RunGraph {
        int n = -1;
        cudaGraphExec_t exec = nullptr;
        cudaEvent_t fork = nullptr;
        cudaStream_t own = nullptr;      // records and replays a run queued on the legacy stream
        int gk[kMaxBuf];
        int ssk[2];
        int slot7 = kSlot7Psi;
        int k = 0;
        double disp = 0;
        ParticleState st{}, st_alt{};
        int64_t launches = 0, sorts = 0;
        int pass_series = 1, pass_count = 0, pass_steps = 0;
    } graph;

    double hubble(double a) const
    {
        return H0 * std::sqrt(p.omega_r / (a * a * a * a) + p.omega_m / (a * a * a) + ol);
    }
    double lna(double kk) const { return lna0 + kk * dlna; }
};

namespace {

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(FDF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define FDF_CUDA(call, what)                                  \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, (what));  \
    } while (0)

cudaEvent_t take_event(fdf_ctx* c)
{
    if (c->pool_used == c->pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->pool.push_back(e);
    }
    return c->pool[c->pool_used++];
}

// Runs one launch on stream s, bracketed by events when timing is on.
template <typename F>
int timed_on(fdf_ctx* c, cudaStream_t s, int cls, const char* what, F&& launch)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->timing) {
        e0 = take_event(c);
        e1 = take_event(c);
        if (e0) cudaEventRecord(e0, s);
    }
    cudaError_t e = launch();
    ++c->launches;
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (c->timing && e0 && e1) {
        cudaEventRecord(e1, s);
        c->marks.push_back({cls, {e0, e1}});
    }
    return FDF_OK;
}

template <typename F>
int timed(fdf_ctx* c, int cls, const char* what, F&& launch)
{
    return timed_on(c, c->stream, cls, what, launch);
}

// Conformal time from a = 0: tau(a0) = int_0^a0 da / (a^2 H), a 32-point
// Gauss-Legendre rule on [0, a0] (the integrand 1/(H0 sqrt(omega_r + omega_m a
// + Omega_L a^4)) is smooth there).
double tau_of(const fdf_ctx* c, double a)
{
    double x[32], w[32];
    gauss_legendre(32, x, w);
    double s = 0;
    for (int j = 0; j < 32; ++j) {
        const double aj = 0.5 * a * (x[j] + 1.0);
        s += w[j] / std::sqrt(c->p.omega_r + c->p.omega_m * aj + c->ol * aj * aj * aj * aj);
    }
    return 0.5 * a * s / c->H0;
}

// Gauss-Legendre nodes of [l1, l2] in ln a (the drift rule, or the kick rule if
// kick): weights W_j (dtau) and a_j^2.
void nodes(const fdf_ctx* c, double l1, double l2, double* W, double* a2, bool kick = false)
{
    const double half = 0.5 * (l2 - l1), mid = 0.5 * (l1 + l2);
    const int n = kick ? c->nkick : c->ngl;
    const double* x = kick ? c->glxk : c->glx;
    const double* w = kick ? c->glwk : c->glw;
    for (int j = 0; j < n; ++j) {
        const double a = std::exp(mid + half * x[j]);
        W[j] = w[j] * half / (a * c->hubble(a));
        a2[j] = a * a;
    }
}

// Constants of a particle pass that do not depend on the sub-steps.
void fill_pass(const fdf_ctx* c, PushArgs& a)
{
    std::memset(&a, 0, sizeof(a));
    a.n = c->n;
    a.n_part = c->p.n_part > 0 ? c->p.n_part : 1;
    for (int s = 0; s < kMaxSpecies; ++s)
        a.sp_begin[s] = s + 1 < c->p.n_species ? (int64_t)(s + 1) * c->p.n_part : INT64_MAX;
    a.n_gl = c->ngl;
    a.n_kick = c->nkick;
    a.uniform_species = c->uniform;
    a.order = c->p.interp_order == 2 ? 2 : 1;
    a.eom = c->p.eom;
    a.wide_series = 1;
    for (int s = 0; s < kMaxSpecies; ++s) a.m2[s] = c->p.m_ev[s] * c->p.m_ev[s];
    const int pb = c->p.pass_blocks > 0 ? c->p.pass_blocks : 2;
    a.grid_blocks = c->sm_count * pb;
    a.pair = pb == 2 ? 1 : 0;
    a.ctr = c->pass_ctr;
    a.tile_gather = c->p.gather_tile > 0 ? 1 : 0;
    a.N = c->p.n_grid;
    a.L = c->p.box_mpc;
    a.invL = 1.0 / c->p.box_mpc;
    a.invh = c->p.n_grid / c->p.box_mpc;
    a.fx_scale = split_ff(4294967296.0 / c->p.box_mpc);
}

// The FP64-state form's coefficients of a sub-step (WideCoef): for each interval, the
// centre a_c (midpoint in ln a), e_j = a_j^2 / a_c^2 - 1 and the fitted polynomials.
// Drift integrals are fitted to 2e-13 of their size, kick integrals (which only scale a
// kick of at most ~1e-3 of |q|) to 1e-9.  u.wide_ok = 0 if a fit failed.
void fill_wide(fdf_ctx* c, bool drift, double d1, double d2, const double* Wd, const double* ad, bool kick,
               double k1, double k2, const double* Wk, const double* ak, SubStep& u)
{
    WideCoef& w = u.wide;
    u.wide_ok = 1;
    auto fit = [&](double l1, double l2, int kind, const double* W, const double* a2, int n, WidePoly& P) {
        const auto key = std::make_tuple(l1, l2, kind);
        auto it = c->wide_fits.find(key);
        if (it == c->wide_fits.end()) {
            const double a2c = std::exp(l1 + l2);       // a_c^2 at the midpoint in ln a
            double e[kMaxGL];
            for (int j = 0; j < n; ++j) e[j] = a2[j] / a2c - 1.0;
            WidePoly Q;
            const bool ok = kind == 0 ? fit_wide_poly(W, e, n, -0.5, kWideD64, 2e-13, Q)
                                      : fit_wide_poly(W, e, n, kind == 1 ? -0.5 : 0.5, kWideK64, 1e-9, Q);
            it = c->wide_fits.emplace(key, std::make_pair(ok, Q)).first;
        }
        P = it->second.second;
        if (!it->second.first) u.wide_ok = 0;
    };
    if (drift) {
        WidePoly P;
        fit(d1, d2, 0, Wd, ad, c->ngl, P);
        double sum = 0;
        for (int j = 0; j < c->ngl; ++j) sum += Wd[j];
        for (int s = 0; s < c->p.n_species; ++s) {
            const double mac = c->p.m_ev[s] * std::exp(0.5 * (d1 + d2));      // m a_c
            w.wsum[s] = sum;
            w.inv_muc[s] = mac > 0 ? 1.0 / (mac * mac) : 0.0;
            w.massless[s] = mac > 0 ? 0 : 1;
            // the species' copy of the polynomial carries the factor 1/(m a_c)
            const double f = mac > 0 ? 1.0 / mac : 0.0;
            for (int k = 0; k < kWideD64; ++k) w.drift[s].c64[k] = P.c64[k] * f;
            for (int k = 0; k <= kWideDeg; ++k) w.drift[s].c32[k] = (float)((double)P.c32[k] * f);
        }
    }
    if (kick) {
        for (int s = 0; s < c->p.n_species; ++s) w.muk[s] = c->p.m_ev[s] * c->p.m_ev[s] * std::exp(k1 + k2);
        fit(k1, k2, 1, Wk, ak, c->nkick, w.kphi);
        fit(k1, k2, 2, Wk, ak, c->nkick, w.kpsi);
        double dt = 0;
        for (int j = 0; j < c->nkick; ++j) dt += Wk[j];
        w.dtau_k = (float)dt;
    }
}

// Coefficients of one sub-step: drift over [d1, d2] (if any), kick over [k1, k2] (if any).
// The split form's drift weights carry the factor 2^32/L (position quanta per Mpc).
void fill_substep(fdf_ctx* c, bool drift, double d1, double d2, bool kick, double k1, double k2, SubStep& u)
{
    std::memset(&u, 0, sizeof(u));
    u.do_drift = drift;
    u.do_kick = kick;
    double Wd[kMaxGL], ad[kMaxGL], Wk[kMaxGL], ak[kMaxGL];
    if (drift) nodes(c, d1, d2, Wd, ad);
    if (kick) nodes(c, k1, k2, Wk, ak, true);
    const int jc = c->ngl / 2;
    const double q32 = 4294967296.0 / c->p.box_mpc;
    for (int s = 0; s < c->p.n_species; ++s) {
        SpeciesCoef& sc = u.sp[s];
        const double m2 = c->p.m_ev[s] * c->p.m_ev[s];
        if (drift) {
            double sum = 0;
            for (int j = 0; j < c->ngl; ++j) {
                sc.Wd[j] = Wd[j];
                sc.mud[j] = m2 * ad[j];
                sum += Wd[j];
            }
            sc.Wd_sum = split_ff(sum * q32);
            sc.mud_c = split_ff(sc.mud[jc]);
            sc.mud_c_f = (float)sc.mud[jc];
            double e[kMaxGL];
            for (int j = 0; j < c->ngl; ++j) {
                sc.Wd_f[j] = (float)(Wd[j] * q32);
                sc.dmud_f[j] = (float)(sc.mud[j] - sc.mud[jc]);
                e[j] = sc.mud[jc] > 0 ? (sc.mud[j] - sc.mud[jc]) / sc.mud[jc] : 0.0;
                u.emax = std::max(u.emax, std::fabs(e[j]));
            }
            // Cd_k = c_k sum_j Wd_j e_j^k with c_k the binomial coefficients of
            // (1 + d)^(-1/2) - 1 = sum_k c_k d^k: c_1 = -1/2, c_k = c_(k-1) (1 - 2k)/(2k)
            double ck = 1.0;
            for (int k = 1; k <= kTaylor; ++k) {
                ck *= (1.0 - 2.0 * k) / (2.0 * k);
                double m = 0;
                for (int j = 0; j < c->ngl; ++j) m += Wd[j] * std::pow(e[j], k);
                sc.Cd[k - 1] = (float)(ck * m * q32);
            }
        }
        if (kick) {
            double dt = 0, ka = 0;
            for (int j = 0; j < c->nkick; ++j) {
                sc.Wk[j] = Wk[j];
                sc.muk[j] = m2 * ak[j];
                sc.Wk_f[j] = (float)Wk[j];
                sc.muk_f[j] = (float)sc.muk[j];
                dt += Wk[j];
                ka += Wk[j] * std::sqrt(ak[j]);
            }
            sc.Ka = c->p.m_ev[s] * ka;
            sc.dtau_k = dt;
            sc.dtau_k_f = (float)dt;
        }
    }
    if (form_of(c->p.precision) == kWide) fill_wide(c, drift, d1, d2, Wd, ad, kick, k1, k2, Wk, ak, u);
}

// The unit Gaussian field of the run (a function of the seed and the mesh only),
// on the fields stream.
int draw_noise(fdf_ctx* c)
{
    const FieldArgs a = make_field_args(c->p, c->nk, c->na, c->lnk0, c->dlnk, c->lnat0, c->dlnat, c->lna0);
    int rc = timed_on(c, c->sf, FDF_K_FIELDS_Z, "noise",
                      [&] { return launch_noise(c->sf, grid_prec(c->p.precision), a, c->noise); });
    if (rc == FDF_OK) c->noise_ready = true;
    return rc;
}

// The eight fields at ln a into G, on stream s; slot 7 as `slot7` says (kSlot7*).
int build_fields(fdf_ctx* c, double lna, void* G, cudaStream_t s, int slot7)
{
    if (!c->noise_ready) {
        if (s != c->sf) FDF_CUDA(cudaStreamSynchronize(c->stream), "sync");
        int rc0 = draw_noise(c);
        if (rc0) return rc0;
        if (s != c->sf) FDF_CUDA(cudaStreamSynchronize(c->sf), "sync");
    }
    FieldArgs a = make_field_args(c->p, c->nk, c->na, c->lnk0, c->dlnk, c->lnat0, c->dlnat, lna);
    a.slot7 = slot7;
    const int prec = grid_prec(c->p.precision);
    int rc = timed_on(c, s, FDF_K_FIELDS_Z, "mode table",
                      [&] { return launch_mode_table(s, prec, a, c->tabs, c->modeA); });
    if (rc) return rc;
    rc = timed_on(c, s, FDF_K_FIELDS_Z, "fields z pass",
                  [&] { return launch_fields_z(s, prec, a, c->modeA, c->noise, c->tw, c->W0); });
    if (rc) return rc;
    rc = timed_on(c, s, FDF_K_FIELDS_Y, "fields y pass",
                  [&] { return launch_fields_y(s, prec, a, c->tw, c->W0, c->W1); });
    if (rc) return rc;
    return timed_on(c, s, FDF_K_FIELDS_X, "fields x pass",
                    [&] { return launch_fields_x(s, prec, a, c->tw, c->W1, G); });
}

int push(fdf_ctx* c, const PushArgs& a)
{
    return timed(c, FDF_K_PUSH, "particle pass", [&] { return launch_push(c->stream, c->p.precision, c->st, a); });
}

// ---- super-steps (Sec. 2.1) --------------------------------------------------------
// The fields are built by transform only at super-steps: steps 0 and n_steps, and
// every step whose transfer functions of phi and psi changed by more than
// superstep_tol since the last super-step.  Between super-steps s < k < e they are
// interpolated linearly in ln a.  The change between steps j0 and j1 is, for
// T = T_psi and T_phi, the largest |T(k, a_j1) - T(k, a_j0)| over 64 ln k points
// spanning the mesh's modes (2 pi/L to sqrt(3) pi N/L), relative to the largest
// |T(k, a_j0)| there; the larger of the two.

// Bilinear read of table `which` (0 T_psi, 1 T_phi), clamped at the edges.
double table_at(const fdf_ctx* c, int which, double lnk, double lna)
{
    auto locate = [](double v, double v0, double dv, int n, int* i, double* f) {
        const double pos = (v - v0) / dv;
        if (pos <= 0.0) {
            *i = 0;
            *f = 0.0;
        } else if (pos >= n - 1) {
            *i = n - 2;
            *f = 1.0;
        } else {
            *i = (int)pos;
            *f = pos - *i;
        }
    };
    int ik, ia;
    double fk, fa;
    locate(lnk, c->lnk0, c->dlnk, c->nk, &ik, &fk);
    locate(lna, c->lnat0, c->dlnat, c->na, &ia, &fa);
    const double* T = c->tab_host.data() + (size_t)which * c->na * c->nk;
    const double* r0 = T + (size_t)ia * c->nk;
    const double* r1 = r0 + c->nk;
    const double v0 = (1.0 - fk) * r0[ik] + fk * r0[ik + 1];
    const double v1 = (1.0 - fk) * r1[ik] + fk * r1[ik + 1];
    return (1.0 - fa) * v0 + fa * v1;
}

double tf_change(const fdf_ctx* c, int j0, int j1)
{
    const double lk0 = std::log(2.0 * kPi / c->p.box_mpc);
    const double lk1 = std::log(std::sqrt(3.0) * kPi * c->p.n_grid / c->p.box_mpc);
    const double la0 = c->lna(j0), la1 = c->lna(j1);
    double worst = 0.0;
    for (int which = 0; which < 2; ++which) {
        double dmax = 0.0, tmax = 0.0;
        for (int i = 0; i < 64; ++i) {
            const double lk = lk0 + (lk1 - lk0) * i / 63.0;
            const double t0 = table_at(c, which, lk, la0), t1 = table_at(c, which, lk, la1);
            dmax = std::max(dmax, std::fabs(t1 - t0));
            tmax = std::max(tmax, std::fabs(t0));
        }
        if (tmax > 0.0) worst = std::max(worst, dmax / tmax);
    }
    return worst;
}

void superstep_schedule(fdf_ctx* c)
{
    const int n = c->p.n_steps;
    c->supersteps = c->p.superstep_tol > 0.0;
    c->is_super.assign(n + 1, c->supersteps ? 0 : 1);
    c->is_super[0] = c->is_super[n] = 1;
    if (!c->supersteps) return;
    int s = 0;
    for (int j = 1; j < n; ++j)
        if (tf_change(c, s, j) > c->p.superstep_tol) {
            c->is_super[j] = 1;
            s = j;
        }
}

// The fields of step k into G on the fields stream: a transform, or with super-steps
// the interpolation between the two bracketing super-steps, which are built into the
// two super-step grids as needed (a step that is itself a super-step is the copy w = 0).
int produce_grid(fdf_ctx* c, int k, void* G)
{
    if (!c->supersteps) return build_fields(c, c->lna(k), G, c->sf, c->slot7);
    int s = k, e = k;
    while (!c->is_super[s]) --s;
    while (!c->is_super[e]) ++e;
    int slot[2] = {-1, -1};
    const int need[2] = {s, e};
    for (int n = 0; n < 2; ++n)
        for (int i = 0; i < 2; ++i)
            if (c->ssk[i] == need[n]) slot[n] = i;
    for (int n = 0; n < 2; ++n) {
        if (slot[n] >= 0) continue;
        if (n == 1 && s == e) {
            slot[1] = slot[0];
            break;
        }
        const int i = slot[1 - n] == 0 ? 1 : 0;   // the grid the other end does not use
        c->ssk[i] = -1;
        int rc = build_fields(c, c->lna(need[n]), c->Gss[i], c->sf, c->slot7);
        if (rc) return rc;
        c->ssk[i] = need[n];
        slot[n] = i;
    }
    const double w = s == e ? 0.0 : (c->lna(k) - c->lna(s)) / (c->lna(e) - c->lna(s));
    return timed_on(c, c->sf, FDF_K_FIELDS_X, "super-step interpolation", [&] {
        return launch_interp_grid(c->sf, grid_prec(c->p.precision), c->p.n_grid, c->Gss[slot[0]], c->Gss[slot[1]], w,
                                  G);
    });
}

// The buffer holding the fields of step k, or -1.
int find_grid(const fdf_ctx* c, int k)
{
    for (int b = 0; b < c->nbuf; ++b)
        if (c->gk[b] == k) return b;
    return -1;
}

// Make the fields of step k available: the frozen set, a buffer that holds them
// already, or a buffer outside `busy` (a bit mask) built now on the fields
// stream, after the last pass that read that buffer.  The caller makes the main
// stream wait for c->built[*buf] before reading.
int ensure_grid(fdf_ctx* c, int k, unsigned busy, const void** G, int* buf)
{
    if (c->frozen) {
        *G = c->Gfrozen;
        *buf = -1;
        return FDF_OK;
    }
    int b = find_grid(c, k);
    if (b < 0) {
        for (int i = 0; i < c->nbuf; ++i) {
            const int cand = ((k % c->nbuf) + c->nbuf + i) % c->nbuf;
            if (!(busy & (1u << cand))) {
                b = cand;
                break;
            }
        }
        if (b < 0) return fail(FDF_EINVAL, "no free grid buffer");
        c->gk[b] = -1;
        if (c->has_release[b]) FDF_CUDA(cudaStreamWaitEvent(c->sf, c->released[b], 0), "wait release");
        int rc = produce_grid(c, k, c->G[b]);
        if (rc) return rc;
        FDF_CUDA(cudaEventRecord(c->built[b], c->sf), "record build");
        c->gk[b] = k;
    }
    *G = c->G[b];
    *buf = b;
    return FDF_OK;
}

// The main stream reads buffer b next: wait for its build.
int acquire_grid(fdf_ctx* c, int b)
{
    if (b >= 0) FDF_CUDA(cudaStreamWaitEvent(c->stream, c->built[b], 0), "wait build");
    return FDF_OK;
}

// The main stream has issued its last read of buffer b.
int release_grid(fdf_ctx* c, int b)
{
    if (b >= 0) {
        FDF_CUDA(cudaEventRecord(c->released[b], c->stream), "record release");
        c->has_release[b] = true;
    }
    return FDF_OK;
}

// Everything issued on the fields stream precedes later work on the main stream.
int join_fields(fdf_ctx* c)
{
    FDF_CUDA(cudaEventRecord(c->joined, c->sf), "record join");
    FDF_CUDA(cudaStreamWaitEvent(c->stream, c->joined, 0), "wait join");
    return FDF_OK;
}

// Sort by the positions the particles will have halfway through the next pass,
// which runs in direction dir from the current step.
int sort_particles(fdf_ctx* c, int dir, bool pre_transform = false)
{
    SortLead lead{};
    if (pre_transform) {
        // the FP32/BF16-grid forms right after sampling: by position alone, carrying the sampled momenta
        lead.pre_transform = 1;
    } else if (form_of(c->p.precision) != kPlain) {
        const double l1 = c->lna(c->k), l2 = c->lna(c->k + 0.5 * c->spp * dir);
        double W[kMaxGL], a2[kMaxGL];
        nodes(c, std::min(l1, l2), std::max(l1, l2), W, a2);
        double dt = 0;
        for (int j = 0; j < c->ngl; ++j) dt += W[j];
        const double am = std::exp(0.5 * (l1 + l2));
        lead.on = 1;
        for (int s = 0; s < c->p.n_species; ++s) {
            lead.dtau_q32[s] = (float)(dir * dt * 4294967296.0 / c->p.box_mpc);
            lead.m2a2[s] = (float)(c->p.m_ev[s] * c->p.m_ev[s] * am * am);
        }
    }
    int rc = timed(c, FDF_K_SORT, "sort", [&] {
        return launch_sort(c->stream, c->p.precision, c->st, c->st_alt, c->n, c->p.n_part > 0 ? c->p.n_part : 1,
                           c->p.n_species, c->p.n_grid, sort_tile_shift(c->p), c->p.box_mpc, lead, c->key, c->hist,
                           c->bsum, c->recs);
    });
    if (rc) return rc;
    std::swap(c->st, c->st_alt);
    c->disp = 0;
    ++c->sorts;
    return FDF_OK;
}

// Typical displacement over one step from ln a = l1 to l2: the mean
// Fermi-Dirac momentum <q> = 3.151 T moving at <q>/eps, for the fastest species.
double typical_displacement(const fdf_ctx* c, double l1, double l2)
{
    const double q = 3.15137 * c->T_ev;
    const double a = std::exp(0.5 * (l1 + l2));
    double mmin = c->p.m_ev[0];
    for (int s = 1; s < c->p.n_species; ++s) mmin = std::min(mmin, c->p.m_ev[s]);
    double W[kMaxGL], a2[kMaxGL];
    nodes(c, l1, l2, W, a2);
    double dt = 0;
    for (int j = 0; j < c->ngl; ++j) dt += W[j];
    return std::fabs(dt) * q / std::sqrt(q * q + mmin * mmin * a * a);
}

// Sort between passes if the schedule says so (c->disp accumulates per step).
int maybe_sort(fdf_ctx* c, int steps_done, int dir)
{
    const int every = c->p.sort_every;
    if (every < 0 || c->n == 0) return FDF_OK;
    bool go;
    if (every > 0) {
        go = steps_done % every < c->spp;
    } else {
        // The gather's working set stays in L2 long after a sort (the touched
        // region grows with the displacement but stays far below L2), so sort
        // when the typical particle has crossed sort_cells cells (4 by default).
        const double cell = c->p.box_mpc / c->p.n_grid;
        go = c->disp > (c->p.sort_cells > 0 ? c->p.sort_cells : 4) * cell;
    }
    return go ? sort_particles(c, dir) : FDF_OK;
}

}  // namespace

FieldArgs fdf::make_field_args(const fdf_params& p, int nk, int na, double lnk0, double dlnk, double lnat0,
                               double dlnat, double lna)
{
    FieldArgs a{};
    a.N = p.n_grid;
    a.logN = ilog2(a.N);
    a.nk = nk;
    a.na = na;
    a.kf = 2.0 * kPi / p.box_mpc;
    a.lnk0 = lnk0;
    a.inv_dlnk = 1.0 / dlnk;
    const double pos = (lna - lnat0) / dlnat;
    if (pos <= 0) {
        a.ia = 0;
        a.fa = 0;
    } else if (pos >= na - 1) {
        a.ia = na - 2;
        a.fa = 1;
    } else {
        a.ia = (int)pos;
        a.fa = pos - a.ia;
    }
    const double aa = std::exp(lna);
    const double H0 = p.h / kC_over_H100;
    const double H = H0 * std::sqrt(p.omega_r / (aa * aa * aa * aa) + p.omega_m / (aa * aa * aa) +
                                    (1.0 - p.omega_m - p.omega_r));
    a.aH = aa * H;
    const double V = p.box_mpc * p.box_mpc * p.box_mpc;
    a.amp0 = std::sqrt(2.0 * kPi * kPi * p.A_s / V);
    a.half_nsm1 = 0.5 * (p.n_s - 1.0);
    a.lnkp = std::log(p.k_pivot);
    a.key0 = (uint32_t)p.seed;
    a.key1 = (uint32_t)(p.seed >> 32);
    a.fixed_amp = (p.flags & FDF_FLAG_FIXED_AMPLITUDE) ? 1 : 0;
    return a;
}

extern "C" {

int fdf_footprint(const fdf_params* p, size_t* bytes)
{
    int rc = validate(p);
    if (rc) return rc;
    if (!bytes) return fail(FDF_EINVAL, "bytes is NULL");
    *bytes = make_layout(*p, 1024, 256, 8192).total;
    return FDF_OK;
}

int fdf_create(const fdf_params* p, const fdf_tables* t, void* stream, void* arena, size_t arena_bytes,
               fdf_ctx** out)
{
    if (!out) return fail(FDF_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    if (!t || !t->lnk || !t->lna || !t->T_psi || !t->T_phi || !t->dTphi_dlna || !t->cdf_t || !t->cdf_F)
        return fail(FDF_EINVAL, "tables incomplete");
    if (t->nk < 2 || t->na < 2 || t->nk > 1024 || t->na > 256 || t->ncdf < 2 || t->ncdf > 8192)
        return fail(FDF_EINVAL, "table sizes out of range (nk 2..1024, na 2..256, ncdf 2..8192)");
    fdf_ctx* c = new (std::nothrow) fdf_ctx;
    if (!c) return fail(FDF_ENOMEM, "host allocation failed");
    c->p = *p;
    c->stream = (cudaStream_t)stream;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            c->sm_count = sms;
    }
    c->n = p->n_part * p->n_species;
    c->H0 = p->h / kC_over_H100;
    c->ol = 1.0 - p->omega_m - p->omega_r;
    c->T_ev = p->T_nu_K * kBoltzmann_eV;
    c->lna0 = -std::log(1.0 + p->z_start);
    c->lnaN = -std::log(1.0 + p->z_end);
    c->dlna = (c->lnaN - c->lna0) / p->n_steps;
    if (c->p.n_gl == 0) c->p.n_gl = auto_nodes(c->dlna);
    c->ngl = c->p.n_gl;
    if (form_of(c->p.precision) == kFixed) {
        // the split form's kick (needed to ~1e-7) takes half the drift's nodes (2 to 4):
        // the error of an n-point rule falls like rho^(-2n), so ceil(n/2) nodes give
        // about the square root of the drift's
        c->nkick = std::min(4, std::max(2, (c->ngl + 1) / 2));
    } else {
        c->nkick = c->ngl;
    }
    gauss_legendre(c->ngl, c->glx, c->glw);
    gauss_legendre(c->nkick, c->glxk, c->glwk);
    c->uniform = 1;
    for (int s = 1; s < p->n_species; ++s)
        if (p->m_ev[s] != p->m_ev[0]) c->uniform = 0;
    c->a0 = std::exp(c->lna0);
    c->tau0 = tau_of(c, c->a0);
    c->nk = t->nk;
    c->na = t->na;
    c->ncdf = t->ncdf;
    if (!uniform_grid(t->lnk, t->nk, &c->lnk0, &c->dlnk) || !uniform_grid(t->lna, t->na, &c->lnat0, &c->dlnat)) {
        delete c;
        return fail(FDF_EINVAL, "lnk and lna must be uniform ascending grids");
    }
    for (int i = 1; i < t->ncdf; ++i)
        if (!(t->cdf_t[i] > t->cdf_t[i - 1]) || !(t->cdf_F[i] >= t->cdf_F[i - 1])) {
            delete c;
            return fail(FDF_EINVAL, "cdf_t must ascend and cdf_F must not descend");
        }
    c->lay = make_layout(c->p, t->nk, t->na, t->ncdf);
    const Layout& L = c->lay;
    if (arena) {
        if (arena_bytes < L.total) {
            delete c;
            return fail(FDF_ENOMEM, "arena smaller than the footprint");
        }
        c->block = (char*)arena;
    } else {
        cudaError_t e = cudaMalloc(&c->block, L.total);
        if (e != cudaSuccess) {
            delete c;
            return fail(FDF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        c->own_block = true;
    }
    char* b = c->block;
    c->tabs = (double*)(b + L.tabs);
    c->modeA = b + L.modeA;
    c->noise = b + L.noise;
    c->cdf_t = (double*)(b + L.cdf_t);
    c->cdf_F = (double*)(b + L.cdf_F);
    c->tw = b + L.tw;
    c->W0 = b + L.W0;
    c->W1 = b + L.W1;
    c->nbuf = L.nbuf;
    c->spp = steps_per_pass(c->p);
    for (int i = 0; i < kMaxBuf; ++i) c->gk[i] = -1;
    for (int i = 0; i < L.nbuf; ++i) c->G[i] = b + L.G[i];
    ParticleState* S2[2] = {&c->st, &c->st_alt};
    for (int h = 0; h < 2; ++h) {
        const StateLayout& S = L.s[h];
        S2[h]->X = (uint32_t*)(b + S.X);
        S2[h]->q0f = (float*)(b + S.q0f);
        S2[h]->dqf = (float*)(b + S.dqf);
        S2[h]->xd = (double*)(b + S.xd);
        S2[h]->qd = (double*)(b + S.qd);
        S2[h]->q0d = (double*)(b + S.q0d);
        S2[h]->sd = p->eom == FDF_EOM_EXACT ? (double*)(b + S.sd) : nullptr;
        S2[h]->qs = (double*)(b + L.qs);
        S2[h]->pmag = (double*)(b + S.pmag);
        S2[h]->id = (uint32_t*)(b + S.id);
    }
    c->key = (uint32_t*)(b + L.key);
    c->hist = (uint32_t*)(b + L.hist);
    c->bsum = (uint32_t*)(b + L.bsum);
    c->recs = b + L.recs;
    c->stage = (double*)(b + L.stage);
    c->dep = (double*)(b + L.dep);
    c->dflag = (int*)(b + L.flag);
    c->pass_ctr = (unsigned long long*)(b + L.ctr);
    // tables and twiddles
    const size_t ntab = (size_t)t->na * t->nk;
    const int N = p->n_grid;
    std::vector<double> tab(3 * ntab);
    std::memcpy(tab.data(), t->T_psi, ntab * 8);
    std::memcpy(tab.data() + ntab, t->T_phi, ntab * 8);
    std::memcpy(tab.data() + 2 * ntab, t->dTphi_dlna, ntab * 8);
    c->tab_host = tab;
    c->Gss[0] = b + L.Gss[0];
    c->Gss[1] = b + L.Gss[1];
    superstep_schedule(c);
    std::vector<double> twd(2 * (size_t)N);
    twiddle_table(N, twd.data());
    // uploads on the context's stream (not the legacy default stream, which would wait
    // for every other blocking stream of the device), then waited for, since the host
    // buffers belong to the caller
    const std::vector<float> twf(twd.begin(), twd.end());
    cudaStream_t s0 = c->stream;
    cudaError_t e = cudaMemcpyAsync(c->tabs, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, s0);
    if (e == cudaSuccess) {
        if (grid_prec(p->precision) == FDF_PREC_F64)
            e = cudaMemcpyAsync(c->tw, twd.data(), twd.size() * 8, cudaMemcpyHostToDevice, s0);
        else e = cudaMemcpyAsync(c->tw, twf.data(), twf.size() * 4, cudaMemcpyHostToDevice, s0);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->cdf_t, t->cdf_t, (size_t)t->ncdf * 8, cudaMemcpyHostToDevice, s0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->cdf_F, t->cdf_F, (size_t)t->ncdf * 8, cudaMemcpyHostToDevice, s0);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dflag, 0, 64, s0);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->pass_ctr, 0, 64, s0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s0);
    // the fields stream takes the priority of the caller's stream
    int prio = 0;
    if (e == cudaSuccess && c->stream) e = cudaStreamGetPriority(c->stream, &prio);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->sf, cudaStreamNonBlocking, prio);
    for (int i = 0; i < c->nbuf && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&c->built[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->released[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->joined, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "uploading tables");
        fdf_destroy(c);
        return rc;
    }
    *out = c;
    return FDF_OK;
}

}  // extern "C"

namespace fdf {

// fdf_sample without its final host synchronisation: everything is enqueued on
// the context's streams, and a failed direction draw shows in the device flag
// word only (ctx_error_flag).  The request server uses it to overlap requests.
int sample_enqueue(fdf_ctx* c)
{
    if (!c) return fail(FDF_EINVAL, "ctx is NULL");
    FDF_CUDA(cudaMemsetAsync(c->dflag, 0, 64, c->stream), "clearing flags");
    const uint32_t k0 = (uint32_t)c->p.seed, k1 = (uint32_t)(c->p.seed >> 32);
    int rc = timed(c, FDF_K_OTHER, "sampling", [&] {
        return launch_sample(c->stream, c->n, k0, k1, c->T_ev, c->cdf_t, c->cdf_F, c->ncdf, c->st.X, c->st.qs,
                             c->st.pmag, c->st.id, c->dflag);
    });
    if (rc) return rc;
    for (int i = 0; i < kMaxBuf; ++i) c->gk[i] = -1;
    c->ssk[0] = c->ssk[1] = -1;
    rc = draw_noise(c);
    if (rc) return rc;
    // The FP32/BF16-grid forms sort right after sampling, so that the transform's gather of the
    // step-0 grid runs over spatially ordered particles (at z_start a particle crosses a
    // negligible part of a cell in the first pass, so no lead is lost).  The plain form
    // keeps its sampled positions in id order and sorts after the transform.
    const bool sort0 = c->p.sort_every >= 0 && c->n > 0;
    const bool split = form_of(c->p.precision) != kPlain;
    if (sort0 && split) {
        rc = sort_particles(c, 1, true);
        if (rc) return rc;
    }
    const void* G0 = nullptr;
    int b0 = -1;
    if (c->st.sd) FDF_CUDA(cudaMemsetAsync(c->st.sd, 0, (size_t)c->n * 8, c->stream), "clearing phi + psi");
    c->slot7 = kSlot7Psi;                // the initial transform reads psi from slot 7
    rc = ensure_grid(c, 0, 0u, &G0, &b0);
    if (rc) return rc;
    rc = acquire_grid(c, b0);
    if (rc) return rc;
    // the dipole term's factor: tau0 as printed, 3 tau0 with the Legendre convention's 2l+1
    const double tau_dip = (c->p.flags & FDF_FLAG_LEGENDRE_DIPOLE) ? 3.0 * c->tau0 : c->tau0;
    rc = timed(c, FDF_K_OTHER, "initial transform", [&] {
        return launch_initial(c->stream, c->p.precision, c->st, c->n, c->p.n_part > 0 ? c->p.n_part : 1,
                              c->p.m_ev, c->a0, tau_dip, c->p.interp_order == 2 ? 2 : 1, c->p.n_grid,
                              c->p.box_mpc, G0);
    });
    if (rc) return rc;
    rc = release_grid(c, b0);
    if (rc) return rc;
    if (c->p.eom == FDF_EOM_EXACT) {
        // the steps' grids carry phi + psi in slot 7: none built so far may be reused
        c->slot7 = kSlot7Sum;
        for (int i = 0; i < kMaxBuf; ++i) c->gk[i] = -1;
        c->ssk[0] = c->ssk[1] = -1;
    } else {
        // the steps' passes read no slot 7: phi_dot is transformed alone from here on (the
        // grid of step 0, built with psi, serves the opening half kick as it is, and so does
        // the super-step grid of step 0 for the steps interpolated from it: at z = 1e9 the
        // potentials are constant and phi_dot's kick term vanishes with the conformal time)
        c->slot7 = kSlot7Zero;
    }
    c->k = 0;
    if (sort0 && !split) {
        rc = sort_particles(c, 1);
        if (rc) return rc;
    }
    c->sampled = true;
    c->stepped = false;
    return FDF_OK;
}

int* ctx_error_flag(fdf_ctx* c) { return c->dflag; }

cudaStream_t ctx_stream(fdf_ctx* c) { return c->stream; }

}  // namespace fdf

namespace fdf {

// ---- a call of fdf_step, pass by pass -------------------------------------------------
// Passes of up to spp leapfrog steps; pass j covers steps [first_j, first_j + len_j).  The
// grids of pass j+1 are built on the fields stream while pass j runs.  fdf_step runs the
// passes one after the other; the request server can launch the passes of several
// contexts together (slice_next gives a pass's arguments, slice_done what follows it).
namespace {

int pass_first(const fdf_ctx* c, int j) { return j * c->spp; }
int pass_len(const fdf_ctx* c, int j) { return std::min(c->spp, c->slice.steps - j * c->spp); }

// The grids pass j reads (its opening half kick's, then one per step), built as needed.
int slice_prepare(fdf_ctx* c, int j, std::vector<int>& bufs, std::vector<const void*>& grids, unsigned busy)
{
    const auto& sl = c->slice;
    bufs.clear();
    grids.clear();
    std::vector<int> ks;
    if (j == 0) ks.push_back(sl.k_start);                       // the opening half kick
    for (int i = 0; i < pass_len(c, j); ++i) ks.push_back(sl.k_start + sl.dir * (pass_first(c, j) + i + 1));
    for (int kk : ks) {
        const void* G = nullptr;
        int b = -1;
        int rc = ensure_grid(c, kk, busy, &G, &b);
        if (rc) return rc;
        if (b >= 0) busy |= 1u << b;
        bufs.push_back(b);
        grids.push_back(G);
    }
    return FDF_OK;
}

unsigned mask_of(const std::vector<int>& bufs)
{
    unsigned m = 0;
    for (int b : bufs)
        if (b >= 0) m |= 1u << b;
    return m;
}

}  // namespace

int slice_begin(fdf_ctx* c, int32_t n)
{
    if (!c) return fail(FDF_EINVAL, "ctx is NULL");
    if (!c->sampled) return fail(FDF_ESTATE, "fdf_step before fdf_sample");
    if (c->slice.active) return fail(FDF_ESTATE, "a slice of steps is still being issued");
    const int64_t target = (int64_t)c->k + n;
    if (target < 0 || target > c->p.n_steps) return fail(FDF_EINVAL, "step index would leave [0, n_steps]");
    if (n == 0) return FDF_OK;
    c->stepped = true;
    c->pass_series = 1;
    c->pass_count = 0;
    c->pass_steps = 0;
    auto& sl = c->slice;
    sl.dir = n > 0 ? 1 : -1;
    sl.steps = n > 0 ? n : -n;
    sl.k_start = c->k;
    sl.passes = (sl.steps + c->spp - 1) / c->spp;
    sl.j = 0;
    int rc = slice_prepare(c, 0, sl.bufs_cur, sl.grids_cur, 0u);
    if (rc) return rc;
    sl.active = true;
    return FDF_OK;
}

bool slice_active(const fdf_ctx* c) { return c->slice.active; }

int slice_next(fdf_ctx* c, PushArgs& a)
{
    auto& sl = c->slice;
    if (!sl.active) return fail(FDF_ESTATE, "no pass to issue");
    const int j = sl.j, dir = sl.dir;
    if (j + 1 < sl.passes) {
        int rc = slice_prepare(c, j + 1, sl.bufs_next, sl.grids_next, mask_of(sl.bufs_cur));
        if (rc) return rc;
    }
    fill_pass(c, a);
    a.nsub = 0;
    size_t gi = 0;
    if (j == 0) {
        fill_substep(c, false, 0, 0, true, c->lna(c->k), c->lna(c->k + 0.5 * dir), a.sub[0]);
        a.G[0] = sl.grids_cur[gi++];
        a.nsub = 1;
    }
    for (int i = 0; i < pass_len(c, j); ++i) {
        const int k0 = c->k, k1 = k0 + dir;
        const bool last = (j == sl.passes - 1) && (i == pass_len(c, j) - 1);
        // drift over the step; merged kick (closing half of this step, opening half
        // of the next) at x_{k+1} with the fields of step k+1, or only the closing half
        if (c->p.eom == FDF_EOM_EXACT) {
            // the halves stay apart: each holds q at its own start (eq:releq)
            fill_substep(c, true, c->lna(k0), c->lna(k1), true, c->lna(k0 + 0.5 * dir), c->lna(k1), a.sub[a.nsub]);
            a.G[a.nsub] = sl.grids_cur[gi];
            ++a.nsub;
            if (!last) {
                fill_substep(c, false, 0, 0, true, c->lna(k1), c->lna(k1 + 0.5 * dir), a.sub[a.nsub]);
                a.G[a.nsub] = sl.grids_cur[gi];
                ++a.nsub;
            }
            ++gi;
        } else {
            fill_substep(c, true, c->lna(k0), c->lna(k1), true, c->lna(k0 + 0.5 * dir),
                         last ? c->lna(k1) : c->lna(k1 + 0.5 * dir), a.sub[a.nsub]);
            a.G[a.nsub] = sl.grids_cur[gi++];
            ++a.nsub;
        }
        c->k = k1;
        c->disp += typical_displacement(c, c->lna(k0), c->lna(k1));
    }
    a.drift_series = 1;
    for (int u = 0; u < a.nsub; ++u) {
        if (a.sub[u].emax > kSeriesMaxE) a.drift_series = 0;
        if (!a.sub[u].wide_ok) a.wide_series = 0;
    }
    const int form = form_of(c->p.precision);
    if ((form == kWide && !a.wide_series) || (form == kFixed && !a.drift_series) || form == kPlain)
        c->pass_series = 0;
    ++c->pass_count;
    c->pass_steps = std::max(c->pass_steps, pass_len(c, j));
    // the context's stream waits for the pass's grids
    for (int b : sl.bufs_cur) {
        int rc = acquire_grid(c, b);
        if (rc) return rc;
    }
    return FDF_OK;
}

int slice_done(fdf_ctx* c)
{
    auto& sl = c->slice;
    for (int b : sl.bufs_cur) {
        int rc = release_grid(c, b);
        if (rc) return rc;
    }
    if (sl.j + 1 < sl.passes) {
        int rc = maybe_sort(c, (c->k - sl.k_start) * sl.dir, sl.dir);
        if (rc) return rc;
    }
    std::swap(sl.bufs_cur, sl.bufs_next);
    std::swap(sl.grids_cur, sl.grids_next);
    if (++sl.j == sl.passes) {
        sl.active = false;
        return join_fields(c);
    }
    return FDF_OK;
}

const ParticleState& ctx_state(const fdf_ctx* c) { return c->st; }
int ctx_precision(const fdf_ctx* c) { return c->p.precision; }

}  // namespace fdf

extern "C" {

int fdf_sample(fdf_ctx* c)
{
    int rc = sample_enqueue(c);
    if (rc) return rc;
    int flag = 0;
    FDF_CUDA(cudaMemcpyAsync(&flag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "reading flags");
    FDF_CUDA(cudaStreamSynchronize(c->stream), "sampling");
    if (flag) {
        c->sampled = false;
        return fail(FDF_EINVAL, "a direction could not be drawn in 64 attempts");
    }
    return FDF_OK;
}

int fdf_step(fdf_ctx* c, int32_t n)
{
    int rc = slice_begin(c, n);
    while (rc == FDF_OK && slice_active(c)) {
        PushArgs a;
        rc = slice_next(c, a);
        if (!rc) rc = push(c, a);
        if (!rc) rc = slice_done(c);
    }
    return rc;
}

int fdf_run_graph(fdf_ctx* c, int32_t n)
{
    if (!c) return fail(FDF_EINVAL, "ctx is NULL");
    if (n < 0 || n > c->p.n_steps) return fail(FDF_EINVAL, "n must be in [0, n_steps]");
    if (c->timing) return fail(FDF_ESTATE, "fdf_run_graph with fdf_timing on");
    if (c->frozen) return fail(FDF_ESTATE, "fdf_run_graph with frozen fields");
    auto& g = c->graph;
    if (!g.fork) FDF_CUDA(cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming), "creating an event");
    // The legacy default stream cannot be captured: a context on it records and
    // replays its run on a private blocking stream, which the legacy stream orders
    // with everything else.
    if (!c->stream && !g.own) FDF_CUDA(cudaStreamCreate(&g.own), "creating the run's stream");
    struct StreamSwap {
        fdf_ctx* c;
        cudaStream_t saved;
        ~StreamSwap() { c->stream = saved; }
    } swap_back{c, c->stream};
    if (!c->stream) c->stream = g.own;
    if (!g.exec || g.n != n) {
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            g.n = -1;
        }
        // The recorded run depends on nothing outside itself: let everything queued
        // finish, and forget the release events recorded before the capture.
        if (!swap_back.saved) FDF_CUDA(cudaStreamSynchronize(nullptr), "fdf_run_graph");
        FDF_CUDA(cudaStreamSynchronize(c->stream), "fdf_run_graph");
        FDF_CUDA(cudaStreamSynchronize(c->sf), "fdf_run_graph");
        for (int b = 0; b < kMaxBuf; ++b) c->has_release[b] = false;
        const int64_t l0 = c->launches, s0 = c->sorts;
        FDF_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed), "beginning the capture");
        // the fields stream joins the capture through an event of the main stream
        cudaError_t e = cudaEventRecord(g.fork, c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->sf, g.fork, 0);
        int rc = e == cudaSuccess ? sample_enqueue(c) : cuda_fail(e, "forking the fields stream");
        if (rc == FDF_OK && n > 0) rc = fdf_step(c, n);
        if (rc == FDF_OK) rc = join_fields(c);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(c->stream, &graph);
        const int64_t captured = c->launches - l0, sorted = c->sorts - s0;
        c->launches = l0;
        c->sorts = s0;
        if (rc == FDF_OK && e != cudaSuccess) rc = cuda_fail(e, "ending the capture");
        if (rc == FDF_OK) {
            e = cudaGraphInstantiate(&g.exec, graph, 0);
            if (e != cudaSuccess) {
                g.exec = nullptr;
                rc = cuda_fail(e, "instantiating the run's graph");
            }
        }
        if (graph) cudaGraphDestroy(graph);
        if (rc != FDF_OK) {
            // the host state describes a run that never executed
            c->sampled = c->stepped = false;
            for (int b = 0; b < kMaxBuf; ++b) {
                c->gk[b] = -1;
                c->has_release[b] = false;
            }
            c->ssk[0] = c->ssk[1] = -1;
            return rc;
        }
        // the host state the run leaves behind, restored after every replay
        g.n = n;
        std::memcpy(g.gk, c->gk, sizeof(g.gk));
        std::memcpy(g.ssk, c->ssk, sizeof(g.ssk));
        g.slot7 = c->slot7;
        g.k = c->k;
        g.disp = c->disp;
        g.st = c->st;
        g.st_alt = c->st_alt;
        g.launches = captured;
        g.sorts = sorted;
        g.pass_series = c->pass_series;
        g.pass_count = c->pass_count;
        g.pass_steps = c->pass_steps;
    }
    FDF_CUDA(cudaGraphLaunch(g.exec, c->stream), "launching the run's graph");
    // later work on the fields stream follows the run, and the grids the run left in
    // its buffers count as built once it ends (the events recorded inside the graph
    // cannot be waited on from outside it)
    FDF_CUDA(cudaEventRecord(g.fork, c->stream), "recording the run's end");
    FDF_CUDA(cudaStreamWaitEvent(c->sf, g.fork, 0), "ordering the fields stream");
    for (int b = 0; b < c->nbuf; ++b) FDF_CUDA(cudaEventRecord(c->built[b], c->stream), "recording the run's grids");
    std::memcpy(c->gk, g.gk, sizeof(g.gk));
    std::memcpy(c->ssk, g.ssk, sizeof(g.ssk));
    for (int b = 0; b < kMaxBuf; ++b) c->has_release[b] = false;
    c->slot7 = g.slot7;
    c->k = g.k;
    c->disp = g.disp;
    c->st = g.st;
    c->st_alt = g.st_alt;
    c->launches += g.launches;
    c->sorts += g.sorts;
    c->pass_series = g.pass_series;
    c->pass_count = g.pass_count;
    c->pass_steps = g.pass_steps;
    c->noise_ready = true;
    c->sampled = true;
    c->stepped = n > 0;
    // the sampler's failure flag, as fdf_sample reads it
    int flag = 0;
    FDF_CUDA(cudaMemcpyAsync(&flag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "reading flags");
    FDF_CUDA(cudaStreamSynchronize(c->stream), "fdf_run_graph");
    if (flag) {
        c->sampled = false;
        return fail(FDF_EINVAL, "a direction could not be drawn in 64 attempts");
    }
    return FDF_OK;
}

int fdf_get(fdf_ctx* c, int32_t species, double* x, double* q, double* w, int32_t out_on_device)
{
    if (!c) return fail(FDF_EINVAL, "ctx is NULL");
    if (!c->sampled) return fail(FDF_ESTATE, "fdf_get before fdf_sample");
    if (species < 0 || species >= c->p.n_species) return fail(FDF_EINVAL, "species out of range");
    const int64_t np = c->p.n_part;
    if (np == 0) return FDF_OK;
    const int64_t begin = species * np;
    // Host buffers that are page-locked and mapped into the device's address space are
    // written by the export kernel itself (over the CPU-GPU link); others go through
    // the staging buffer and a copy each.
    bool direct = out_on_device != 0;
    double *xm = x, *qm = q, *wm = w;
    if (!direct) {
        direct = true;
        for (double** ptr : {&xm, &qm, &wm}) {
            if (!*ptr) continue;
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, *ptr) != cudaSuccess || at.type != cudaMemoryTypeHost ||
                !at.devicePointer) {
                cudaGetLastError();
                direct = false;
                break;
            }
            *ptr = (double*)at.devicePointer;
        }
    }
    double* xs = direct ? xm : (x ? c->stage : nullptr);
    double* qs = direct ? qm : (q ? c->stage + 3 * np : nullptr);
    double* ws = direct ? wm : (w ? c->stage + 6 * np : nullptr);
    // a sorted state leaves id order: go through the sort's record buffer
    int rc = timed(c, FDF_K_OTHER, "export", [&] {
        if (c->sorts > 0 && c->recs)
            return launch_export_records(c->stream, c->p.precision, c->st, c->n, begin, np, c->p.box_mpc, c->T_ev,
                                         c->recs, xs, qs, ws);
        return launch_export(c->stream, c->p.precision, c->st, c->n, begin, np, c->p.box_mpc, c->T_ev, xs, qs, ws);
    });
    if (rc) return rc;
    if (!direct) {
        if (x) FDF_CUDA(cudaMemcpyAsync(x, xs, 3 * np * 8, cudaMemcpyDeviceToHost, c->stream), "copy x");
        if (q) FDF_CUDA(cudaMemcpyAsync(q, qs, 3 * np * 8, cudaMemcpyDeviceToHost, c->stream), "copy q");
        if (w) FDF_CUDA(cudaMemcpyAsync(w, ws, np * 8, cudaMemcpyDeviceToHost, c->stream), "copy w");
    }
    FDF_CUDA(cudaStreamSynchronize(c->stream), "fdf_get");
    return FDF_OK;
}

int fdf_get_initial(fdf_ctx* c, int32_t species, uint32_t* X, double* q_sampled, double* pm, int32_t out_on_device)
{
    if (!c) return fail(FDF_EINVAL, "ctx is NULL");
    if (!c->sampled || c->stepped) return fail(FDF_ESTATE, "valid between fdf_sample and the first fdf_step");
    if (species < 0 || species >= c->p.n_species) return fail(FDF_EINVAL, "species out of range");
    const int64_t np = c->p.n_part, n = c->n, begin = species * np;
    if (np == 0) return FDF_OK;
    // positions and |q_sampled| follow the particle permutation: un-permute by id
    uint32_t* Xs = out_on_device ? X : (X ? (uint32_t*)c->stage : nullptr);
    double* ps = out_on_device ? pm : (pm ? c->stage + 2 * np : nullptr);
    double* qss = out_on_device ? q_sampled : (q_sampled ? c->stage + 3 * np : nullptr);
    int rc = timed(c, FDF_K_OTHER, "export initial", [&] {
        return launch_export_initial(c->stream, c->p.precision, c->st, n, begin, np, Xs, ps, qss);
    });
    if (rc) return rc;
    if (!out_on_device) {
        if (X) FDF_CUDA(cudaMemcpyAsync(X, Xs, 3 * np * 4, cudaMemcpyDeviceToHost, c->stream), "copy X");
        if (pm) FDF_CUDA(cudaMemcpyAsync(pm, ps, np * 8, cudaMemcpyDeviceToHost, c->stream), "copy p");
        if (q_sampled)
            FDF_CUDA(cudaMemcpyAsync(q_sampled, qss, 3 * np * 8, cudaMemcpyDeviceToHost, c->stream), "copy q_sampled");
    }
    FDF_CUDA(cudaStreamSynchronize(c->stream), "fdf_get_initial");
    return FDF_OK;
}

}  // extern "C"

namespace fdf {

// The deposit into device memory, enqueued on the context's stream without
// waiting for it (fdf_deposit with out_on_device, minus its synchronisation).
int deposit_enqueue(fdf_ctx* c, int32_t species, int32_t quantity, int32_t parity, double* out_dev)
{
    if (!c) return fail(FDF_EINVAL, "ctx is NULL");
    if (!c->sampled) return fail(FDF_ESTATE, "fdf_deposit before fdf_sample");
    if (species < -1 || species >= c->p.n_species) return fail(FDF_EINVAL, "species out of range");
    if (quantity < FDF_Q_W_EPS || quantity > FDF_Q_W_QZ) return fail(FDF_EINVAL, "unknown quantity");
    if (parity < -1 || parity > 1) return fail(FDF_EINVAL, "parity must be -1, 0 or 1");
    if (!out_dev) return fail(FDF_EINVAL, "out is NULL");
    const size_t N3 = (size_t)c->p.n_grid * c->p.n_grid * c->p.n_grid;
    FDF_CUDA(cudaMemsetAsync(out_dev, 0, N3 * 8, c->stream), "clearing the deposit grid");
    const int64_t np = c->p.n_part;
    const int64_t begin = species < 0 ? 0 : species * np;
    const int64_t count = species < 0 ? c->n : np;
    const double a = std::exp(c->lna(c->k));
    return timed(c, FDF_K_OTHER, "deposit", [&] {
        return launch_deposit(c->stream, c->p.precision, c->st, c->n, begin, count, np > 0 ? np : 1, c->p.m_ev, a,
                              c->T_ev, quantity, parity, c->p.interp_order == 2 ? 2 : 1, c->p.n_grid,
                              c->p.box_mpc, c->p.deposit_presum > 0, out_dev);
    });
}

double* ctx_deposit_grid(fdf_ctx* c) { return c->dep; }

}  // namespace fdf

extern "C" {

int fdf_deposit(fdf_ctx* c, int32_t species, int32_t quantity, double* out, int32_t out_on_device)
{
    return fdf_deposit_subset(c, species, quantity, -1, out, out_on_device);
}

int fdf_accel_terms(fdf_ctx* c, int32_t species, double* rms)
{
    if (!c) return fail(FDF_EINVAL, "ctx is NULL");
    if (!rms) return fail(FDF_EINVAL, "rms is NULL");
    if (!c->sampled) return fail(FDF_ESTATE, "fdf_accel_terms before fdf_sample");
    if (species < -1 || species >= c->p.n_species) return fail(FDF_EINVAL, "species out of range");
    for (int j = 0; j < 5; ++j) rms[j] = 0.0;
    const int64_t np = c->p.n_part;
    const int64_t begin = species < 0 ? 0 : species * np, count = species < 0 ? c->n : np;
    if (count == 0) return FDF_OK;
    // the fields of the current step (a buffer already holding them, or a build)
    const void* G = nullptr;
    int b = -1;
    int rc = ensure_grid(c, c->k, 0u, &G, &b);
    if (rc) return rc;
    rc = acquire_grid(c, b);
    if (rc) return rc;
    double* sums = c->stage;             // 5 doubles of the staging area (>= 7 n_part doubles)
    FDF_CUDA(cudaMemsetAsync(sums, 0, 5 * sizeof(double), c->stream), "clearing the sums");
    rc = timed(c, FDF_K_OTHER, "acceleration terms", [&] {
        return launch_accel_terms(c->stream, c->p.precision, c->st, c->n, begin, count, np, c->p.m_ev,
                                  std::exp(c->lna(c->k)), c->p.interp_order == 2 ? 2 : 1, c->p.n_grid,
                                  c->p.box_mpc, G, sums);
    });
    if (rc) return rc;
    rc = release_grid(c, b);
    if (rc) return rc;
    double h[5];
    FDF_CUDA(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "reading the sums");
    FDF_CUDA(cudaStreamSynchronize(c->stream), "fdf_accel_terms");
    for (int j = 0; j < 5; ++j) rms[j] = std::sqrt(h[j] / (double)count);
    return FDF_OK;
}

int fdf_deposit_subset(fdf_ctx* c, int32_t species, int32_t quantity, int32_t parity, double* out,
                       int32_t out_on_device)
{
    if (!c) return fail(FDF_EINVAL, "ctx is NULL");
    if (!c->sampled) return fail(FDF_ESTATE, "fdf_deposit before fdf_sample");
    if (!out) return fail(FDF_EINVAL, "out is NULL");
    const size_t N3 = (size_t)c->p.n_grid * c->p.n_grid * c->p.n_grid;
    double* grid = out_on_device ? out : c->dep;
    int rc = deposit_enqueue(c, species, quantity, parity, grid);
    if (rc) return rc;
    if (!out_on_device)
        FDF_CUDA(cudaMemcpyAsync(out, grid, N3 * 8, cudaMemcpyDeviceToHost, c->stream), "copy deposit");
    FDF_CUDA(cudaStreamSynchronize(c->stream), "fdf_deposit");
    return FDF_OK;
}

int fdf_build_fields(fdf_ctx* c, double lna, double* out, int32_t out_on_device)
{
    if (!c) return fail(FDF_EINVAL, "ctx is NULL");
    if (!out || !std::isfinite(lna)) return fail(FDF_EINVAL, "bad arguments");
    const int N = c->p.n_grid;
    const size_t N3 = (size_t)N * N * N;
    FDF_CUDA(cudaStreamSynchronize(c->sf), "fdf_build_fields");
    FDF_CUDA(cudaStreamSynchronize(c->stream), "fdf_build_fields");
    int buf = 0;
    for (int i = 0; i < c->nbuf; ++i)
        if (c->gk[i] != c->k) buf = i;
    c->gk[buf] = -1;
    // slots 0-6 as the steps' passes read them (phi_dot transformed alone), then slot 7 (psi)
    // from a second build, as the initial transform reads it
    double* dst = out;
    if (!out_on_device) FDF_CUDA(cudaMalloc(&dst, 8 * N3 * 8), "allocating the field copy");
    int rc = FDF_OK;
    for (int pass = 0; pass < 2 && rc == FDF_OK; ++pass) {
        rc = build_fields(c, lna, c->G[buf], c->stream, pass == 0 ? kSlot7Zero : kSlot7Psi);
        if (rc) break;
        rc = timed(c, FDF_K_OTHER, "field export", [&] {
            return launch_fields_to_f64(c->stream, grid_prec(c->p.precision), N, c->G[buf], dst,
                                        pass == 0 ? 0x7Fu : 0x80u);
        });
    }
    if (!rc && !out_on_device) {
        cudaError_t e = cudaMemcpyAsync(out, dst, 8 * N3 * 8, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy fields");
    }
    if (!out_on_device) cudaFree(dst);
    if (rc) return rc;
    FDF_CUDA(cudaStreamSynchronize(c->stream), "fdf_build_fields");
    return FDF_OK;
}

int fdf_set_fields(fdf_ctx* c, const double* fields, int32_t on_device)
{
    if (!c) return fail(FDF_EINVAL, "ctx is NULL");
    FDF_CUDA(cudaStreamSynchronize(c->sf), "fdf_set_fields");
    if (!fields) {
        c->frozen = false;
        for (int i = 0; i < kMaxBuf; ++i) c->gk[i] = -1;
        return FDF_OK;
    }
    const int N = c->p.n_grid;
    const size_t N3 = (size_t)N * N * N;
    if (!c->Gfrozen) FDF_CUDA(cudaMalloc(&c->Gfrozen, N3 * grid_bytes_per_cell(c->p.precision)), "allocating");
    const double* src = fields;
    double* tmp = nullptr;
    if (!on_device) {
        FDF_CUDA(cudaMalloc(&tmp, 8 * N3 * 8), "allocating");
        cudaError_t e = cudaMemcpyAsync(tmp, fields, 8 * N3 * 8, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return cuda_fail(e, "copy fields");
        }
        src = tmp;
    }
    int rc = timed(c, FDF_K_OTHER, "field import",
                   [&] { return launch_fields_from_f64(c->stream, grid_prec(c->p.precision), N, src, c->Gfrozen); });
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (tmp) cudaFree(tmp);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "fdf_set_fields");
    c->frozen = true;
    return FDF_OK;
}

int fdf_supersteps(fdf_ctx* c, int32_t* is_super, int32_t len, int32_t* count)
{
    if (!c) return fail(FDF_EINVAL, "ctx is NULL");
    int n = 0;
    for (size_t j = 0; j < c->is_super.size(); ++j) {
        n += c->is_super[j];
        if (is_super && (int64_t)j < len) is_super[j] = c->is_super[j];
    }
    if (count) *count = n;
    return FDF_OK;
}

int fdf_pass_info(fdf_ctx* c, int32_t* info)
{
    if (!c) return fail(FDF_EINVAL, "ctx is NULL");
    if (!info) return fail(FDF_EINVAL, "info is NULL");
    info[0] = form_of(c->p.precision);
    info[1] = c->pass_series;
    info[2] = c->pass_count;
    info[3] = c->pass_steps;
    return FDF_OK;
}

int fdf_state(fdf_ctx* c, int32_t* step, double* lna)
{
    if (!c) return fail(FDF_EINVAL, "ctx is NULL");
    if (step) *step = c->k;
    if (lna) *lna = c->lna(c->k);
    return FDF_OK;
}

int fdf_timing(fdf_ctx* c, int32_t enable)
{
    if (!c) return fail(FDF_EINVAL, "ctx is NULL");
    if (enable) {
        FDF_CUDA(cudaStreamSynchronize(c->stream), "fdf_timing");
        FDF_CUDA(cudaStreamSynchronize(c->sf), "fdf_timing");
        c->marks.clear();
        c->pool_used = 0;
    }
    c->timing = enable != 0;
    return FDF_OK;
}

int fdf_kernel_time(fdf_ctx* c, int32_t which, double* ms, int64_t* launches)
{
    if (!c) return fail(FDF_EINVAL, "ctx is NULL");
    if (which < 0 || which >= FDF_K_COUNT) return fail(FDF_EINVAL, "unknown kernel class");
    FDF_CUDA(cudaStreamSynchronize(c->stream), "fdf_kernel_time");
    FDF_CUDA(cudaStreamSynchronize(c->sf), "fdf_kernel_time");
    double total = 0;
    int64_t cnt = 0;
    for (auto& m : c->marks) {
        if (m.first != which) continue;
        float t = 0;
        FDF_CUDA(cudaEventElapsedTime(&t, m.second.first, m.second.second), "event time");
        total += t;
        ++cnt;
    }
    if (ms) *ms = total;
    if (launches) *launches = cnt;
    return FDF_OK;
}

int64_t fdf_launch_count(const fdf_ctx* c) { return c ? c->launches : 0; }

const char* fdf_error_string(int code)
{
    switch (code) {
        case FDF_OK: return "ok";
        case FDF_EINVAL: return "invalid argument";
        case FDF_ENOMEM: return "out of device memory";
        case FDF_ECUDA: return "CUDA error";
        case FDF_ESTATE: return "call out of order";
        case FDF_ETIMEOUT: return "device wait timed out";
        case FDF_ENAN: return "non-finite value";
        case FDF_ENOSYS: return "not supported";
        default: return "unknown error";
    }
}

const char* fdf_last_error(void) { return g_last_error.c_str(); }

void fdf_destroy(fdf_ctx* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->sf) {
        cudaStreamSynchronize(c->sf);
        cudaStreamDestroy(c->sf);
    }
    for (int i = 0; i < kMaxBuf; ++i) {
        if (c->built[i]) cudaEventDestroy(c->built[i]);
        if (c->released[i]) cudaEventDestroy(c->released[i]);
    }
    if (c->joined) cudaEventDestroy(c->joined);
    if (c->graph.exec) cudaGraphExecDestroy(c->graph.exec);
    if (c->graph.fork) cudaEventDestroy(c->graph.fork);
    if (c->graph.own) cudaStreamDestroy(c->graph.own);
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    if (c->Gfrozen) cudaFree(c->Gfrozen);
    if (c->own_block && c->block) cudaFree(c->block);
    delete c;
}

}  // extern "C"
