// k_sample.cu -- pre-initial particle sampling (Sec. 2.1 of Elbers 2022):
// positions uniform in the periodic box, |q| from the Fermi-Dirac distribution
// fbar(q) = 1/(1 + e^{q/T}) by inversion of its tabulated CDF, and an
// isotropic direction by rejection from the cube.
//
// Every particle is addressed by its global index g (species-major) so the
// draw does not depend on the launch shape.  Philox4x32-10 keyed by the seed
// with counter (g_lo, g_hi, stream, attempt):
//   stream 0: X_c = word c (c = 0, 1, 2); x_c = L X_c / 2^32
//   stream 1: u from words 0,1 (53 bits) -> t = F^{-1}(u) -> |q| = T t
//   streams 2, 3 (attempt a): v = 2 u - 1 from (2: words 0,1), (2: words 2,3),
//     (3: words 0,1); accept 1e-300 < |v|^2 <= 1; n = v / |v|.
// Only correctly rounded IEEE operations are used (explicit _rn intrinsics, so
// no FMA contraction), which makes the result exact and reproducible.
#include "device_math.cuh"

namespace fdf {

// u = m 2^-53 with the 53-bit integer m = (w0 >> 5) 2^26 + (w1 >> 6): the integer is
// formed exactly in 64 bits and converted exactly (m < 2^53), so only one FP64
// conversion and one exact power-of-two scaling are spent (the GPU's FP64 rate is low).
__device__ __forceinline__ uint64_t m53(uint32_t w0, uint32_t w1)
{
    return ((uint64_t)(w0 >> 5) << 26) | (uint64_t)(w1 >> 6);
}

__device__ __forceinline__ double u53(uint32_t w0, uint32_t w1)
{
    return __dmul_rn(__ull2double_rn(m53(w0, w1)), 1.1102230246251565404e-16);  // 2^-53
}

// v = 2u - 1 = (m - 2^52) 2^-52, exact (|m - 2^52| <= 2^52)
__device__ __forceinline__ double v53(uint32_t w0, uint32_t w1)
{
    return __dmul_rn(__ll2double_rn((long long)m53(w0, w1) - (1ll << 52)), 2.220446049250313080847e-16);  // 2^-52
}

__device__ __forceinline__ double fd_inverse(const double* __restrict__ t, const double* __restrict__ F, int n,
                                             double u)
{
    if (u >= F[n - 1]) return t[n - 1];
    // F and u are non-negative, so their IEEE bit patterns order like their values:
    // the bisection compares 64-bit integers instead of FP64 values
    const long long ub = __double_as_longlong(u);
    const long long* Fb = reinterpret_cast<const long long*>(F);
    int lo = 0, hi = n - 1;  // F[lo] <= u < F[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (Fb[mid] <= ub) lo = mid;
        else hi = mid;
    }
    const double du = __dsub_rn(u, F[lo]);
    const double dt = __dsub_rn(t[lo + 1], t[lo]);
    const double dF = __dsub_rn(F[lo + 1], F[lo]);
    return __dadd_rn(t[lo], __ddiv_rn(__dmul_rn(du, dt), dF));
}

// Attempt `att` of the direction of particle (g0, g1): v from streams 2 and 3;
// accepted when 1e-300 < |v|^2 <= 1.
__device__ __forceinline__ bool direction_attempt(uint32_t g0, uint32_t g1, uint32_t att, uint32_t key0, uint32_t key1,
                                                  double& v0, double& v1, double& v2, double& r2)
{
    const uint4 a = philox4x32_10(make_uint4(g0, g1, 2u, att), key0, key1);
    const uint4 b = philox4x32_10(make_uint4(g0, g1, 3u, att), key0, key1);
    v0 = v53(a.x, a.y);
    v1 = v53(a.z, a.w);
    v2 = v53(b.x, b.y);
    r2 = __dadd_rn(__dadd_rn(__dmul_rn(v0, v0), __dmul_rn(v1, v1)), __dmul_rn(v2, v2));
    return (r2 > 1e-300) && (r2 <= 1.0);
}

constexpr uint32_t kMaxAttempts = 64;

// The directions of a warp's particles, the whole warp working on every round.  A
// particle's direction is its lowest accepted attempt (at most kMaxAttempts), as a
// loop over its attempts would find; but instead of each lane looping until the
// warp's unluckiest lane accepts, every round spreads the attempts of the particles
// still pending over all 32 lanes: with np pending, lane l tries attempt
// next + l / np of the (l mod np)-th pending particle.  Lanes without a particle
// (live = false) only help.  Returns whether this lane's particle got a direction.
__device__ bool warp_direction(bool live, uint32_t g0, uint32_t g1, uint32_t key0, uint32_t key1, double& v0,
                               double& v1, double& v2, double& r2)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned pending = __ballot_sync(full, live);
    uint32_t next = 0;      // the owner's next untried attempt
    bool ok = false;
    while (pending) {
        const int np = __popc(pending);
        const int k = lane % np, rep = lane / np;
        unsigned m = pending;                              // the k-th pending lane
        for (int j = 0; j < k; ++j) m &= m - 1u;
        const int owner = __ffs(m) - 1;
        const uint32_t og0 = __shfl_sync(full, g0, owner), og1 = __shfl_sync(full, g1, owner);
        const uint32_t att = __shfl_sync(full, next, owner) + (uint32_t)rep;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, ar2 = 0.0;
        const bool acc = att < kMaxAttempts && direction_attempt(og0, og1, att, key0, key1, a0, a1, a2, ar2);
        const unsigned accepted = __ballot_sync(full, acc);
        // an owner's lanes are its rank r + j np, j = 0, 1, ...: the lowest accepted one wins
        const bool mine = (pending >> lane) & 1u;
        const int r = mine ? __popc(pending & ((1u << lane) - 1u)) : 0;
        unsigned lanes = 0u;
        if (mine)
            for (int l = r; l < 32; l += np) lanes |= 1u << l;
        const int win = mine ? __ffs(accepted & lanes) - 1 : -1;
        const int src = win >= 0 ? win : lane;
        const double w0 = __shfl_sync(full, a0, src), w1 = __shfl_sync(full, a1, src);
        const double w2 = __shfl_sync(full, a2, src), wr2 = __shfl_sync(full, ar2, src);
        bool done = false;
        if (mine) {
            if (win >= 0) {
                v0 = w0;
                v1 = w1;
                v2 = w2;
                r2 = wr2;
                ok = true;
                done = true;
            } else {
                next += (uint32_t)__popc(lanes);
                done = next >= kMaxAttempts;
            }
        }
        pending &= ~__ballot_sync(full, done);
    }
    return ok;
}

__global__ void __launch_bounds__(256) k_sample(int64_t n, uint32_t key0, uint32_t key1, double T_ev,
                                                const double* __restrict__ cdf_t, const double* __restrict__ cdf_F,
                                                int ncdf, uint32_t* __restrict__ X, double* __restrict__ qs,
                                                double* __restrict__ pmag, uint32_t* __restrict__ id, int* flag)
{
    // warp-uniform trip count: every lane takes part in the warp's direction rounds
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < n; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        const bool live = i < n;
        const uint32_t g0 = (uint32_t)i, g1 = (uint32_t)((uint64_t)i >> 32);
        double v0 = 0.0, v1 = 0.0, v2 = 0.0, r2 = 0.0;
        bool ok = warp_direction(live, g0, g1, key0, key1, v0, v1, v2, r2);
        if (!live) continue;
        uint4 w = philox4x32_10(make_uint4(g0, g1, 0u, 0u), key0, key1);
        X[i] = w.x;
        X[n + i] = w.y;
        X[2 * n + i] = w.z;
        w = philox4x32_10(make_uint4(g0, g1, 1u, 0u), key0, key1);
        const double qmag = __dmul_rn(T_ev, fd_inverse(cdf_t, cdf_F, ncdf, u53(w.x, w.y)));
        if (!ok) {
            atomicOr(flag, 1);
            r2 = 1.0;
            v0 = 1.0;
            v1 = v2 = 0.0;
        }
        const double s = __dsqrt_rn(r2);
        const double q0 = __dmul_rn(qmag, __ddiv_rn(v0, s));
        const double q1 = __dmul_rn(qmag, __ddiv_rn(v1, s));
        const double q2 = __dmul_rn(qmag, __ddiv_rn(v2, s));
        qs[i] = q0;
        qs[n + i] = q1;
        qs[2 * n + i] = q2;
        pmag[i] = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(q0, q0), __dmul_rn(q1, q1)), __dmul_rn(q2, q2)));
        id[i] = (uint32_t)i;
    }
}

cudaError_t launch_sample(cudaStream_t s, int64_t n, uint32_t key0, uint32_t key1, double T_ev, const double* cdf_t,
                          const double* cdf_F, int ncdf, uint32_t* X, double* qs, double* pmag, uint32_t* id,
                          int* flag)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_sample<<<(unsigned)blocks, 256, 0, s>>>(n, key0, key1, T_ev, cdf_t, cdf_F, ncdf, X, qs, pmag, id, flag);
    return cudaGetLastError();
}

}  // namespace fdf
